// Reduction of the candidate dFOM array to the accepted candidate ids (Sec. III: the
// CombineGlobally stage that emits a single proposal V*; Sec. V for the top-k variant).
// The arrays are small (one FP64 per candidate): with a workspace, the greedy choice is a pass of
// many CTAs over contiguous chunks and one CTA that finishes it; without one (and for each
// problem of a batch) one CTA sweeps the array.  Comparisons are on integer keys of the doubles.
#include <math.h>

#include <mutex>

#include "gf_internal.cuh"
#include "gf_stage_bodies.cuh"

namespace gf {

constexpr int kSelThreads = 1024;
constexpr int64_t kSelMultiMin = 32768;   // greedy choice over many CTAs from this many candidates

__device__ __forceinline__ void cand_anchor(int64_t c, int kind, int nx, int64_t P, int& ax, int& ay) {
  if (kind == GF_KIND_SINGLE) {
    ay = (int)(c / nx);
    ax = (int)(c - (int64_t)ay * nx);
  } else {
    int64_t a = c % P;
    ay = (int)(a / (nx - 1));
    ax = (int)(a - (int64_t)ay * (nx - 1));
  }
}

__global__ void __launch_bounds__(kSelThreads) k_select_best(const double* __restrict__ dfom, int64_t ncand,
                                                             double tie_rel, int32_t* idx, double* val,
                                                             int32_t* status) {
  select_best_body(dfom, ncand, tie_rel, idx, val, status);
}

// Batched selection: one CTA per problem of the device table.
__global__ void __launch_bounds__(kSelThreads) k_select_best_batch(const BatchItem* __restrict__ items,
                                                                   double tie_rel) {
  batch_select_body(items[blockIdx.x], tie_rel);
}

void launch_select_batch(const BatchItem* items, int nprob, double tie_rel, cudaStream_t st) {
  k_select_best_batch<<<nprob, kSelThreads, 0, st>>>(items, tie_rel);
}

// Top-k with exclusion: repeatedly take the best (dfom, id) candidate that is positive and
// whose anchor is farther than excl_radius (Chebyshev) from every taken anchor.  This equals
// scanning the (-dfom, id)-sorted list and skipping conflicts.
__global__ void __launch_bounds__(kSelThreads) k_select_topk(const double* __restrict__ dfom, int64_t ncand,
                                                             int kind, int nx, int ny, int k, int excl,
                                                             int32_t* idx, double* val, int32_t* status) {
  __shared__ int tax[256], tay[256];
  const int64_t P = (int64_t)(nx - 1) * (ny - 1);
  int ntaken = 0;
  for (int t = 0; t < k; ++t) {
    double bv = -INFINITY;
    int64_t bid = INT64_MAX;
    for (int64_t c = threadIdx.x; c < ncand; c += blockDim.x) {
      double v = dfom[c];
      if (!(v > 0.0) || !better(v, c, bv, bid)) continue;
      int ax, ay;
      cand_anchor(c, kind, nx, P, ax, ay);
      bool clash = false;
      for (int q = 0; q < ntaken && !clash; ++q) {
        int ddx = ax - tax[q], ddy = ay - tay[q];
        clash = max(abs(ddx), abs(ddy)) <= excl;
      }
      if (!clash) { bv = v; bid = c; }
    }
    block_best(bv, bid);
    if (!(bv > 0.0)) break;
    if (threadIdx.x == 0) {
      int ax, ay;
      cand_anchor(bid, kind, nx, P, ax, ay);
      tax[t] = ax;
      tay[t] = ay;
      idx[t] = (int32_t)bid;
      val[t] = bv;
    }
    __syncthreads();
    ntaken = t + 1;
  }
  if (threadIdx.x == 0) {
    for (int t = ntaken; t < k; ++t) { idx[t] = -1; val[t] = -INFINITY; }
    *status = ntaken > 0 ? GF_OK : GF_ENOIMPROVE;
  }
}

// ---- multi-CTA top-k with exclusion: k passes; in pass t every CTA finds its best improving
// candidate that conflicts with none of the t already taken (with excl < 0 a candidate only
// conflicts with itself), and the last CTA to finish (atomic ticket after a memory fence -- no
// CTA waits for another) reduces the per-CTA results and appends the winner.  Exactly the
// sorted-scan result.
struct TopkScratch {
  int32_t counter;      // CTAs finished in the current pass
  int32_t ntaken;
  int32_t done;         // no improving, non-conflicting candidate is left
  int32_t pad;
  uint32_t arrive;      // one-launch form: arrivals at its grid barriers (monotonic)
  int32_t err;          // one-launch form: a barrier wait gave up
  int32_t ax[256], ay[256];
};
constexpr int kTopkBlocks = 148;
constexpr int kTopkThreads = 256;

__global__ void __launch_bounds__(kTopkThreads) k_topk_pass(const double* __restrict__ dfom, int64_t ncand,
                                                           int kind, int nx, int ny, int excl, int pass,
                                                           TopkScratch* sc, double* part_v, int64_t* part_i,
                                                           int32_t* idx, double* val) {
  if (sc->done) return;
  __shared__ int tax[256], tay[256];
  __shared__ bool s_last;
  const int nt = pass;
  for (int q = threadIdx.x; q < nt; q += blockDim.x) { tax[q] = sc->ax[q]; tay[q] = sc->ay[q]; }
  __syncthreads();
  const int64_t P = (int64_t)(nx - 1) * (ny - 1);
  double bv = -INFINITY;
  int64_t bid = INT64_MAX;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncand; c += (int64_t)gridDim.x * blockDim.x) {
    const double v = dfom[c];
    if (!(v > 0.0) || !better(v, c, bv, bid)) continue;
    bool clash = false;
    if (excl < 0) {
      // no exclusion zone: only the candidates already taken are skipped (tax holds their ids)
      for (int q = 0; q < nt && !clash; ++q) clash = c == (int64_t)tax[q];
    } else {
      int ax, ay;
      cand_anchor(c, kind, nx, P, ax, ay);
      for (int q = 0; q < nt && !clash; ++q) clash = max(abs(ax - tax[q]), abs(ay - tay[q])) <= excl;
    }
    if (!clash) { bv = v; bid = c; }
  }
  block_best(bv, bid);
  if (threadIdx.x == 0) {
    part_v[blockIdx.x] = bv;
    part_i[blockIdx.x] = bid;
    __threadfence();
    const int ticket = atomicAdd(&sc->counter, 1);
    s_last = ticket == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double v = -INFINITY;
  int64_t id = INT64_MAX;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const double pv = ((volatile double*)part_v)[b];
    const int64_t pi = ((volatile int64_t*)part_i)[b];
    if (better(pv, pi, v, id)) { v = pv; id = pi; }
  }
  block_best(v, id);
  if (threadIdx.x == 0) {
    if (v > 0.0) {
      int ax, ay;
      cand_anchor(id, kind, nx, P, ax, ay);
      sc->ax[nt] = excl < 0 ? (int32_t)id : ax;
      sc->ay[nt] = ay;
      idx[nt] = (int32_t)id;
      val[nt] = v;
      sc->ntaken = nt + 1;
    } else {
      sc->done = 1;
    }
    sc->counter = 0;
  }
}

__global__ void k_topk_begin(TopkScratch* sc) {
  sc->counter = 0;
  sc->ntaken = 0;
  sc->done = 0;
  sc->arrive = 0u;
  sc->err = 0;
}

__global__ void k_topk_end(const TopkScratch* sc, int k, int32_t* idx, double* val, int32_t* status) {
  const int nt = sc->err ? 0 : sc->ntaken;
  for (int t = nt + threadIdx.x; t < k; t += blockDim.x) {
    idx[t] = -1;
    val[t] = -INFINITY;
  }
  if (threadIdx.x == 0) *status = sc->err ? GF_ETIMEOUT : (nt > 0 ? GF_OK : GF_ENOIMPROVE);
}

// ---- the same passes in one cooperative launch ----------------------------------------------
// CTA b keeps the best valid candidate of its chunk [b chunk, (b + 1) chunk) -- dFOM > 0, not
// taken, outside every exclusion zone (excl < 0: only the taken ids are skipped).  A pass
// publishes every CTA's best (double-buffered by pass parity), meets at a grid barrier, and every
// CTA reduces the same nb entries to the same winner; then only a CTA whose best is the winner or
// lies in the winner's zone scans its chunk again: a zone only removes candidates, so every other
// CTA's best is still its chunk's best.  The winners are those of the passes of k_topk_pass, in
// the same order.  The barrier is a monotonic arrival count with a bounded wait: a wait that gives
// up sets the error word, every CTA leaves at its next barrier, and k_topk_end reports
// GF_ETIMEOUT.  The cooperative launch guarantees that all CTAs are resident together.
constexpr uint64_t kTopkWaitNs = 2000000000ull;

__device__ __forceinline__ uint64_t topk_clock() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// the best valid candidate of [c0, c1) in every thread of the CTA (key LLONG_MIN: none)
__device__ __forceinline__ void topk_chunk_best(const double* __restrict__ dfom, int64_t c0, int64_t c1, int kind,
                                                int nx, int64_t P, int excl, int nt, const int* tax, const int* tay,
                                                long long& bk, int64_t& bid) {
  bk = LLONG_MIN;
  bid = INT64_MAX;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const double v = dfom[c];
    if (!(v > 0.0)) continue;
    const long long kc = ord_key(v);
    if (!(kc > bk || (kc == bk && c < bid))) continue;
    bool clash = false;
    if (excl < 0) {
      for (int q = 0; q < nt && !clash; ++q) clash = c == (int64_t)tax[q];
    } else {
      int ax, ay;
      cand_anchor(c, kind, nx, P, ax, ay);
      for (int q = 0; q < nt && !clash; ++q) clash = max(abs(ax - tax[q]), abs(ay - tay[q])) <= excl;
    }
    if (!clash) { bk = kc; bid = c; }
  }
  block_best_key(bk, bid);
}

__global__ void __launch_bounds__(kTopkThreads) k_topk_coop(const double* __restrict__ dfom, int64_t ncand,
                                                           int64_t chunk, int kind, int nx, int ny, int excl, int k,
                                                           TopkScratch* sc, long long* pk, int64_t* pi,
                                                           int32_t* idx, double* val, uint32_t extra,
                                                           uint64_t wait_ns) {
  // extra: arrivals a barrier waits for beyond the grid's (0; the self-test's 1 never comes)
  __shared__ int tax[256], tay[256];
  __shared__ int s_stop;
  const int nb = (int)gridDim.x, b = (int)blockIdx.x;
  const int64_t P = (int64_t)(nx - 1) * (ny - 1);
  const int64_t c0 = b * chunk, c1 = c0 + chunk < ncand ? c0 + chunk : ncand;
  long long bk;
  int64_t bid;
  topk_chunk_best(dfom, c0, c1, kind, nx, P, excl, 0, tax, tay, bk, bid);
  int nt = 0;
  for (int t = 0; t < k; ++t) {
    const int buf = t & 1;
    if (threadIdx.x == 0) {
      pk[buf * nb + b] = bk;
      pi[buf * nb + b] = bid;
      __threadfence();
      atomicAdd(&sc->arrive, 1u);
      const uint32_t target = (uint32_t)nb * (uint32_t)(t + 1) + extra;
      const uint64_t t0 = topk_clock();
      int stop = 0;
      for (;;) {
        uint32_t a;
        asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(a) : "l"(&sc->arrive) : "memory");
        if ((int)(a - target) >= 0) break;
        if (*reinterpret_cast<volatile int32_t*>(&sc->err)) { stop = 1; break; }
        if (topk_clock() - t0 > wait_ns) { atomicExch(&sc->err, 1); stop = 1; break; }
      }
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;
    long long wk = LLONG_MIN;
    int64_t wi = INT64_MAX;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) key_better(__ldcg(pk + buf * nb + q), __ldcg(pi + buf * nb + q), wk, wi);
    block_best_key(wk, wi);
    if (wk == LLONG_MIN) break;                           // nothing valid is left (every CTA)
    int wax, way;
    if (excl < 0) {
      wax = (int)wi;
      way = 0;
    } else {
      cand_anchor(wi, kind, nx, P, wax, way);
    }
    if (threadIdx.x == 0) {
      tax[nt] = wax;
      tay[nt] = way;
      if (b == 0) {
        idx[nt] = (int32_t)wi;
        val[nt] = dfom[wi];
      }
    }
    ++nt;
    __syncthreads();
    bool stale = bid == wi;
    if (!stale && bid != INT64_MAX && excl >= 0) {
      int ax, ay;
      cand_anchor(bid, kind, nx, P, ax, ay);
      stale = max(abs(ax - wax), abs(ay - way)) <= excl;
    }
    if (stale) topk_chunk_best(dfom, c0, c1, kind, nx, P, excl, nt, tax, tay, bk, bid);
  }
  if (b == 0 && threadIdx.x == 0) sc->ntaken = nt;
}

// scratch: TopkScratch | per-CTA partials | the one-launch form's bests (two buffers) | the
// explore list of the epsilon-greedy policy
static size_t topk_part_off() { return (sizeof(TopkScratch) + 63) & ~size_t(63); }
static size_t topk_coop_off() { return topk_part_off() + kTopkBlocks * (sizeof(double) + sizeof(int64_t)); }
static size_t explore_off() { return topk_coop_off() + 2 * kTopkBlocks * (sizeof(long long) + sizeof(int64_t)); }
constexpr int kExploreTop = 4;      // Sec. V: exploration draws among the four best improving actions

size_t topk_scratch_bytes() { return explore_off() + kExploreTop * (sizeof(double) + sizeof(int32_t)) + 64; }

static void launch_topk_passes(const gf_geom& g, int kind, int k, int excl, const double* dfom, int64_t ncand,
                               int32_t* idx, double* val, void* ws, cudaStream_t st) {
  TopkScratch* sc = reinterpret_cast<TopkScratch*>(ws);
  double* part_v = reinterpret_cast<double*>(reinterpret_cast<char*>(ws) + topk_part_off());
  int64_t* part_i = reinterpret_cast<int64_t*>(part_v + kTopkBlocks);
  int64_t blocks = (ncand + kTopkThreads - 1) / kTopkThreads;
  if (blocks > kTopkBlocks) blocks = kTopkBlocks;
  k_topk_begin<<<1, 1, 0, st>>>(sc);
  // one cooperative launch where the device can hold every CTA at once (checked once per device)
  static std::mutex mu;
  static int coop_of[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int coop = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64) {
      if (coop_of[dev] == 0) {
        int attr = 0, per_sm = 0, sms = 0;
        cudaDeviceGetAttribute(&attr, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_topk_coop, kTopkThreads, 0);
        coop_of[dev] = (attr && per_sm * sms >= kTopkBlocks) ? 1 : -1;
        cudaGetLastError();
      }
      coop = coop_of[dev] > 0;
    }
  }
  if (coop) {
    const int64_t chunk = (ncand + blocks - 1) / blocks;
    const int nb = (int)((ncand + chunk - 1) / chunk);
    long long* pk = reinterpret_cast<long long*>(reinterpret_cast<char*>(ws) + topk_coop_off());
    int64_t* pi = reinterpret_cast<int64_t*>(pk + 2 * kTopkBlocks);
    int gnx = g.nx, gny = g.ny;
    uint32_t extra = 0;
    uint64_t wait_ns = kTopkWaitNs;
    void* args[] = {(void*)&dfom, (void*)&ncand, (void*)&chunk, (void*)&kind, (void*)&gnx, (void*)&gny, (void*)&excl,
                    (void*)&k, (void*)&sc, (void*)&pk, (void*)&pi, (void*)&idx, (void*)&val, (void*)&extra,
                    (void*)&wait_ns};
    if (cudaLaunchCooperativeKernel((const void*)k_topk_coop, dim3((unsigned)nb), dim3(kTopkThreads), args, 0, st) ==
        cudaSuccess)
      return;
    cudaGetLastError();                                  // refused: the passes below
  }
  for (int t = 0; t < k; ++t)
    k_topk_pass<<<(unsigned)blocks, kTopkThreads, 0, st>>>(dfom, ncand, kind, g.nx, g.ny, excl, t, sc, part_v,
                                                           part_i, idx, val);
}

// epsilon-greedy (Sec. V): the greedy choice is already in idx[0] / val[0] / status; when
// u[0] < epsilon it is replaced by rank floor(u[1] m) of the m <= 4 best improving candidates
// in (-dFOM, id) order.  u: two uniform numbers in [0, 1) drawn by the caller.
__global__ void k_egreedy_pick(const TopkScratch* __restrict__ sc, const int32_t* __restrict__ top_i,
                               const double* __restrict__ top_v, double epsilon, const double* __restrict__ u,
                               int32_t* idx, double* val, const int32_t* __restrict__ status) {
  if (threadIdx.x != 0 || *status != GF_OK) return;
  const int m = sc->ntaken < kExploreTop ? sc->ntaken : kExploreTop;
  if (m < 1 || !(u[0] < epsilon)) return;
  int r = (int)(u[1] * (double)m);
  if (r > m - 1) r = m - 1;
  if (r < 0) r = 0;
  idx[0] = top_i[r];
  val[0] = top_v[r];
}

void launch_select_egreedy(const gf_geom& g, const gf_cand_spec& spec, const double* dfom, int64_t ncand,
                           double epsilon, const double* u, int32_t* idx, double* val, int32_t* status, void* ws,
                           cudaStream_t st) {
  k_select_best<<<1, kSelThreads, 0, st>>>(dfom, ncand, spec.tie_rel, idx, val, status);
  int32_t* top_i = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(ws) + explore_off());
  double* top_v = reinterpret_cast<double*>(reinterpret_cast<char*>(ws) + explore_off() + 64);
  launch_topk_passes(g, spec.kind, kExploreTop, -1, dfom, ncand, top_i, top_v, ws, st);   // no exclusion
  k_egreedy_pick<<<1, 32, 0, st>>>(reinterpret_cast<const TopkScratch*>(ws), top_i, top_v, epsilon, u, idx, val,
                                   status);
}

// The greedy choice over many CTAs: CTA b takes the contiguous chunk [b chunk, (b + 1) chunk)
// and writes its best (key, id); the finishing CTA reduces those to the maximum m, and the lowest
// id with dfom >= m - tie_rel |m| lies in the first chunk whose best reaches that threshold (the
// chunks before it hold nothing that does), so only that chunk is scanned again.  The same ids
// and values as select_best_body.
__global__ void __launch_bounds__(256) k_select_part(const double* __restrict__ dfom, int64_t ncand, int64_t chunk,
                                                     long long* __restrict__ pk, int64_t* __restrict__ pi) {
  const int64_t c0 = blockIdx.x * chunk, c1 = c0 + chunk < ncand ? c0 + chunk : ncand;
  long long bk = ord_key(-INFINITY);
  int64_t bid = INT64_MAX;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) key_better(ord_key(dfom[c]), c, bk, bid);
  block_best_key(bk, bid);
  if (threadIdx.x == 0) {
    pk[blockIdx.x] = bk;
    pi[blockIdx.x] = bid;
  }
}

__global__ void __launch_bounds__(256) k_select_finish(const double* __restrict__ dfom, int64_t ncand, int64_t chunk,
                                                       const long long* __restrict__ pk,
                                                       const int64_t* __restrict__ pi, int nb, double tie_rel,
                                                       int32_t* idx, double* val, int32_t* status) {
  long long bk = ord_key(-INFINITY);
  int64_t bid = INT64_MAX;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) key_better(pk[b], pi[b], bk, bid);
  block_best_key(bk, bid);
  const double m = key_value(bk);
  if (!(m > 0.0)) {
    if (threadIdx.x == 0) { idx[0] = -1; val[0] = m; *status = GF_ENOIMPROVE; }
    return;
  }
  double thr = m - tie_rel * fabs(m);
  if (!(thr <= m)) thr = m;                               // m = +inf
  const long long tk = ord_key(thr);
  int64_t fb = INT64_MAX;                                 // the first chunk reaching the threshold
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (pk[b] >= tk && b < fb) fb = b;
  long long same = 0;
  block_best_key(same, fb);
  const int64_t c0 = fb * chunk, c1 = c0 + chunk < ncand ? c0 + chunk : ncand;
  int64_t first = INT64_MAX;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x)
    if (ord_key(dfom[c]) >= tk) { first = c; break; }
  same = 0;
  block_best_key(same, first);
  if (threadIdx.x == 0) {
    idx[0] = (int32_t)first;
    val[0] = dfom[first];
    *status = GF_OK;
  }
}

void launch_select(const gf_geom& g, const gf_cand_spec& spec, const double* dfom, int64_t ncand,
                   int32_t* idx, double* val, int32_t* status, void* ws, cudaStream_t st) {
  if (spec.k <= 1) {
    if (ws == nullptr || ncand < kSelMultiMin) {
      k_select_best<<<1, kSelThreads, 0, st>>>(dfom, ncand, spec.tie_rel, idx, val, status);
      return;
    }
    long long* pk = reinterpret_cast<long long*>(reinterpret_cast<char*>(ws) + topk_part_off());
    int64_t* pi = reinterpret_cast<int64_t*>(pk + kTopkBlocks);
    const int64_t chunk = (ncand + kTopkBlocks - 1) / kTopkBlocks;
    const int nb = (int)((ncand + chunk - 1) / chunk);
    k_select_part<<<nb, 256, 0, st>>>(dfom, ncand, chunk, pk, pi);
    k_select_finish<<<1, 256, 0, st>>>(dfom, ncand, chunk, pk, pi, nb, spec.tie_rel, idx, val, status);
    return;
  }
  if (ws == nullptr) {
    k_select_topk<<<1, kSelThreads, 0, st>>>(dfom, ncand, spec.kind, g.nx, g.ny, spec.k, spec.excl_radius, idx, val,
                                             status);
    return;
  }
  launch_topk_passes(g, spec.kind, spec.k, spec.excl_radius, dfom, ncand, idx, val, ws, st);
  k_topk_end<<<1, 256, 0, st>>>(reinterpret_cast<const TopkScratch*>(ws), spec.k, idx, val, status);
}

// The one-launch top-k with a barrier that waits for one arrival more than the grid gives:
// every CTA's wait runs out after wait_ns and the status word reports GF_ETIMEOUT, without a
// fault.  ws: selection scratch, then 4096 zero dFOM values, 64 ids and 64 values.  False when
// the device cannot launch the cooperative form.
size_t topk_selftest_bytes() { return topk_scratch_bytes() + 4096 * sizeof(double) + 64 * (sizeof(int32_t) + sizeof(double)); }

bool launch_topk_selftest(void* ws, uint64_t wait_ns, int32_t* status, cudaStream_t st) {
  int dev = 0, attr = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&attr, cudaDevAttrCooperativeLaunch, dev);
  if (!attr) return false;
  char* base = reinterpret_cast<char*>(ws);
  TopkScratch* sc = reinterpret_cast<TopkScratch*>(base);
  const double* dfom = reinterpret_cast<const double*>(base + topk_scratch_bytes());
  int32_t* idx = reinterpret_cast<int32_t*>(base + topk_scratch_bytes() + 4096 * sizeof(double));
  double* val = reinterpret_cast<double*>(idx + 64);
  cudaMemsetAsync(base + topk_scratch_bytes(), 0, 4096 * sizeof(double), st);
  k_topk_begin<<<1, 1, 0, st>>>(sc);
  int64_t ncand = 4096, chunk = 256;
  int kind = GF_KIND_SINGLE, nx = 64, ny = 64, excl = 0, k = 2;
  long long* pk = reinterpret_cast<long long*>(base + topk_coop_off());
  int64_t* pi = reinterpret_cast<int64_t*>(pk + 2 * kTopkBlocks);
  uint32_t extra = 1;
  void* args[] = {(void*)&dfom, (void*)&ncand, (void*)&chunk, (void*)&kind, (void*)&nx, (void*)&ny, (void*)&excl,
                  (void*)&k, (void*)&sc, (void*)&pk, (void*)&pi, (void*)&idx, (void*)&val, (void*)&extra,
                  (void*)&wait_ns};
  if (cudaLaunchCooperativeKernel((const void*)k_topk_coop, dim3(16), dim3(kTopkThreads), args, 0, st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  k_topk_end<<<1, 256, 0, st>>>(sc, k, idx, val, status);
  return true;
}

}  // namespace gf
