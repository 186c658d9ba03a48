// Reduction of the candidate dFOM array to the accepted candidate ids (Sec. III: the
// CombineGlobally stage that emits a single proposal V*; Sec. V for the top-k variant).
// The arrays are small (one FP64 per candidate): with a workspace, the greedy choice is a pass of
// many CTAs over contiguous chunks and one CTA that finishes it; without one (and for each
// problem of a batch) one CTA sweeps the array.  Comparisons are on integer keys of the doubles.
#include <math.h>

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
}

__global__ void k_topk_end(const TopkScratch* sc, int k, int32_t* idx, double* val, int32_t* status) {
  const int nt = sc->ntaken;
  for (int t = nt + threadIdx.x; t < k; t += blockDim.x) {
    idx[t] = -1;
    val[t] = -INFINITY;
  }
  if (threadIdx.x == 0) *status = nt > 0 ? GF_OK : GF_ENOIMPROVE;
}

// scratch: TopkScratch | per-CTA partials | the explore list of the epsilon-greedy policy
static size_t topk_part_off() { return (sizeof(TopkScratch) + 63) & ~size_t(63); }
static size_t explore_off() { return topk_part_off() + kTopkBlocks * (sizeof(double) + sizeof(int64_t)); }
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

}  // namespace gf
