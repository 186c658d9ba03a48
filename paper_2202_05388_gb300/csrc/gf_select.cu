// Reduction of the candidate dFOM array to the accepted candidate ids (Sec. III: the
// CombineGlobally stage that emits a single proposal V*; Sec. V for the top-k variant).
// The arrays are small (one FP64 per candidate), so one CTA sweeps them with warp-shuffle
// (value, id) reductions and writes the result and the device status word.
#include <math.h>

#include "gf_internal.cuh"

namespace gf {

constexpr int kSelThreads = 1024;

// (v, id) ordering: larger v first, then smaller id.  NaN never wins.
__device__ __forceinline__ bool better(double v, int64_t id, double bv, int64_t bid) {
  return v > bv || (v == bv && id < bid);
}

__device__ void block_best(double& v, int64_t& id) {
  __shared__ double sv[32];
  __shared__ int64_t si[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_down_sync(0xffffffffu, v, o);
    int64_t oi = __shfl_down_sync(0xffffffffu, id, o);
    if (better(ov, oi, v, id)) { v = ov; id = oi; }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { sv[w] = v; si[w] = id; }
  __syncthreads();
  if (w == 0) {
    v = l < (int)(blockDim.x >> 5) ? sv[l] : -INFINITY;
    id = l < (int)(blockDim.x >> 5) ? si[l] : INT64_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_down_sync(0xffffffffu, v, o);
      int64_t oi = __shfl_down_sync(0xffffffffu, id, o);
      if (better(ov, oi, v, id)) { v = ov; id = oi; }
    }
    if (l == 0) { sv[0] = v; si[0] = id; }
  }
  __syncthreads();
  v = sv[0];
  id = si[0];
  __syncthreads();
}

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

// Greedy policy: m = max dfom; lowest id with dfom >= m - tie_rel |m|.
__global__ void __launch_bounds__(kSelThreads) k_select_best(const double* __restrict__ dfom, int64_t ncand,
                                                             double tie_rel, int32_t* idx, double* val,
                                                             int32_t* status) {
  double bv = -INFINITY;
  int64_t bid = INT64_MAX;
  for (int64_t c = threadIdx.x; c < ncand; c += blockDim.x) {
    double v = dfom[c];
    if (better(v, c, bv, bid)) { bv = v; bid = c; }
  }
  block_best(bv, bid);
  const double m = bv;
  if (!(m > 0.0)) {
    if (threadIdx.x == 0) { idx[0] = -1; val[0] = m; *status = GF_ENOIMPROVE; }
    return;
  }
  const double thr = m - tie_rel * fabs(m);
  int64_t first = INT64_MAX;
  for (int64_t c = threadIdx.x; c < ncand && c < first; c += blockDim.x) {
    if (dfom[c] >= thr) first = c;
  }
  double dummy = 0.0;
  block_best(dummy, first);    // all values equal: picks the smallest id
  if (threadIdx.x == 0) {
    idx[0] = (int32_t)first;
    val[0] = dfom[first];
    *status = GF_OK;
  }
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

void launch_select(const gf_geom& g, const gf_cand_spec& spec, const double* dfom, int64_t ncand,
                   int32_t* idx, double* val, int32_t* status, void* ws, cudaStream_t st) {
  (void)ws;
  if (spec.k <= 1)
    k_select_best<<<1, kSelThreads, 0, st>>>(dfom, ncand, spec.tie_rel, idx, val, status);
  else
    k_select_topk<<<1, kSelThreads, 0, st>>>(dfom, ncand, spec.kind, g.nx, g.ny, spec.k,
                                             spec.excl_radius, idx, val, status);
}

}  // namespace gf
