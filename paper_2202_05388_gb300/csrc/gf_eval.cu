// Exact dFOM of every candidate flip (Sec. II-A, Eqs. 4-9 evaluated at the monitor point,
// FOM of Eq. 1 = sum over wavelengths of |E(r_m)|^2).  Each candidate only needs entries of
// G inside its own pixel set, the field at those pixels and the monitor row of G -- the
// locality the paper's partitioned dFOM stage relies on (Sec. III) -- so one thread owns one
// candidate anchor and reads its inputs from the contiguous band arrays (coalesced across
// neighbouring anchors).
#include <math.h>

#include "gf_internal.cuh"
#include "gf_stage_bodies.cuh"

namespace gf {

__global__ void k_eval_single(EvalArgs a, const uint8_t* __restrict__ state, int dir_mask,
                              double* __restrict__ dfom) {
  eval_single_body(a, state, dir_mask, dfom);
}

__global__ void __launch_bounds__(128) k_eval_brush(EvalArgs a, const uint8_t* __restrict__ state,
                                                    int dir_mask, double* __restrict__ dfom) {
  eval_brush_body(a, state, dir_mask, dfom);
}

// Batched forms: blockIdx.y selects the problem of the device table; the x dimension strides
// over that problem's pixels or anchors exactly as in the single-problem kernels.
__device__ __forceinline__ void batch_eval_args(const BatchItem* items, int dtype, EvalArgs& sa,
                                                const uint8_t*& s_state, double*& s_dfom) {
  if (threadIdx.x == 0) {
    const BatchItem& it = items[blockIdx.y];
    sa.nlam = 1;
    sa.dtype = dtype;
    sa.nx = it.nx;
    sa.ny = it.ny;
    sa.chi = it.chi;
    sa.c_begin = 0;
    sa.c_end = -1;
    sa.lam[0].G = it.G;
    sa.lam[0].ldg = it.ldg;
    sa.lam[0].E = it.E;
    sa.lam[0].bands = it.bands;
    s_state = it.state;
    s_dfom = it.dfom;
  }
  __syncthreads();
}

__global__ void k_eval_single_batch(const BatchItem* __restrict__ items, int dtype, int dir_mask) {
  __shared__ EvalArgs sa;
  __shared__ const uint8_t* s_state;
  __shared__ double* s_dfom;
  batch_eval_args(items, dtype, sa, s_state, s_dfom);
  eval_single_body(sa, s_state, dir_mask, s_dfom);
}

__global__ void __launch_bounds__(128) k_eval_brush_batch(const BatchItem* __restrict__ items, int dtype,
                                                          int dir_mask) {
  __shared__ EvalArgs sa;
  __shared__ const uint8_t* s_state;
  __shared__ double* s_dfom;
  batch_eval_args(items, dtype, sa, s_state, s_dfom);
  eval_brush_body(sa, s_state, dir_mask, s_dfom);
}

void launch_eval_batch(const BatchItem* items, int nprob, int dtype, const gf_cand_spec& spec, int64_t widest,
                       cudaStream_t st) {
  const int threads = spec.kind == GF_KIND_SINGLE ? 256 : 128;
  int64_t b = (widest + threads - 1) / threads;       // widest: pixels (single) or anchors (brush)
  if (b > 1216) b = 1216;
  dim3 grid((unsigned)(b < 1 ? 1 : b), (unsigned)nprob);
  if (spec.kind == GF_KIND_SINGLE)
    k_eval_single_batch<<<grid, threads, 0, st>>>(items, dtype, spec.dir_mask);
  else
    k_eval_brush_batch<<<grid, threads, 0, st>>>(items, dtype, spec.dir_mask | (spec.aligned ? kEvalAligned : 0));
}

void launch_eval(const EvalArgs& a, const uint8_t* state, const gf_cand_spec& spec, double* dfom,
                 cudaStream_t st) {
  const int64_t N = (int64_t)a.nx * a.ny;
  if (spec.kind == GF_KIND_SINGLE) {
    int64_t b = (N + 255) / 256;
    k_eval_single<<<(int)(b < 4864 ? b : 4864), 256, 0, st>>>(a, state, spec.dir_mask, dfom);
  } else {
    const int64_t P = (int64_t)(a.nx - 1) * (a.ny - 1);
    int64_t b = (P + 127) / 128;
    k_eval_brush<<<(int)(b < 9728 ? b : 9728), 128, 0, st>>>(a, state, spec.dir_mask | (spec.aligned ? kEvalAligned : 0),
                                                             dfom);
  }
}

}  // namespace gf
