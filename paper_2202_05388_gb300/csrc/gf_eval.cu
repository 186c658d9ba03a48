// Exact dFOM of every candidate flip (Sec. II-A, Eqs. 4-9 evaluated at the monitor point,
// FOM of Eq. 1 = sum over wavelengths of |E(r_m)|^2).  Each candidate only needs entries of
// G inside its own pixel set, the field at those pixels and the monitor row of G -- the
// locality the paper's partitioned dFOM stage relies on (Sec. III) -- so one thread owns one
// candidate anchor and reads its inputs from the contiguous band arrays (coalesced across
// neighbouring anchors).
#include <math.h>

#include "gf_internal.cuh"

namespace gf {

constexpr int kEvalAligned = 4;    // dir_mask bit set by the launchers: only even anchors

// Solve A y = b for a 4x4 complex system by Gaussian elimination with partial pivoting.
// Rows u with active[u] == false are identity rows with b[u] = 0, which reproduces the
// elimination of the reduced system over the active pixels (same pivots, same arithmetic on
// the active entries).  Returns false when a pivot is zero or below
// kSingularRel * ||A_active||_inf.
template <int P>
__device__ __forceinline__ bool solve_small(cplx (&A)[P][P], cplx (&b)[P], const bool (&active)[P]) {
  double norm = 0.0;
#pragma unroll
  for (int u = 0; u < P; ++u) {
    double s = 0.0;
#pragma unroll
    for (int v = 0; v < P; ++v) s += cabs1(A[u][v]);
    if (active[u]) norm = fmax(norm, s);
  }
  const double thresh = kSingularRel * norm;
  bool ok = true;
#pragma unroll
  for (int c = 0; c < P; ++c) {
    // pivot: first row >= c with the largest modulus
    int r = c;
    double best = cabs1(A[c][c]);
#pragma unroll
    for (int rr = c + 1; rr < P; ++rr) {
      double m = cabs1(A[rr][c]);
      if (m > best) { best = m; r = rr; }
    }
    if (!(best >= thresh) || !(best > 0.0)) ok = false;
#pragma unroll
    for (int rr = c + 1; rr < P; ++rr) {
      if (rr == r) {
#pragma unroll
        for (int v = 0; v < P; ++v) { cplx t = A[c][v]; A[c][v] = A[rr][v]; A[rr][v] = t; }
        cplx t = b[c]; b[c] = b[rr]; b[rr] = t;
      }
    }
    cplx piv = ok ? A[c][c] : mk(1.0, 0.0);
#pragma unroll
    for (int rr = c + 1; rr < P; ++rr) {
      cplx f = cdiv(A[rr][c], piv);
#pragma unroll
      for (int v = c; v < P; ++v) A[rr][v] = A[rr][v] - f * A[c][v];
      b[rr] = b[rr] - f * b[c];
    }
  }
#pragma unroll
  for (int c = P - 1; c >= 0; --c) {
    cplx acc = b[c];
#pragma unroll
    for (int v = c + 1; v < P; ++v) acc = acc - A[c][v] * b[v];
    b[c] = cdiv(acc, ok ? A[c][c] : mk(1.0, 0.0));
  }
  return ok;
}

// Single-pixel candidates: id = j.  p = 1, so Eq. 9 is y = E_j / (1 - G_jj d_chi).
__device__ __forceinline__ void eval_single_body(const EvalArgs& a, const uint8_t* __restrict__ state,
                                                 int dir_mask, double* __restrict__ dfom) {
  const int64_t N = (int64_t)a.nx * a.ny;
  const int64_t jend = a.c_end >= 0 && a.c_end < N ? a.c_end : N;
  for (int64_t j = a.c_begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < jend;
       j += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t s = state[j];
    double d = 0.0;
    if (s == 0 && (dir_mask & GF_DIR_FILL)) d = a.chi;
    if (s != 0 && (dir_mask & GF_DIR_CLEAR)) d = -a.chi;
    double total = 0.0;
    bool valid = d != 0.0;
    for (int l = 0; l < a.nlam && valid; ++l) {
      const EvalLam& L = a.lam[l];
      cplx gjj = L.bands[j];
      cplx Ej = L.E[j];
      cplx EN = L.E[N];
      cplx gNj = ldG(L.G, a.dtype, L.ldg, N, j);
      cplx A = mk(1.0 - gjj.re * d, -gjj.im * d);
      if (!(cabs1(A) > 0.0)) { valid = false; break; }   // 1x1: singular only when zero
      cplx y = cdiv(Ej, A);
      cplx Em = EN + d * (gNj * y);
      total += abs2(Em) - abs2(EN);
    }
    dfom[j] = valid ? total : -INFINITY;
  }
}

// 2x2 brush candidates: id = dir*P + a, anchor a = iy*(nx-1) + ix; pixels
// q0 = (ix,iy), q1 = (ix+1,iy), q2 = (ix,iy+1), q3 = (ix+1,iy+1).  One thread evaluates both
// directions of its anchor.
__device__ __forceinline__ void eval_brush_body(const EvalArgs& a, const uint8_t* __restrict__ state,
                                                int dir_mask, double* __restrict__ dfom) {
  const int nx = a.nx;
  const int64_t N = (int64_t)nx * a.ny;
  const int64_t P = (int64_t)(nx - 1) * (a.ny - 1);
  // local pixel offsets and the band that holds G[q_u, q_v]
  const int px[4] = {0, 1, 0, 1}, py[4] = {0, 0, 1, 1};
  const int band_of[9] = {8, 6, 4, 2, 0, 1, 3, 5, 7};   // index (ddy+1)*3 + (ddx+1)
  const int64_t aend = a.c_end >= 0 && a.c_end < P ? a.c_end : P;
  for (int64_t an = a.c_begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; an < aend;
       an += (int64_t)gridDim.x * blockDim.x) {
    const int ay = (int)(an / (nx - 1)), ax = (int)(an - (int64_t)ay * (nx - 1));
    const int64_t j0 = (int64_t)ay * nx + ax;
    int64_t q[4] = {j0, j0 + 1, j0 + nx, j0 + nx + 1};
    uint8_t s[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) s[u] = state[q[u]];
    double total[2] = {0.0, 0.0};
    bool valid[2];
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      bool any = false;
#pragma unroll
      for (int u = 0; u < 4; ++u) any |= (s[u] == (dir == 0 ? 0 : 1));
      valid[dir] = any && (dir_mask & (dir == 0 ? GF_DIR_FILL : GF_DIR_CLEAR)) &&
                   !((dir_mask & kEvalAligned) && ((ax | ay) & 1));
    }
    for (int l = 0; l < a.nlam; ++l) {
      const EvalLam& L = a.lam[l];
      cplx EN = L.E[N];
#pragma unroll
      for (int dir = 0; dir < 2; ++dir) {
        if (!valid[dir]) continue;
        const double dval = dir == 0 ? a.chi : -a.chi;
        bool act[4];
        double d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          act[u] = s[u] == (dir == 0 ? 0 : 1);
          d[u] = act[u] ? dval : 0.0;
        }
        cplx A[4][4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            int b = band_of[(py[v] - py[u] + 1) * 3 + (px[v] - px[u] + 1)];
            cplx g = L.bands[(int64_t)b * N + q[u]];
            cplx e = mk(u == v ? 1.0 : 0.0, 0.0);
            A[u][v] = act[u] ? e - d[v] * g : e;
          }
          y[u] = act[u] ? L.E[q[u]] : mk(0.0, 0.0);
        }
        if (!solve_small<4>(A, y, act)) { valid[dir] = false; continue; }
        cplx dE = mk(0.0, 0.0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (act[u]) dE = dE + d[u] * (ldG(L.G, a.dtype, L.ldg, N, q[u]) * y[u]);
        }
        cplx Em = EN + dE;
        total[dir] += abs2(Em) - abs2(EN);
      }
    }
    dfom[an] = valid[0] ? total[0] : -INFINITY;
    dfom[P + an] = valid[1] ? total[1] : -INFINITY;
  }
}

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
