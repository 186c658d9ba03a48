// Device bodies of the step's stages (Fig. 1: evaluate, select, capacitance solve, panels, G
// update, field and FOM, bands) that several kernels share: the single-problem kernels, the
// batched per-stage kernels and the persistent batch kernel (which runs them as work items with a
// virtual block index and count).  Included by the translation units that launch them.
// Inputs that a stage of the persistent kernel produces earlier in the same launch (dFOM, the
// workspace, G, E, state) are read through plain pointers, never `const __restrict__` ones: the
// read-only data path is only valid for data that no thread writes during the launch.
#pragma once

#include <limits.h>
#include <math.h>

#include "gf_internal.cuh"

namespace gf {

// ----------------------------------------------------------------------------- operand digits
// of the tensor-core complex128 update (see gf_update_tc.cu)
constexpr int kOzW = 9;            // bits per digit
constexpr int kOzS = 6;            // digits per value
constexpr int kOzLv = 6;           // levels a + b = 2 .. 7
constexpr int kOzK = 8;            // real K (2 p, p <= 4)
constexpr int kOzM = 128;          // rows per tile (TMEM lanes)
constexpr int kOzN = 32;           // real output columns per tile (16 complex)
constexpr int kOzSliceA = kOzM * kOzK * 4;      // bytes of one digit slice of an A tile
constexpr int kOzSliceB = kOzN * kOzK * 4;      // bytes of one digit slice of a B tile
constexpr int kOzTileA = kOzS * kOzSliceA;      // 24 KB
constexpr int kOzTileB = kOzS * kOzSliceB;      // 6 KB
constexpr uint64_t kOzTimeoutNs = 2000000000ull;
constexpr int kOzMaxBatch = kBatchMax;
constexpr int kOzBBlockG = kOzTileB + 64;       // B digit slices + 16 column exponents (global block)

// byte offset of element (r, k) inside one K-major, no-swizzle digit slice (8x16-byte core
// matrices; K-direction core-matrix stride 128 B, row-group stride 256 B)
__host__ __device__ __forceinline__ int oz_off(int r, int k) {
  return (r >> 3) * 256 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

// six signed 9-bit digits of x in (-1, 1): x = sum_a d[a] 2^(-9(a+1)) + r, |r| <= 2^-55
// The digits of x = v 2^-E (|v| < 2^E), six signed digits of kOzW = 9 bits from the top:
// the FP64 sequence d_a = rint(r_a 2^(9(a+1))), r_(a+1) = r_a - d_a 2^(-9(a+1)) (r_0 = x, every
// step exact) restated in integers, since on GB300 each of its FP64 operations, roundings and
// conversions would run on the narrow FP64 pipe, which then bounds the preparation:
// X = x 2^54 rounded to an integer (ties to even), then d_a = X_a / 2^(45 - 9a) rounded to the
// nearest integer (ties to even), X_(a+1) = X_a - d_a 2^(45 - 9a), and the last digit is the
// remainder.  The digits sum to x rounded at 2^-54, as the FP64 sequence's do, within the same
// bounds (|d_0| <= 512, |d_a| <= 256); where the rounding at 2^-54 first makes a digit's
// remainder an exact tie, the two resolve it differently from that digit on (about one value in
// 2000, the same sum).  A CPU model of both is in tests/test_oz_digits_cpu.py.
__device__ __forceinline__ void oz_digits_i(double v, int E, float (&d)[kOzS]) {
  const long long b = __double_as_longlong(v);
  const int ef = (int)((b >> 52) & 0x7FF);
  const long long M = (b & 0x000FFFFFFFFFFFFFll) | (ef ? 0x0010000000000000ll : 0ll);
  const int sh = (ef ? ef : 1) - 1075 + 54 - E;           // v 2^(54 - E) = M 2^sh
  long long X;
  if (sh >= 0) {
    X = M << (sh < 63 ? sh : 63);                         // |v| < 2^E keeps M 2^sh below 2^54
  } else if (sh > -54) {
    const int s = -sh;
    const long long q = M >> s, rem = M & ((1ll << s) - 1), half = 1ll << (s - 1);
    X = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
  } else {
    X = 0;                                                // below half a unit of 2^-54
  }
  if (b < 0) X = -X;
#pragma unroll
  for (int a = 0; a < kOzS - 1; ++a) {
    const int sft = 45 - kOzW * a;
    const long long da = (X + (1ll << (sft - 1)) - 1 + ((X >> sft) & 1)) >> sft;
    d[a] = (float)da;
    X -= da << sft;
  }
  d[kOzS - 1] = (float)X;
}

// The smallest E with m < 2^E for the largest |v| of a row (column), m > 0, given as the bit
// pattern of m (non-negative doubles order as their bit patterns do); 0 for a zero row, whose
// digits are 0 under any exponent
__device__ __forceinline__ int oz_exponent_bits(long long mb) {
  if (mb <= 0) return 0;
  const int ef = (int)(mb >> 52);
  return (ef ? ef - 1023 : (63 - __clzll(mb)) - 1074) + 1;
}
__device__ __forceinline__ long long oz_mag(double v) { return __double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFll; }

// ---- operand preparation (once per step, O(n p) work) --------------------------------------
__device__ __forceinline__ void oz_prep_rows_body(const cplx* C0, int pmax, int64_t n,
                                                  int64_t nrows_pad, const UpdCtl* ctl,
                                                  uint8_t* __restrict__ ozA, int32_t* __restrict__ ozE, int64_t vb = -1, int64_t vg = -1) {
  // vb, vg: a virtual block index and count (a work item of a persistent kernel); -1: the grid's
  const int64_t vb_ = vb < 0 ? (int64_t)blockIdx.x : vb, vg_ = vg < 0 ? (int64_t)gridDim.x : vg;
  if (ctl->skip || ctl->nv > 4) return;
  const int p = ctl->nv;
  for (int64_t i = vb_ * (int64_t)blockDim.x + threadIdx.x; i < nrows_pad;
       i += (int64_t)vg_ * blockDim.x) {
    double v[kOzK];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      cplx c = (i < n && k < p) ? C0[i * pmax + k] : mk(0.0, 0.0);
      v[k] = c.re;
      v[4 + k] = c.im;
    }
    long long mb = 0;
#pragma unroll
    for (int k = 0; k < kOzK; ++k) mb = oz_mag(v[k]) > mb ? oz_mag(v[k]) : mb;
    const int E = oz_exponent_bits(mb);
    ozE[i] = E;
    uint8_t* tile = ozA + (i / kOzM) * (int64_t)kOzTileA;
    const int r = (int)(i % kOzM);
    float dg[kOzK][kOzS];
#pragma unroll
    for (int k = 0; k < kOzK; ++k) oz_digits_i(v[k], E, dg[k]);
#pragma unroll
    for (int a = 0; a < kOzS; ++a) {
      float4* q0 = reinterpret_cast<float4*>(tile + a * kOzSliceA + oz_off(r, 0));
      float4* q1 = reinterpret_cast<float4*>(tile + a * kOzSliceA + oz_off(r, 4));
      *q0 = make_float4(dg[0][a], dg[1][a], dg[2][a], dg[3][a]);
      *q1 = make_float4(dg[4][a], dg[5][a], dg[6][a], dg[7][a]);
    }
  }
}

__device__ __forceinline__ void oz_prep_cols_body(const cplx* S, int64_t n, int64_t ncols_pad,
                                                  const UpdCtl* ctl, uint8_t* __restrict__ ozB, int64_t vb = -1, int64_t vg = -1) {
  // vb, vg: a virtual block index and count (a work item of a persistent kernel); -1: the grid's
  const int64_t vb_ = vb < 0 ? (int64_t)blockIdx.x : vb, vg_ = vg < 0 ? (int64_t)gridDim.x : vg;
  if (ctl->skip || ctl->nv > 4) return;
  const int p = ctl->nv;
  // one thread per complex column j; writes real columns 2j and 2j+1
  for (int64_t j = vb_ * (int64_t)blockDim.x + threadIdx.x; j < ncols_pad;
       j += (int64_t)vg_ * blockDim.x) {
    double sr[4], si[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      cplx s = (j < n && k < p) ? S[(int64_t)k * n + j] : mk(0.0, 0.0);
      sr[k] = s.re;
      si[k] = s.im;
    }
    long long mb = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      mb = oz_mag(sr[k]) > mb ? oz_mag(sr[k]) : mb;
      mb = oz_mag(si[k]) > mb ? oz_mag(si[k]) : mb;
    }
    const int F = oz_exponent_bits(mb);
    float dr[4][kOzS], di[4][kOzS];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      oz_digits_i(sr[k], F, dr[k]);
      oz_digits_i(si[k], F, di[k]);
    }
    const int64_t c_re = 2 * j;
    uint8_t* tile = ozB + (c_re / kOzN) * (int64_t)kOzBBlockG;
    const int c = (int)(c_re % kOzN);            // even; c + 1 is the imaginary column
    reinterpret_cast<int32_t*>(tile + kOzTileB)[c / 2] = F;
#pragma unroll
    for (int a = 0; a < kOzS; ++a) {
      uint8_t* sl = tile + a * kOzSliceB;
      *reinterpret_cast<float4*>(sl + oz_off(c, 0)) = make_float4(dr[0][a], dr[1][a], dr[2][a], dr[3][a]);
      *reinterpret_cast<float4*>(sl + oz_off(c, 4)) = make_float4(-di[0][a], -di[1][a], -di[2][a], -di[3][a]);
      *reinterpret_cast<float4*>(sl + oz_off(c + 1, 0)) = make_float4(di[0][a], di[1][a], di[2][a], di[3][a]);
      *reinterpret_cast<float4*>(sl + oz_off(c + 1, 4)) = make_float4(dr[0][a], dr[1][a], dr[2][a], dr[3][a]);
    }
  }
}


// ----------------------------------------------------------------------------- candidate dFOM
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
  double dinv[P];
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
    dinv[c] = 1.0 / abs2(piv);
#pragma unroll
    for (int rr = c + 1; rr < P; ++rr) {
      cplx f = cdiv_r(A[rr][c], piv, dinv[c]);
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
    b[c] = cdiv_r(acc, ok ? A[c][c] : mk(1.0, 0.0), dinv[c]);
  }
  return ok;
}

// The same elimination with the pivot rule decided without square roots and the arithmetic in
// fused multiply-adds: pivots are searched on |a|^2, and the rule |pivot| >= kSingularRel
// ||A_active||_inf is decided against bounds of the norm (with s = sum of |re| + |im| over a row,
// s / sqrt 2 <= sum |z| <= s, so a pivot clears the rule when |pivot|^2 >= (kSingularRel s_max)^2
// and fails it when |pivot|^2 < (kSingularRel s_max)^2 / 2).  Returns 1 (solved), 0 (singular by
// the rule) or -1 when a pivot falls between the two, where only the exact norm decides: the
// caller then solves the system again with solve_small.  (On GB300 every square root, division
// and unfused multiply-add is work on the narrow FP64 pipe, which bounds the evaluation.)
template <int P>
__device__ __forceinline__ int solve_small_fast(cplx (&A)[P][P], cplx (&b)[P], const bool (&active)[P]) {
  double nu = 0.0;
#pragma unroll
  for (int u = 0; u < P; ++u) {
    double su = 0.0;
#pragma unroll
    for (int v = 0; v < P; ++v) su += fabs(A[u][v].re) + fabs(A[u][v].im);
    if (active[u]) nu = fmax(nu, su);
  }
  // squared thresholds, widened by a relative 1e-9 against the rounding of the squares
  const double t2 = (kSingularRel * nu) * (kSingularRel * nu);
  const double tu2 = t2 * (1.0 + 1e-9), tl2 = t2 * (0.5 * (1.0 - 1e-9));
  int st = 1;
  double dinv[P];
#pragma unroll
  for (int c = 0; c < P; ++c) {
    int r = c;
    double best = fma(A[c][c].re, A[c][c].re, A[c][c].im * A[c][c].im);
#pragma unroll
    for (int rr = c + 1; rr < P; ++rr) {
      const double m = fma(A[rr][c].re, A[rr][c].re, A[rr][c].im * A[rr][c].im);
      if (m > best) { best = m; r = rr; }
    }
    if (!(best > 0.0) || best < tl2) st = 0;
    else if (!(best >= tu2) && st == 1) st = -1;
#pragma unroll
    for (int rr = c + 1; rr < P; ++rr) {
      if (rr == r) {
#pragma unroll
        for (int v = 0; v < P; ++v) { cplx t = A[c][v]; A[c][v] = A[rr][v]; A[rr][v] = t; }
        cplx t = b[c]; b[c] = b[rr]; b[rr] = t;
      }
    }
    if (st == 0) A[c][c] = mk(1.0, 0.0);
    const cplx piv = A[c][c];
    dinv[c] = 1.0 / fma(piv.re, piv.re, piv.im * piv.im);
    // multipliers a conj(piv) / |piv|^2, then the eliminations a - f u
    const cplx pc = mk(piv.re * dinv[c], -piv.im * dinv[c]);
#pragma unroll
    for (int rr = c + 1; rr < P; ++rr) {
      const cplx a0 = A[rr][c];
      const cplx f = mk(fma(a0.re, pc.re, -(a0.im * pc.im)), fma(a0.re, pc.im, a0.im * pc.re));
#pragma unroll
      for (int v = c + 1; v < P; ++v) A[rr][v] = cfms(f, A[c][v], A[rr][v]);
      b[rr] = cfms(f, b[c], b[rr]);
    }
  }
#pragma unroll
  for (int c = P - 1; c >= 0; --c) {
    cplx acc = b[c];
#pragma unroll
    for (int v = c + 1; v < P; ++v) acc = cfms(A[c][v], b[v], acc);
    const cplx pv = A[c][c];
    const cplx pc = mk(pv.re * dinv[c], -pv.im * dinv[c]);
    b[c] = mk(fma(acc.re, pc.re, -(acc.im * pc.im)), fma(acc.re, pc.im, acc.im * pc.re));
  }
  return st;
}

// Single-pixel candidates: id = j.  p = 1, so Eq. 9 is y = E_j / (1 - G_jj d_chi).
__device__ __forceinline__ void eval_single_body(const EvalArgs& a, const uint8_t* state,
                                                 int dir_mask, double* __restrict__ dfom, int64_t vb = -1, int64_t vg = -1) {
  // vb, vg: a virtual block index and count (a work item of a persistent kernel); -1: the grid's
  const int64_t vb_ = vb < 0 ? (int64_t)blockIdx.x : vb, vg_ = vg < 0 ? (int64_t)gridDim.x : vg;
  const int64_t N = (int64_t)a.nx * a.ny;
  const int64_t jend = a.c_end >= 0 && a.c_end < N ? a.c_end : N;
  for (int64_t j = a.c_begin + vb_ * (int64_t)blockDim.x + threadIdx.x; j < jend;
       j += (int64_t)vg_ * blockDim.x) {
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
__device__ __forceinline__ void eval_brush_body(const EvalArgs& a, const uint8_t* state,
                                                int dir_mask, double* __restrict__ dfom, int64_t vb = -1, int64_t vg = -1) {
  // vb, vg: a virtual block index and count (a work item of a persistent kernel); -1: the grid's
  const int64_t vb_ = vb < 0 ? (int64_t)blockIdx.x : vb, vg_ = vg < 0 ? (int64_t)gridDim.x : vg;
  const int nx = a.nx;
  const int64_t N = (int64_t)nx * a.ny;
  const int64_t P = (int64_t)(nx - 1) * (a.ny - 1);
  // local pixel offsets and the band that holds G[q_u, q_v]
  const int px[4] = {0, 1, 0, 1}, py[4] = {0, 0, 1, 1};
  const int band_of[9] = {8, 6, 4, 2, 0, 1, 3, 5, 7};   // index (ddy+1)*3 + (ddx+1)
  const int64_t aend = a.c_end >= 0 && a.c_end < P ? a.c_end : P;
  for (int64_t an = a.c_begin + vb_ * (int64_t)blockDim.x + threadIdx.x; an < aend;
       an += (int64_t)vg_ * blockDim.x) {
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
      cplx gN[4];                                         // the monitor row, both directions
#pragma unroll
      for (int u = 0; u < 4; ++u) gN[u] = ldG(L.G, a.dtype, L.ldg, N, q[u]);
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
        auto build = [&]() {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              int b = band_of[(py[v] - py[u] + 1) * 3 + (px[v] - px[u] + 1)];
              const cplx g = L.bands[(int64_t)b * N + q[u]];
              const double e = u == v ? 1.0 : 0.0;
              A[u][v] = act[u] ? mk(fma(-d[v], g.re, e), -(d[v] * g.im)) : mk(e, 0.0);
            }
            y[u] = act[u] ? L.E[q[u]] : mk(0.0, 0.0);
          }
        };
        build();
        int st = solve_small_fast<4>(A, y, act);
        if (st < 0) {                                     // a pivot near the threshold: the exact rule
          build();
          st = solve_small<4>(A, y, act) ? 1 : 0;
        }
        if (st == 0) { valid[dir] = false; continue; }
        cplx dE = mk(0.0, 0.0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (act[u]) dE = cfma(gN[u], mk(d[u] * y[u].re, d[u] * y[u].im), dE);
        }
        cplx Em = EN + dE;
        total[dir] += abs2(Em) - abs2(EN);
      }
    }
    dfom[an] = valid[0] ? total[0] : -INFINITY;
    dfom[P + an] = valid[1] ? total[1] : -INFINITY;
  }
}


// ----------------------------------------------------------------------------- selection
// (v, id) ordering: larger v first, then smaller id.  NaN never wins.
__device__ __forceinline__ bool better(double v, int64_t id, double bv, int64_t bid) {
  return v > bv || (v == bv && id < bid);
}

__device__ __forceinline__ void block_best(double& v, int64_t& id) {
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

// Greedy policy: m = max dfom; lowest id with dfom >= m - tie_rel |m|.
// An integer key that orders as the doubles do (-0 equal to +0, NaN below everything), so that
// the comparisons of a selection run on the integer units: the bit pattern, with the magnitude
// bits of negative values inverted.  key_value inverts it.
__device__ __forceinline__ long long ord_key(double v) {
  long long b = __double_as_longlong(v);
  if ((b & 0x7FFFFFFFFFFFFFFFll) > 0x7FF0000000000000ll) return LLONG_MIN;
  if (b == (long long)0x8000000000000000ull) b = 0;
  return b >= 0 ? b : b ^ 0x7FFFFFFFFFFFFFFFll;
}
__device__ __forceinline__ double key_value(long long k) {
  return __longlong_as_double(k >= 0 ? k : k ^ 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ void key_better(long long k, int64_t id, long long& bk, int64_t& bid) {
  if (k > bk || (k == bk && id < bid)) { bk = k; bid = id; }
}
// the block's best (key, id), in every thread
__device__ __forceinline__ void block_best_key(long long& k, int64_t& id) {
  __shared__ long long sk[32];
  __shared__ int64_t si[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) key_better(__shfl_down_sync(0xffffffffu, k, o), __shfl_down_sync(0xffffffffu, id, o), k, id);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { sk[w] = k; si[w] = id; }
  __syncthreads();
  if (w == 0) {
    k = l < (int)(blockDim.x >> 5) ? sk[l] : LLONG_MIN;
    id = l < (int)(blockDim.x >> 5) ? si[l] : INT64_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) key_better(__shfl_down_sync(0xffffffffu, k, o), __shfl_down_sync(0xffffffffu, id, o), k, id);
    if (l == 0) { sk[0] = k; si[0] = id; }
  }
  __syncthreads();
  k = sk[0];
  id = si[0];
}

// The greedy choice (Sec. II): the largest dFOM, and among the candidates within tie_rel of it
// (relative) the lowest id.  One CTA; each thread keeps four loads in flight, and the comparisons
// are on integer keys (on GB300 a double comparison is an instruction on the narrow FP64 pipe).
__device__ __forceinline__ void select_best_body(const double* dfom, int64_t ncand, double tie_rel,
                                                 int32_t* idx, double* val, int32_t* status) {
  const int64_t st = blockDim.x;
  long long bk = ord_key(-INFINITY);
  int64_t bid = INT64_MAX;
  int64_t c = threadIdx.x;
  for (; c + 3 * st < ncand; c += 4 * st) {
    const double v0 = dfom[c], v1 = dfom[c + st], v2 = dfom[c + 2 * st], v3 = dfom[c + 3 * st];
    key_better(ord_key(v0), c, bk, bid);
    key_better(ord_key(v1), c + st, bk, bid);
    key_better(ord_key(v2), c + 2 * st, bk, bid);
    key_better(ord_key(v3), c + 3 * st, bk, bid);
  }
  for (; c < ncand; c += st) key_better(ord_key(dfom[c]), c, bk, bid);
  block_best_key(bk, bid);
  const double m = key_value(bk);
  if (!(m > 0.0)) {
    if (threadIdx.x == 0) { idx[0] = -1; val[0] = m; *status = GF_ENOIMPROVE; }
    return;
  }
  double thr = m - tie_rel * fabs(m);
  if (!(thr <= m)) thr = m;                               // m = +inf
  const long long tk = ord_key(thr);
  // each thread's first candidate at or above the threshold
  int64_t first = INT64_MAX;
  c = threadIdx.x;
  for (; c + 3 * st < ncand; c += 4 * st) {
    const double v0 = dfom[c], v1 = dfom[c + st], v2 = dfom[c + 2 * st], v3 = dfom[c + 3 * st];
    if (ord_key(v0) >= tk) { first = c; break; }
    if (ord_key(v1) >= tk) { first = c + st; break; }
    if (ord_key(v2) >= tk) { first = c + 2 * st; break; }
    if (ord_key(v3) >= tk) { first = c + 3 * st; break; }
  }
  if (first == INT64_MAX)
    for (; c < ncand; c += st)
      if (ord_key(dfom[c]) >= tk) { first = c; break; }
  long long same = 0;
  block_best_key(same, first);                            // equal keys: the smallest id
  if (threadIdx.x == 0) {
    idx[0] = (int32_t)first;
    val[0] = dfom[first];
    *status = GF_OK;
  }
}

// One problem's selection (one CTA): greedy, or epsilon-greedy (Sec. V) with the problem's own
// uniform stream: the explore list (the four best improving candidates in (-dFOM, id) order) comes
// from four block-wide passes that skip the ids already taken.
__device__ __forceinline__ void batch_select_body(const BatchItem& it, double tie_rel) {
  select_best_body(it.dfom, it.ncand, tie_rel, it.idx, it.val, it.status);
  if (!(it.epsilon > 0.0)) return;
  __shared__ int s_go;
  __shared__ int64_t s_top[4];
  __shared__ double s_val[4];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int32_t t = *it.step;
    *it.step = t + 1;
    s_go = 0;
    if (t >= it.horizon) {
      *it.status = GF_ENOMEM;                     // the uniform stream is exhausted
    } else if (*it.status == GF_OK && it.uniforms[2 * (int64_t)t] < it.epsilon) {
      s_go = 1;
    }
  }
  __syncthreads();
  if (!s_go) return;
  int m = 0;
  for (int pass = 0; pass < 4; ++pass) {
    double bv = -INFINITY;
    int64_t bid = INT64_MAX;
    for (int64_t c = threadIdx.x; c < it.ncand; c += blockDim.x) {
      const double v = it.dfom[c];
      if (!(v > 0.0) || !better(v, c, bv, bid)) continue;
      bool taken = false;
      for (int q = 0; q < pass; ++q) taken |= s_top[q] == c;
      if (!taken) { bv = v; bid = c; }
    }
    block_best(bv, bid);
    if (!(bv > 0.0)) break;
    if (threadIdx.x == 0) { s_top[pass] = bid; s_val[pass] = bv; }
    __syncthreads();
    m = pass + 1;
  }
  if (threadIdx.x == 0 && m > 0) {
    const int32_t t = *it.step - 1;
    int r = (int)(it.uniforms[2 * (int64_t)t + 1] * (double)m);
    if (r > m - 1) r = m - 1;
    if (r < 0) r = 0;
    it.idx[0] = (int32_t)s_top[r];
    it.val[0] = s_val[r];
  }
}

// ----------------------------------------------------------------------------- bands
__device__ __forceinline__ void bands_body(int nx, int ny, int dtype, const void* G, int64_t ldg,
                                           cplx* __restrict__ bands, int64_t vb = -1, int64_t vg = -1) {
  // vb, vg: a virtual block index and count (a work item of a persistent kernel); -1: the grid's
  const int64_t vb_ = vb < 0 ? (int64_t)blockIdx.x : vb, vg_ = vg < 0 ? (int64_t)gridDim.x : vg;
  const int64_t N = (int64_t)nx * ny;
  // a thread per pixel: its nine entries lie in three runs of three neighbouring columns of row
  // i, loaded together; each band is then written with consecutive pixels in consecutive threads
  for (int64_t i = vb_ * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)vg_ * blockDim.x) {
    const int iy = (int)(i / nx), ix = (int)(i - (int64_t)iy * nx);
    cplx v[GF_NBANDS];
#pragma unroll
    for (int b = 0; b < GF_NBANDS; ++b) {
      int ddx, ddy;
      band_offset(b, ddx, ddy);
      const int jx = ix + ddx, jy = iy + ddy;
      v[b] = (jx >= 0 && jx < nx && jy >= 0 && jy < ny) ? ldG(G, dtype, ldg, i, (int64_t)jy * nx + jx) : mk(0.0, 0.0);
    }
#pragma unroll
    for (int b = 0; b < GF_NBANDS; ++b) bands[(int64_t)b * N + i] = v[b];
  }
}

// ----------------------------------------------------------------------------- capacitance
struct CapArgs {
  UpdArgs u;
  int kind, dir_mask, k;
  int pmax;
};

// Blocked right-looking LU with partial pivoting of the row-major p x p complex matrix A (global
// memory), for p <= kLuMaxBlocked, by the whole CTA.  Panels of kLuNB columns are factored in
// shared memory (pivot = largest modulus, lowest row on ties, as in the unblocked form); their row
// interchanges are then applied to the rest of the rows, U12 = L11^{-1} A12 is solved column by
// column and the trailing matrix receives the rank-kLuNB update -- every element independently,
// so the global-memory traffic is parallel instead of a chain of dependent accesses.  The result
// (L below the diagonal with unit diagonal, U on and above it, piv[c] = row exchanged with row c
// at step c) is the unblocked factorisation's.  Returns false (in every thread) when a pivot is
// zero or below thresh.
constexpr int kLuNB = 8;
constexpr int kLuMaxBlocked = 256;
constexpr int kCapSmemP = 64;          // capacitance systems up to this size in shared memory (64 KB)
constexpr int kCapClusterMinP = 32;    // joint sets above this size: a cluster of CTAs per wavelength

// sP: shared memory for kLuMaxBlocked x kLuNB entries (the panel, row-major [row][j])
inline __device__ bool lu_blocked(cplx* __restrict__ A, int p, int32_t* __restrict__ piv, double thresh, cplx* sP) {
  __shared__ int s_pv[kLuNB];
  __shared__ int s_bad2, s_pr;
  __shared__ cplx s_inv;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_bad2 = 0;
  __syncthreads();
  for (int c0 = 0; c0 < p; c0 += kLuNB) {
    const int nb = p - c0 < kLuNB ? p - c0 : kLuNB;
    const int m = p - c0;
    for (int t = tid; t < m * nb; t += nt) {
      const int r = t / nb, j = t - r * nb;
      sP[r * kLuNB + j] = A[(int64_t)(c0 + r) * p + c0 + j];
    }
    __syncthreads();
    // ---- panel factorisation in shared memory.  The pivot search is one warp's: the largest
    // |a|^2 (the order of the moduli), lowest row on ties; its lane 0 also forms 1 / pivot, so
    // each row's multiplier is a product instead of a division.
    for (int j = 0; j < nb; ++j) {
      if (wid == 0) {
        double bv = -1.0;
        int br = 0x7fffffff;
        for (int r = j + lane; r < m; r += 32) {
          const double v = abs2(sP[r * kLuNB + j]);
          if (v > bv) { bv = v; br = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const double ov = __shfl_down_sync(0xffffffffu, bv, o);
          const int orr = __shfl_down_sync(0xffffffffu, br, o);
          if (ov > bv || (ov == bv && orr < br)) { bv = ov; br = orr; }
        }
        if (lane == 0) {
          if (!(bv >= thresh * thresh) || !(bv > 0.0)) {
            s_bad2 = 1;
          } else {
            const cplx pv = sP[br * kLuNB + j];
            const double d = rcp_nr(bv);
            s_inv = mk(pv.re * d, -pv.im * d);
          }
          s_pr = br;
          s_pv[j] = c0 + br;
          piv[c0 + j] = c0 + br;
        }
      }
      __syncthreads();
      if (s_bad2) return false;
      const int pr = s_pr;
      if (pr != j && tid < nb) {
        const cplx t0 = sP[j * kLuNB + tid];
        sP[j * kLuNB + tid] = sP[pr * kLuNB + tid];
        sP[pr * kLuNB + tid] = t0;
      }
      __syncthreads();
      const cplx inv = s_inv;
      for (int r = j + 1 + tid; r < m; r += nt) {
        const cplx f = sP[r * kLuNB + j] * inv;
        sP[r * kLuNB + j] = f;
        for (int k = j + 1; k < nb; ++k) sP[r * kLuNB + k] = cfms(f, sP[j * kLuNB + k], sP[r * kLuNB + k]);
      }
      __syncthreads();
    }
    for (int t = tid; t < m * nb; t += nt) {
      const int r = t / nb, j = t - r * nb;
      A[(int64_t)(c0 + r) * p + c0 + j] = sP[r * kLuNB + j];
    }
    // ---- the panel's interchanges on the columns outside it (one thread per column)
    for (int v = tid; v < p; v += nt) {
      if (v >= c0 && v < c0 + nb) continue;
      for (int j = 0; j < nb; ++j) {
        const int r = s_pv[j];
        if (r != c0 + j) {
          const cplx t0 = A[(int64_t)(c0 + j) * p + v];
          A[(int64_t)(c0 + j) * p + v] = A[(int64_t)r * p + v];
          A[(int64_t)r * p + v] = t0;
        }
      }
    }
    __syncthreads();
    const int w = p - c0 - nb;                   // trailing width
    if (w > 0) {
      // ---- U12 = L11^{-1} A12 (unit lower, one thread per column); for p <= kLuMaxBlocked / 2
      // the block is also kept in the free half of the panel buffer for the trailing update
      cplx* sU = p <= kLuMaxBlocked / 2 ? sP + (kLuMaxBlocked / 2) * kLuNB : nullptr;
      for (int v = tid; v < w; v += nt) {
        cplx x[kLuNB];
#pragma unroll
        for (int j = 0; j < kLuNB; ++j)
          if (j < nb) x[j] = A[(int64_t)(c0 + j) * p + c0 + nb + v];
#pragma unroll
        for (int j = 1; j < kLuNB; ++j)
          if (j < nb)
#pragma unroll
            for (int i = 0; i < kLuNB; ++i)
              if (i < j) x[j] = cfms(sP[j * kLuNB + i], x[i], x[j]);
#pragma unroll
        for (int j = 1; j < kLuNB; ++j)
          if (j < nb) A[(int64_t)(c0 + j) * p + c0 + nb + v] = x[j];
        if (sU)
#pragma unroll
          for (int j = 0; j < kLuNB; ++j)
            if (j < nb) sU[j * w + v] = x[j];
      }
      __syncthreads();
      // ---- A22 -= L21 U12, every element independently (coalesced along the row)
      for (int e = tid; e < w * w; e += nt) {
        const int i = e / w, v = e - i * w;
        const int64_t o = (int64_t)(c0 + nb + i) * p + c0 + nb + v;
        cplx acc = A[o];
#pragma unroll
        for (int j = 0; j < kLuNB; ++j)
          if (j < nb)
            acc = cfms(sP[(nb + i) * kLuNB + j], sU ? sU[j * w + v] : A[(int64_t)(c0 + j) * p + c0 + nb + v], acc);
        A[o] = acc;
      }
    }
    __syncthreads();
  }
  return true;
}

// A = I - G_VV D (row-major p x p, Eq. 9) and y = E_V for one wavelength; returns the pivot
// threshold kSingularRel ||A||_inf (every thread).
inline __device__ double cap_build(const CapArgs& a, const UpdLam& U, int p, const int32_t* V,
                            const double* dchi, cplx* A, cplx* y) {
  __shared__ double s_red[32];
  const int tid = threadIdx.x;
  for (int t = tid; t < p * p; t += blockDim.x) {
    int r = t / p, c = t % p;
    cplx g = U.vrows ? ldG(U.vrows, a.u.dtype, U.ldv, r, V[c]) : ldG(U.G, a.u.dtype, U.ldg, V[r], V[c]);
    cplx e = mk(r == c ? 1.0 : 0.0, 0.0);
    A[t] = e - dchi[c] * g;
  }
  for (int t = tid; t < p; t += blockDim.x) y[t] = U.E[V[t]];
  __syncthreads();
  // ||A||_inf
  double rs = 0.0;
  for (int r = tid; r < p; r += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < p; ++c) s += cabs1(A[r * p + c]);
    rs = fmax(rs, s);
  }
  for (int o = 16; o > 0; o >>= 1) rs = fmax(rs, __shfl_down_sync(0xffffffffu, rs, o));
  if ((tid & 31) == 0) s_red[tid >> 5] = rs;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s_red[w]);
    s_red[0] = m;
  }
  __syncthreads();
  const double thresh = kSingularRel * s_red[0];
  __syncthreads();
  return thresh;
}

// With the factors of A (L below the diagonal, U on and above, piv), y <- A^{-1} y after y was
// permuted and reduced by L (y_is_lower: the unit-lower solve is still to do), the dFOM of Eq. 4
// at the monitor's unknowns (Eq. 1) into the return value (every thread), and y <- D y.
inline __device__ double cap_tail(const CapArgs& a, const UpdLam& U, int p, const int32_t* V,
                           const double* dchi, const cplx* A, const int32_t* piv, cplx* y,
                           bool lower_done) {
  __shared__ double s_red[32];
  __shared__ double s_bv[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = (int)(blockDim.x >> 5);
  if (!lower_done) {
    // y = P E_V, then the unit-lower solve (column-oriented: one synchronisation per column)
    if (tid == 0)
      for (int c = 0; c < p; ++c) {
        const int r = piv[c];
        if (r != c) { cplx t0 = y[c]; y[c] = y[r]; y[r] = t0; }
      }
    __syncthreads();
    for (int c = 0; c < p; ++c) {
      const cplx yc = y[c];
      for (int r = c + 1 + tid; r < p; r += blockDim.x) y[r] = cfms(A[r * p + c], yc, y[r]);
      __syncthreads();
    }
  }
  // upper solve for y in blocks of kLuNB rows from the bottom: one thread solves the block's
  // triangle, then every row above takes the block's terms (two synchronisations per block)
  for (int b1 = p; b1 > 0; b1 -= kLuNB) {
    const int b0 = b1 - kLuNB > 0 ? b1 - kLuNB : 0;
    if (tid == 0)
      for (int c = b1 - 1; c >= b0; --c) {
        cplx acc = y[c];
        for (int v = c + 1; v < b1; ++v) acc = acc - A[c * p + v] * y[v];
        y[c] = cdiv(acc, A[c * p + c]);
      }
    __syncthreads();
    for (int r = tid; r < b0; r += blockDim.x) {
      cplx acc = y[r];
      for (int v = b0; v < b1; ++v) acc = acc - A[r * p + v] * y[v];
      y[r] = acc;
    }
    __syncthreads();
  }
  // Eq. 4 at the monitor's unknowns (Eq. 1): the gathers of the monitor row are spread over
  // the block and reduced
  double df = 0.0;
  for (int mc = 0; mc < a.u.mcount; ++mc) {
    const int64_t m = a.u.mrow + mc;
    cplx part = mk(0.0, 0.0);
    // G[m, V[u]]; from the row panel as G[V[u], m] (reciprocity)
    for (int u = tid; u < p; u += blockDim.x) {
      const cplx gm = U.vrows ? ldG(U.vrows, a.u.dtype, U.ldv, u, m) : ldG(U.G, a.u.dtype, U.ldg, m, V[u]);
      part = part + dchi[u] * (gm * y[u]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      part.re += __shfl_down_sync(0xffffffffu, part.re, o);
      part.im += __shfl_down_sync(0xffffffffu, part.im, o);
    }
    if (lane == 0) { s_bv[wid] = part.re; s_red[wid] = part.im; }
    __syncthreads();
    if (tid == 0) {
      cplx dE = mk(0.0, 0.0);
      for (int w = 0; w < nw; ++w) dE = dE + mk(s_bv[w], s_red[w]);
      const cplx EN = U.E[m];
      df += abs2(EN + dE) - abs2(EN);
    }
    __syncthreads();
  }
  if (tid == 0) s_red[0] = df;
  for (int u = tid; u < p; u += blockDim.x) y[u] = dchi[u] * y[u];      // D y for the field update
  __syncthreads();
  df = s_red[0];
  __syncthreads();
  return df;
}

// cap_lam for p <= kMaxPixelsPerCand (a candidate's pixels, one monitor unknown) in warp 0,
// without block-wide barriers: lane (r, c) = 8 r + c holds entry (r, c) of [A | y] (c < 4: A,
// c = 4: y) and, outside the interchanges, G[m, V[r]] (c = 5) and E[m] (lane 6), gathered in one
// round of loads.  Each step of the general path (cap_build's row sums, lu_blocked's pivot,
// reciprocal, interchange, multipliers and eliminations, cap_tail's forward and upper solves and
// Eq. 4) is one warp instruction sequence over the lanes, with the operands of every element in
// the general path's order -- the same bits (the forward solve's updates of y are its
// eliminations; the upper solve's reciprocals are formed in parallel, cdiv_r giving cdiv's bits).
// On GB300 a warp's FP64 instruction costs the SM's FP64 pipe the same with one lane or 32, so
// one lane running the whole solve would take as long as the barriers it saves.  Returns as
// cap_lam, after one barrier that gives every thread the outcome.
inline __device__ bool cap_lam_small(const CapArgs& a, const WsLayout& L, char* ws, int l, int p,
                                     const int32_t* V, const double* dchi, double* df_out) {
  constexpr int Q = kMaxPixelsPerCand;
  static_assert(Q == 4, "four rows of eight lanes");
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ double s_out;
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  if (tid < 32) {
    const UpdLam& U = a.u.lam[l];
    const int lane = tid, r = lane >> 3, c = lane & 7;
    const bool rowv = r < p;
    const int64_t m = a.u.mrow;
    const int32_t vr = rowv ? V[r] : 0;
    const double dr = rowv ? dchi[r] : 0.0;
    cplx x = mk(0.0, 0.0);
    if (rowv && c < p) {
      const int32_t vc = V[c];
      const cplx g = U.vrows ? ldG(U.vrows, a.u.dtype, U.ldv, r, vc) : ldG(U.G, a.u.dtype, U.ldg, vr, vc);
      x = mk(r == c ? 1.0 : 0.0, 0.0) - dchi[c] * g;
    } else if (rowv && c == 4) {
      x = U.E[vr];
    } else if (rowv && c == 5) {
      x = U.vrows ? ldG(U.vrows, a.u.dtype, U.ldv, r, m) : ldG(U.G, a.u.dtype, U.ldg, m, vr);
    } else if (lane == 6) {
      x = U.E[m];
    }
    auto sh = [&](cplx v, int src) { return mk(__shfl_sync(FULL, v.re, src), __shfl_sync(FULL, v.im, src)); };
    // cap_build's threshold: each row's sum of |a| in column order, the largest over the rows
    const double ax = (rowv && c < p) ? cabs1(x) : 0.0;
    double srow = 0.0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const double t = __shfl_sync(FULL, ax, (lane & ~7) + q);
      if (q < p) srow += t;
    }
    double rs = 0.0;
#pragma unroll
    for (int rr = 0; rr < Q; ++rr) {
      const double t = __shfl_sync(FULL, srow, rr * 8);
      if (rr < p) rs = fmax(rs, t);
    }
    const double thresh = kSingularRel * rs;
    bool ok = true;
    int pv[Q] = {0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      if (j >= p || !ok) continue;
      // the pivot: the largest |a|^2 of column j at or below row j, the lowest row on ties
      const double v = abs2(x);
      double bv = -1.0;
      int br = j;
#pragma unroll
      for (int rr = 0; rr < Q; ++rr) {
        const double t = __shfl_sync(FULL, v, rr * 8 + j);
        if (rr >= j && rr < p && t > bv) { bv = t; br = rr; }
      }
      if (!(bv >= thresh * thresh) || !(bv > 0.0)) { ok = false; continue; }
      const cplx pvv = sh(x, br * 8 + j);
      const double d = rcp_nr(bv);
      const cplx inv = mk(pvv.re * d, -pvv.im * d);
      pv[j] = br;
      // the interchange of rows j and br (A and y)
      const cplx xj = sh(x, j * 8 + c), xb = sh(x, br * 8 + c);
      if (c <= 4 && br != j) {
        if (r == j) x = xb;
        else if (r == br) x = xj;
      }
      // the multipliers, then the eliminations of the columns right of j and of y
      if (r > j && r < p && c == j) x = x * inv;
      const cplx f = sh(x, r * 8 + j), u = sh(x, j * 8 + c);
      if (r > j && r < p && ((c > j && c < p) || c == 4)) x = cfms(f, u, x);
    }
    double df = 0.0;
    if (ok) {
      // the upper solve from the bottom, the solution in every lane
      const double dd = (rowv && c == r) ? 1.0 / abs2(x) : 0.0;
      cplx xs[Q];
#pragma unroll
      for (int cc = Q - 1; cc >= 0; --cc) {
        xs[cc] = mk(0.0, 0.0);
        if (cc >= p) continue;
        cplx acc = sh(x, cc * 8 + 4);
#pragma unroll
        for (int v = 0; v < Q; ++v)
          if (v > cc && v < p) acc = acc - sh(x, cc * 8 + v) * xs[v];
        xs[cc] = cdiv_r(acc, sh(x, cc * 8 + cc), __shfl_sync(FULL, dd, cc * 8 + cc));
      }
      // Eq. 4 at the monitor: the block reduction's order for terms 0..3, (t0 + t2) + (t1 + t3)
      cplx t[Q];
#pragma unroll
      for (int uu = 0; uu < Q; ++uu) {
        const cplx gm = sh(x, uu * 8 + 5);
        const double du = __shfl_sync(FULL, dr, uu * 8);
        t[uu] = uu < p ? du * (gm * xs[uu]) : mk(0.0, 0.0);
      }
      const cplx dE = (t[0] + t[2]) + (t[1] + t[3]);
      const cplx EN = sh(x, 6);
      df = abs2(EN + dE) - abs2(EN);
      // outputs: the factors, the interchanges, D y
      cplx* Aw = reinterpret_cast<cplx*>(ws + L.lu + l * L.lu_s);
      int32_t* piv = reinterpret_cast<int32_t*>(ws + L.piv + l * L.piv_s);
      cplx* yw = reinterpret_cast<cplx*>(ws + L.yd + l * L.yd_s);
      if (rowv && c < p) Aw[r * p + c] = x;
      cplx xl = xs[0];
      int pl = pv[0];
#pragma unroll
      for (int q = 1; q < Q; ++q)
        if (lane == q) { xl = xs[q]; pl = pv[q]; }
      if (lane < p) {
        piv[lane] = pl;
        yw[lane] = dchi[lane] * xl;
      }
    }
    if (lane == 0) {
      s_ok = ok ? 1 : 0;
      s_out = df;
    }
  }
  __syncthreads();
  const bool ok = s_ok != 0;
  *df_out = s_out;
  __syncthreads();
  return ok;
}

// One wavelength of the capacitance solve for the set V (p pixels, contrasts dchi): A = I - G_VV D
// (Eq. 9), its LU with partial pivoting, y = A^{-1} E_V and the dFOM of Eq. 4 at the monitor into
// *df (every thread); the factors, pivots and D y go to the wavelength's workspace slots.  With sA
// (shared memory for kCapSmemP^2 + kCapSmemP entries) a system of p <= kCapSmemP and its
// right-hand side are built, factorised and solved there and copied to the workspace once.
// Returns false (in every thread) when A is singular.
inline __device__ bool cap_lam(const CapArgs& a, const WsLayout& L, char* ws, int l, int p, const int32_t* V,
                        const double* dchi, cplx* sA, double* df_out) {
  if (p <= kMaxPixelsPerCand && a.u.mcount == 1) return cap_lam_small(a, L, ws, l, p, V, dchi, df_out);
  const int tid = threadIdx.x;
  const UpdLam& U = a.u.lam[l];
  cplx* Aw = reinterpret_cast<cplx*>(ws + L.lu + l * L.lu_s);
  const bool in_smem = sA && p <= kCapSmemP;
  cplx* A = in_smem ? sA : Aw;
  int32_t* piv = reinterpret_cast<int32_t*>(ws + L.piv + l * L.piv_s);
  cplx* yw = reinterpret_cast<cplx*>(ws + L.yd + l * L.yd_s);
  cplx* y = in_smem ? sA + kCapSmemP * kCapSmemP : yw;
  const double thresh = cap_build(a, U, p, V, dchi, A, y);
  // LU with partial pivoting (row-major, in place; L below the diagonal, unit diagonal).
  __shared__ int s_piv;
  __shared__ int s_bad;
  __shared__ double s_bv[32];
  __shared__ int s_br[32];
  __shared__ cplx s_f[kLuMaxBlocked * kLuNB];   // blocked: the panel; unblocked: multipliers
  if (tid == 0) s_bad = 0;
  const int nw = (int)(blockDim.x >> 5), lane = tid & 31, wid = tid >> 5;
  bool lower_done = false;
  if (p <= kLuMaxBlocked) {
    if (!lu_blocked(A, p, piv, thresh, s_f)) return false;
  } else {
    // unblocked form for very large joint sets (p > 256): pivot search across the block,
    // multipliers per row, trailing update with a warp per row and lanes along the columns; y
    // is permuted and reduced alongside
    lower_done = true;
    for (int c = 0; c < p; ++c) {
      double bv = -1.0;
      int br = 0x7fffffff;
      for (int rr = c + tid; rr < p; rr += blockDim.x) {
        const double m = cabs1(A[rr * p + c]);
        if (m > bv) { bv = m; br = rr; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int orr = __shfl_down_sync(0xffffffffu, br, o);
        if (ov > bv || (ov == bv && orr < br)) { bv = ov; br = orr; }
      }
      if (lane == 0) { s_bv[wid] = bv; s_br[wid] = br; }
      __syncthreads();
      if (tid == 0) {
        double b = s_bv[0];
        int r = s_br[0];
        for (int w = 1; w < nw; ++w)
          if (s_bv[w] > b || (s_bv[w] == b && s_br[w] < r)) { b = s_bv[w]; r = s_br[w]; }
        if (!(b >= thresh) || !(b > 0.0)) s_bad = 1;
        s_piv = r;
        piv[c] = r;
      }
      __syncthreads();
      const int r = s_piv;
      if (s_bad) break;
      if (r != c) {
        for (int v = tid; v < p; v += blockDim.x) {
          cplx t0 = A[c * p + v];
          A[c * p + v] = A[r * p + v];
          A[r * p + v] = t0;
        }
        if (tid == 0) { cplx t0 = y[c]; y[c] = y[r]; y[r] = t0; }
      }
      __syncthreads();
      const cplx pv = A[c * p + c];
      const cplx yc = y[c];
      for (int rr = c + 1 + tid; rr < p; rr += blockDim.x) {
        const cplx f = cdiv(A[rr * p + c], pv);
        s_f[rr] = f;
        A[rr * p + c] = f;
        y[rr] = y[rr] - f * yc;
      }
      __syncthreads();
      for (int rr = c + 1 + wid; rr < p; rr += nw) {
        const cplx f = s_f[rr];
        for (int v = c + 1 + lane; v < p; v += 32) A[rr * p + v] = A[rr * p + v] - f * A[c * p + v];
      }
      __syncthreads();
    }
    __syncthreads();
    if (s_bad) return false;
  }
  const double df = cap_tail(a, U, p, V, dchi, A, piv, y, lower_done);
  if (in_smem) {                                 // the factors and D y for the later kernels
    for (int t = tid; t < p * p; t += blockDim.x) Aw[t] = A[t];
    for (int t = tid; t < p; t += blockDim.x) yw[t] = y[t];
  }
  __syncthreads();
  *df_out = df;
  __syncthreads();
  return true;
}

// Single CTA: the set V of the accepted candidates, every wavelength's solve (cap_lam; with pre,
// the first attempt's solves were done by k_capacitance_lam and are read from the control block),
// the joint decision and the fallback to the best single candidate.  The p x p matrices live in
// the workspace (p can reach 4k), or in sA for p <= kCapSmemP.
__device__ __forceinline__ void capacitance_body(const CapArgs& a, const WsLayout& L, char* ws,
                                                 const uint8_t* state, const int32_t* idx, int32_t* status,
                                                 cplx* sA = nullptr, bool pre = false) {
  UpdCtl* ctl = reinterpret_cast<UpdCtl*>(ws + L.ctl);
  int32_t* V = reinterpret_cast<int32_t*>(ws + L.V);
  double* dchi = reinterpret_cast<double*>(ws + L.dchi);
  __shared__ int s_nv, s_ncand, s_fail;
  const int tid = threadIdx.x;

  if (tid == 0) {
    s_fail = 0;
    s_ncand = 0;
    s_nv = 0;
    if (*status != GF_OK) {
      s_fail = 1;
    } else {
      int nv = 0, nc = 0;
      for (int c = 0; c < a.k; ++c) {
        int32_t id = idx[c];
        if (id < 0) break;
        int m = cand_pixels(id, a.kind, a.dir_mask, a.u.nx, a.u.ny, a.u.chi, state, V + nv, dchi + nv, a.u.nz);
        if (m == 0) continue;
        nv += m;
        ++nc;
      }
      s_nv = nv;
      s_ncand = nc;
      if (nv == 0) s_fail = 2;
    }
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) {
      ctl->skip = 1;
      ctl->nv = 0;
      ctl->ncand = 0;
      ctl->joint_dfom = 0.0;
    }
    return;
  }

  for (int attempt = 0; attempt < 2; ++attempt) {
    const int p = s_nv;
    double total = 0.0;
    bool singular = false;
    for (int l = 0; l < a.u.nlam; ++l) {
      double df = 0.0;
      if (pre && attempt == 0) {                     // the per-wavelength kernel solved it
        df = ctl->lam_df[l];
        if (ctl->lam_bad[l]) { singular = true; break; }
      } else if (!cap_lam(a, L, ws, l, p, V, dchi, sA, &df)) {
        singular = true;
        break;
      }
      total += df;
    }
    if (singular) {
      if (tid == 0) {
        *status = GF_ESINGULAR;
        ctl->skip = 1;
        ctl->nv = 0;
        ctl->ncand = 0;
        ctl->joint_dfom = 0.0;
      }
      return;
    }
    if (s_ncand > 1 && !(total > 0.0) && attempt == 0) {
      // the joint set does not improve the FOM: apply the best candidate alone
      __syncthreads();
      if (tid == 0) {
        int m = cand_pixels(idx[0], a.kind, a.dir_mask, a.u.nx, a.u.ny, a.u.chi, state, V, dchi, a.u.nz);
        s_nv = m;
        s_ncand = 1;
      }
      __syncthreads();
      continue;
    }
    if (tid == 0) {
      ctl->skip = 0;
      ctl->nv = s_nv;
      ctl->ncand = s_ncand;
      ctl->joint_dfom = total;
    }
    return;
  }
}

// ----------------------------------------------------------------------------- panels
// Column j: R[:, j] = A^{-1} G[V, j] (Eq. 14) and S[:, j] = D R[:, j]; row j of the rows held:
// C0[j, :] = G[j, V].
__device__ __forceinline__ void panels_body(const UpdArgs& a, const WsLayout& L, char* ws, int want_S, int64_t vb = -1, int64_t vg = -1) {
  // vb, vg: a virtual block index and count (a work item of a persistent kernel); -1: the grid's
  const int64_t vb_ = vb < 0 ? (int64_t)blockIdx.x : vb, vg_ = vg < 0 ? (int64_t)gridDim.x : vg;
  const UpdCtl* ctl = reinterpret_cast<const UpdCtl*>(ws + L.ctl);
  if (ctl->skip) return;
  const int p = ctl->nv;
  const int32_t* V = reinterpret_cast<const int32_t*>(ws + L.V);
  const double* dchi = reinterpret_cast<const double*>(ws + L.dchi);
  const int64_t n = L.n;
  for (int l = 0; l < a.nlam; ++l) {
    const UpdLam& U = a.lam[l];
    const cplx* A = reinterpret_cast<const cplx*>(ws + L.lu + l * L.lu_s);
    const int32_t* piv = reinterpret_cast<const int32_t*>(ws + L.piv + l * L.piv_s);
    cplx* C0 = reinterpret_cast<cplx*>(ws + L.C0 + l * L.panel_s);
    cplx* S = reinterpret_cast<cplx*>(ws + L.S + l * L.panel_s);
    const int64_t jend = U.rows > n ? U.rows : n;
    // the reciprocals 1 / |u_cc|^2 of the upper solve, once per CTA instead of a division per
    // column; the first barrier keeps the previous wavelength's or work item's readers
    __shared__ double s_dinv[kMaxPixelsPerCand];
    if (want_S && p <= kMaxPixelsPerCand) {
      __syncthreads();
      if (threadIdx.x < p) s_dinv[threadIdx.x] = 1.0 / abs2(A[threadIdx.x * p + threadIdx.x]);
      __syncthreads();
    }
    for (int64_t j = vb_ * (int64_t)blockDim.x + threadIdx.x; j < jend;
         j += (int64_t)vg_ * blockDim.x) {
      if (j < U.rows)
        for (int u = 0; u < p; ++u) C0[j * L.pmax + u] = ldG(U.G, a.dtype, U.ldg, j, V[u]);
      if (!want_S || j >= n) continue;
      if (p <= kMaxPixelsPerCand) {
        cplx x[kMaxPixelsPerCand];
#pragma unroll
        for (int u = 0; u < kMaxPixelsPerCand; ++u)
          if (u < p) x[u] = U.vrows ? ldG(U.vrows, a.dtype, U.ldv, u, j) : ldG(U.G, a.dtype, U.ldg, V[u], j);
        // P A = L U with full-row interchanges: apply all interchanges in order first,
        // then the unit-lower solve, then the upper solve (fused multiply-adds: the panels of
        // a step run this for every column of G, on the narrow FP64 pipe)
#pragma unroll
        for (int c = 0; c < kMaxPixelsPerCand; ++c) {
          if (c < p) {
            int r = piv[c];
#pragma unroll
            for (int rr = 0; rr < kMaxPixelsPerCand; ++rr)
              if (rr == r && rr != c) { cplx t = x[c]; x[c] = x[rr]; x[rr] = t; }
          }
        }
#pragma unroll
        for (int c = 0; c < kMaxPixelsPerCand; ++c) {
          if (c < p) {
#pragma unroll
            for (int rr = c + 1; rr < kMaxPixelsPerCand; ++rr)
              if (rr < p) x[rr] = cfms(A[rr * p + c], x[c], x[rr]);
          }
        }
#pragma unroll
        for (int c = kMaxPixelsPerCand - 1; c >= 0; --c) {
          if (c < p) {
            cplx acc = x[c];
#pragma unroll
            for (int v = c + 1; v < kMaxPixelsPerCand; ++v)
              if (v < p) acc = cfms(A[c * p + v], x[v], acc);
            const cplx u = A[c * p + c];
            x[c] = mk(fma(acc.re, u.re, acc.im * u.im) * s_dinv[c], fma(acc.im, u.re, -(acc.re * u.im)) * s_dinv[c]);
          }
        }
#pragma unroll
        for (int u = 0; u < kMaxPixelsPerCand; ++u)
          if (u < p) S[(int64_t)u * n + j] = dchi[u] * x[u];
      } else {
        // general p: the column of R lives in S itself (row stride n)
        for (int u = 0; u < p; ++u)
          S[(int64_t)u * n + j] = U.vrows ? ldG(U.vrows, a.dtype, U.ldv, u, j) : ldG(U.G, a.dtype, U.ldg, V[u], j);
        for (int c = 0; c < p; ++c) {
          int r = piv[c];
          if (r != c) {
            cplx t = S[(int64_t)c * n + j];
            S[(int64_t)c * n + j] = S[(int64_t)r * n + j];
            S[(int64_t)r * n + j] = t;
          }
        }
        for (int c = 0; c < p; ++c) {
          cplx xc = S[(int64_t)c * n + j];
          for (int rr = c + 1; rr < p; ++rr)
            S[(int64_t)rr * n + j] = S[(int64_t)rr * n + j] - A[rr * p + c] * xc;
        }
        for (int c = p - 1; c >= 0; --c) {
          cplx acc = S[(int64_t)c * n + j];
          for (int v = c + 1; v < p; ++v) acc = acc - A[c * p + v] * S[(int64_t)v * n + j];
          S[(int64_t)c * n + j] = cdiv(acc, A[c * p + c]);
        }
        for (int u = 0; u < p; ++u) S[(int64_t)u * n + j] = dchi[u] * S[(int64_t)u * n + j];
      }
    }
  }
}

// complex128, the FP64 FMA update of column j for rows [i0, i1): G[i, j] += sum_u C0[i, u] S[u, j]
// in the order of k_rank_update_f64 (the same bits).  P > 0: compile-time rank; P == 0: runtime p.
template <int P>
__device__ __forceinline__ void f64_update_rows(double2* G, int64_t ldg, int64_t n, int64_t i0, int64_t i1, int pmax,
                                                int p, const cplx* C0, const cplx* S, int64_t j) {
  cplx s[P > 0 ? P : 1];
  if (P > 0) {
#pragma unroll
    for (int u = 0; u < P; ++u) s[u] = S[(int64_t)u * n + j];
  }
  // eight rows' loads in flight before their arithmetic (one row at a time, each thread waited a
  // full memory latency per row)
  constexpr int U = 8;
  for (int64_t i = i0; i < i1; i += U) {
    double2 g[U];
#pragma unroll
    for (int q = 0; q < U; ++q)
      if (i + q < i1) g[q] = G[(i + q) * ldg + j];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      if (i + q < i1) {
        const int64_t r = i + q;
        cplx acc = mk(g[q].x, g[q].y);
        if (P > 0) {
#pragma unroll
          for (int u = 0; u < P; ++u) acc = cfma(C0[r * pmax + u], s[u], acc);
        } else {
          for (int u = 0; u < p; ++u) acc = cfma(C0[r * pmax + u], S[(int64_t)u * n + j], acc);
        }
        G[r * ldg + j] = make_double2(acc.re, acc.im);
      }
    }
  }
}
constexpr int kF64BatchRows = 16;                 // rows of one batched FP64 update tile (x 256 columns)
__device__ __forceinline__ void f64_update_tile(double2* G, int64_t ldg, int64_t n, int pmax, int p, const cplx* C0,
                                                const cplx* S, int64_t rt, int64_t ct) {
  const int64_t j = ct * 256 + threadIdx.x;       // 256 threads: one column each
  if (j >= n || threadIdx.x >= 256) return;
  const int64_t i0 = rt * kF64BatchRows, i1 = i0 + kF64BatchRows < n ? i0 + kF64BatchRows : n;
  switch (p) {
    case 1: f64_update_rows<1>(G, ldg, n, i0, i1, pmax, p, C0, S, j); break;
    case 2: f64_update_rows<2>(G, ldg, n, i0, i1, pmax, p, C0, S, j); break;
    case 3: f64_update_rows<3>(G, ldg, n, i0, i1, pmax, p, C0, S, j); break;
    case 4: f64_update_rows<4>(G, ldg, n, i0, i1, pmax, p, C0, S, j); break;
    default: f64_update_rows<0>(G, ldg, n, i0, i1, pmax, p, C0, S, j); break;
  }
}

// complex64 storage, rank p <= 4, FP32 arithmetic on the CUDA cores: the update is a pure
// HBM stream (4p FP32 FMA per 16 bytes moved), so no tensor-core form is needed.  A tile is
// 32 rows x 512 complex columns; each thread owns two adjacent columns (one 16-byte vector per
// row) and keeps their S entries in registers; the tile's C0 rows are staged in shared memory.
// G is touched once per step, so its loads and stores carry the streaming (evict-first) hint
// and leave L2 to the panels.  Three CTAs fit an SM; launches use a multiple of that.
constexpr int kF32Threads = 256;
constexpr int kF32Rows = 32;
constexpr int kF32Cols = 2 * kF32Threads;

template <int R = kF32Rows>
__device__ __forceinline__ void c64_fp32_tile(float2* __restrict__ G, int64_t ldg, int64_t n, int64_t m, int pmax, int p,
                                              const cplx* C0, const cplx* S,
                                              int64_t rt, int64_t ct, float2 (*sC)[kC64Fp32MaxP]) {
  // R: rows of the tile (the tuned batch kernel instantiates 16, 32 and 64)
  const int64_t i0 = rt * R;
  const int64_t j = ct * kF32Cols + 2 * threadIdx.x;
  __syncthreads();                                   // previous tile done with sC
  for (int t = threadIdx.x; t < R * kC64Fp32MaxP; t += kF32Threads) {
    const int r = t / kC64Fp32MaxP, u = t % kC64Fp32MaxP;
    const int64_t i = i0 + r;
    cplx c = (i < m && u < p) ? C0[i * pmax + u] : mk(0.0, 0.0);
    sC[r][u] = make_float2((float)c.re, (float)c.im);
  }
  __syncthreads();
  if (j >= n) return;
  const bool two = j + 1 < n;
  float2 s0[kC64Fp32MaxP], s1[kC64Fp32MaxP];
#pragma unroll
  for (int u = 0; u < kC64Fp32MaxP; ++u) {
    cplx a = u < p ? S[(int64_t)u * n + j] : mk(0.0, 0.0);
    cplx b = (u < p && two) ? S[(int64_t)u * n + j + 1] : mk(0.0, 0.0);
    s0[u] = make_float2((float)a.re, (float)a.im);
    s1[u] = make_float2((float)b.re, (float)b.im);
  }
  const int rows = (int)(m - i0 < R ? m - i0 : R);
  constexpr int U = 8;
  for (int r0 = 0; r0 < rows; r0 += U) {
    float4 g[U];
#pragma unroll
    for (int q = 0; q < U; ++q)
      if (r0 + q < rows) g[q] = __ldcs(reinterpret_cast<const float4*>(G + (i0 + r0 + q) * ldg + j));
#pragma unroll
    for (int q = 0; q < U; ++q) {
      if (r0 + q < rows) {
        float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
#pragma unroll
        for (int u = 0; u < kC64Fp32MaxP; ++u) {
          const float2 c = sC[r0 + q][u];
          ar = fmaf(c.x, s0[u].x, fmaf(-c.y, s0[u].y, ar));
          ai = fmaf(c.x, s0[u].y, fmaf(c.y, s0[u].x, ai));
          br = fmaf(c.x, s1[u].x, fmaf(-c.y, s1[u].y, br));
          bi = fmaf(c.x, s1[u].y, fmaf(c.y, s1[u].x, bi));
        }
        float4 v = g[q];
        v.x += ar;
        v.y += ai;
        if (two) {
          v.z += br;
          v.w += bi;
        }
        __stcs(reinterpret_cast<float4*>(G + (i0 + r0 + q) * ldg + j), v);
      }
    }
  }
}

// ----------------------------------------------------------------------------- field, state, FOM
__device__ __forceinline__ void finish_body(const UpdArgs& a, const WsLayout& L, char* ws, uint8_t* __restrict__ state,
                                            double* __restrict__ fom_out, int32_t* __restrict__ applied, int64_t vb = -1, int64_t vg = -1) {
  // vb, vg: a virtual block index and count (a work item of a persistent kernel); -1: the grid's
  const int64_t vb_ = vb < 0 ? (int64_t)blockIdx.x : vb, vg_ = vg < 0 ? (int64_t)gridDim.x : vg;
  const UpdCtl* ctl = reinterpret_cast<const UpdCtl*>(ws + L.ctl);
  const int64_t n = L.n;
  const int64_t N = n - 1;
  const bool skip = ctl->skip != 0;
  const int p = skip ? 0 : ctl->nv;
  const int32_t* V = reinterpret_cast<const int32_t*>(ws + L.V);
  (void)N;
  for (int64_t i = vb_ * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)vg_ * blockDim.x) {
    // the first monitor unknown's thread also updates the others, so that it can sum the FOM
    if (i > a.mrow && i < a.mrow + a.mcount) continue;
    const int reps = i == a.mrow ? a.mcount : 1;
    double f = 0.0;
    for (int q = 0; q < reps; ++q) {
      const int64_t ii = i + q;
      for (int l = 0; l < a.nlam; ++l) {
        const cplx* C0 = reinterpret_cast<const cplx*>(ws + L.C0 + l * L.panel_s);
        const cplx* yd = reinterpret_cast<const cplx*>(ws + L.yd + l * L.yd_s);
        const UpdLam& U = a.lam[l];
        cplx e = U.E[ii];
        if (U.vrows)        // G[ii, V[u]] read as G[V[u], ii] from the row panel (reciprocity)
          for (int u = 0; u < p; ++u) e = cfma(ldG(U.vrows, a.dtype, U.ldv, u, ii), yd[u], e);
        else
          for (int u = 0; u < p; ++u) e = cfma(C0[ii * L.pmax + u], yd[u], e);
        if (p > 0) a.lam[l].E[ii] = e;
        f += abs2(e);
      }
    }
    if (i == a.mrow) {
      *fom_out = f;
      if (applied) *applied = skip ? 0 : ctl->ncand;
    }
  }
  if (vb_ == 0) {   // one flip per point (the unknowns of a point are consecutive in V)
    for (int t = threadIdx.x; t < p; t += blockDim.x)
      if (V[t] % a.ncomp == 0) state[V[t] / a.ncomp] ^= 1;
  }
}

}  // namespace gf
