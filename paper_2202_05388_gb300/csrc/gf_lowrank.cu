// Deferred (low-rank) form of the greedy step: G is never materialised.
//
// Eq. 10 applied step after step gives G_t = G0 + sum_s C_s D_s R_s with C_s = G_s[:, V_s] and
// R_s = A_s^{-1} G_s[V_s, :] (Eq. 14).  G is symmetric (reciprocity of the scalar Green's
// function; the update preserves it), so G_s[V_s, :] = C_s^T and every term is
// C_s M_s C_s^T with the p_s x p_s block M_s = D_s A_s^{-1}.  The state of a problem is then
//   * G0 implicitly: its table of values by pixel offset plus the monitor column (gf_fill_g0's
//     table, kept in the workspace);
//   * the stored columns C_s (n x sum p_s, column-major) and blocks M_s;
//   * the data candidate evaluation reads, kept explicit: the nine bands (G_VV blocks of
//     Eq. 8), the monitor row G[N, :] and the field E.
// A step computes the p new columns G[:, V] = G0[:, V] + sum_s C_s (M_s C_s[V, :]^T) (an n x K
// by K x p product, K = columns stored), solves the p x p capacitance system (Eqs. 8-9, 14),
// appends the term and updates bands, monitor row and E by O(n p) work (Eqs. 10 and 4
// restricted to those entries).  Memory is O(n K) instead of O(n^2).
#include <math.h>

#include <atomic>

#include "gf_internal.cuh"

namespace gf {

constexpr int kLrP = 4;            // pixels per candidate at most (2x2 brush)
constexpr int kLrPMax = 32;        // pixels per step at most (k candidates: k p <= 32)
constexpr int kLrSlices = 16;      // slices x column groups of the column product, at most

struct LrCount {
  int32_t nterms, ncols, ncoef, pad;
};

// Per-step scratch written by the pixel / capacitance kernels.
struct LrStep {
  int32_t skip, p, col0, p1;     // p1: pixels of the best candidate (the set applied alone on fallback)
  int32_t ncand, pad[3];         // candidates applied
  int32_t V[kLrPMax];
  double dchi[kLrPMax];
  cplx dy[kLrPMax];              // D y, y = A^{-1} E_V
  cplx M[kLrPMax * kLrPMax];     // D A^{-1}, row-major p x p (stride p)
};

// workspace layout: G0 table (2N) | M blocks (packed, p_s x p_s per term) | term first column |
// term width | term block offset | column -> term | counters | step | w (K x kLrPMax) | partial
// columns of the column product (kLrSlices x 4 x n)
struct LrLayout {
  size_t table, coef, tcol, tp, tco, colterm, count, step, w, part, total;
};

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

static LrLayout lr_layout(const gf_geom& g, int max_cols) {
  const int64_t N = (int64_t)g.nx * g.ny;
  LrLayout L;
  size_t o = 0;
  L.table = o; o = up256(o + sizeof(cplx) * (size_t)(2 * N));
  L.coef = o; o = up256(o + sizeof(cplx) * kLrPMax * (size_t)max_cols);   // sum of p_s^2 <= kLrPMax K
  L.tcol = o; o = up256(o + sizeof(int32_t) * (size_t)max_cols);
  L.tp = o; o = up256(o + sizeof(int32_t) * (size_t)max_cols);
  L.tco = o; o = up256(o + sizeof(int32_t) * (size_t)max_cols);
  L.colterm = o; o = up256(o + sizeof(int32_t) * (size_t)max_cols);
  L.count = o; o = up256(o + sizeof(LrCount));
  L.step = o; o = up256(o + sizeof(LrStep));
  L.w = o; o = up256(o + sizeof(cplx) * kLrPMax * (size_t)max_cols);
  L.part = o; o = up256(o + sizeof(cplx) * kLrSlices * kLrP * (size_t)(N + 1));
  L.total = o;
  return L;
}

struct LrArgs {
  int nx, ny;
  int64_t N, n;
  double chi;
  int max_cols;
  cplx* E;
  cplx* bands;
  cplx* mon;
  cplx* U;
  const cplx* table;
  cplx* coef;
  int32_t* tcol;
  int32_t* tp;
  int32_t* tco;
  int32_t* colterm;
  LrCount* count;
  LrStep* step;
  cplx* w;
  cplx* part;
};

// G0[i, j] of a pixel column j (i may be the monitor N)
__device__ __forceinline__ cplx g0_entry(const LrArgs& a, int64_t i, int64_t j) {
  if (i == a.N) return a.table[a.N + j];
  const int iy = (int)(i / a.nx), ix = (int)(i - (int64_t)iy * a.nx);
  const int jy = (int)(j / a.nx), jx = (int)(j - (int64_t)jy * a.nx);
  const int dy = iy > jy ? iy - jy : jy - iy, dx = ix > jx ? ix - jx : jx - ix;
  return a.table[(int64_t)dy * a.nx + dx];
}

// ---- initial state: bands, monitor row and field of the vacuum background; no terms
__global__ void k_lr_init(LrArgs a) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < GF_NBANDS * a.N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / a.N);
    const int64_t i = t - (int64_t)b * a.N;
    const int iy = (int)(i / a.nx), ix = (int)(i % a.nx);
    int ddx, ddy;
    band_offset(b, ddx, ddy);
    const int jx = ix + ddx, jy = iy + ddy;
    cplx v = mk(0.0, 0.0);
    if (jx >= 0 && jx < a.nx && jy >= 0 && jy < a.ny) v = a.table[(int64_t)(ddy < 0 ? -ddy : ddy) * a.nx + (ddx < 0 ? -ddx : ddx)];
    a.bands[t] = v;
  }
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.n; j += (int64_t)gridDim.x * blockDim.x)
    a.mon[j] = j < a.N ? a.table[a.N + j] : mk(0.0, 0.0);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.count->nterms = 0;
    a.count->ncols = 0;
    a.count->ncoef = 0;
  }
}

// ---- the chosen candidates' pixels, in selection order (device status and capacity checks)
__global__ void k_lr_pixels(LrArgs a, int kind, int dir_mask, const uint8_t* __restrict__ state,
                            const int32_t* __restrict__ idx, int k, int32_t* status) {
  if (threadIdx.x != 0) return;
  LrStep* s = a.step;
  s->skip = 1;
  s->p = 0;
  s->ncand = 0;
  if (*status != GF_OK || idx[0] < 0) return;
  int p = 0, nc = 0, p1 = 0;
  for (int c = 0; c < k; ++c) {
    if (idx[c] < 0) break;
    const int m = cand_pixels(idx[c], kind, dir_mask, a.nx, a.ny, a.chi, state, s->V + p, s->dchi + p);
    if (m == 0) continue;
    if (nc == 0) p1 = m;
    p += m;
    ++nc;
  }
  if (p == 0) return;
  const LrCount c = *a.count;
  if (c.ncols + p > a.max_cols || c.nterms + 1 > a.max_cols || c.ncoef + p * p > kLrPMax * a.max_cols) {
    *status = GF_ENOMEM;        // term storage full: materialise (gf_lowrank_materialize) and restart
    return;
  }
  s->p = p;
  s->p1 = p1;
  s->ncand = nc;
  s->col0 = c.ncols;
  s->skip = 0;
}

// ---- w[k][u] = (M_s C_s[v_u, :]^T)_a for stored column k = first column of term s + a
__global__ void k_lr_w(LrArgs a) {
  const LrStep* s = a.step;
  if (s->skip) return;
  const int p = s->p;
  const int K = s->col0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t info = a.colterm[k];
    const int term = info >> 5, row = info & 31;
    const int c0 = a.tcol[term], pt = a.tp[term];
    const cplx* M = a.coef + a.tco[term];
    for (int u = 0; u < p; ++u) {
      cplx acc = mk(0.0, 0.0);
      for (int b = 0; b < pt; ++b) acc = cfma(M[row * pt + b], a.U[(int64_t)(c0 + b) * a.n + s->V[u]], acc);
      a.w[(int64_t)k * kLrPMax + u] = acc;
    }
  }
}

// ---- the p new columns: C[:, u] = G0[:, v_u] + sum_k U[:, k] w[k][u], appended to U
//
// The product runs on the FP32 pipe in double-float arithmetic (a value is an unevaluated sum
// hi + lo of two floats, about 48 bits): GB300's FP64 pipe runs at 1/64 of the FP32 rate, and the
// FP64 form of this product kept it 97% busy.  Each FP64 entry of U and w is split into hi (its
// sign, exponent and first 23 mantissa bits) and lo (the remaining 29 bits, rounded to a float)
// with integer and FP32 operations only; products use the error-free product of Dekker (the rounding
// error of hi*hi from one FMA) plus the two cross terms, and sums use Knuth's error-free sum and a
// renormalisation.  Every step is an _rn intrinsic, so the compiler cannot contract the sums into
// FMAs (which would lose the error terms).  The result is converted back to FP64 once per entry.
// Per multiply-add the error is about 2^-47 of the magnitudes involved; the columns agree with the
// FP64 form to about 1e-13 relative over a whole run.
struct dflt {
  float h, l;
};

__device__ __forceinline__ dflt df_split(double x) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned sgn = (unsigned)((unsigned long long)b >> 63) << 31;
  // hi: sign, exponent and the first 23 mantissa bits, exact for |x| in [2^-126, 2^128); below
  // that 0, above it inf.  Only integer and FP32 operations: a branch to a conversion would be
  // predicated into every split and keep GB300's narrow FP64 pipe busy.
  const unsigned hb = e < 897 ? sgn
                    : e > 1150 ? (sgn | 0x7F800000u)
                               : (sgn | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7FFFFF));
  // lo = (low 29 mantissa bits) * 2^(e - 1075), with the sign of x, rounded once: the 29-bit
  // integer's high 23 and low 6 bits become exact floats through the 2^23 bias and one FMA joins
  // them.  Where 2^(e - 1075) is not a normal float (|x| < 2^-74) lo is 0: an absolute error
  // below 2^-97 |x|.
  const unsigned m29 = (unsigned)(b & 0x1FFFFFFF);
  const float fa = __fsub_rn(__uint_as_float(0x4B000000u | (m29 >> 6)), 8388608.0f);
  const float fb = __fsub_rn(__uint_as_float(0x4B000000u | (m29 & 63u)), 8388608.0f);
  const int se = (e < 949 || e > 1150) ? 0 : e - 948;          // biased exponent of 2^(e - 1075)
  const float l = __fmul_rn(__fmaf_rn(fa, 64.0f, fb), __uint_as_float((unsigned)se << 23));
  return {__uint_as_float(hb), sgn ? -l : l};
}

__device__ __forceinline__ double df_to(dflt a) { return (double)a.h + (double)a.l; }

// c += a b
__device__ __forceinline__ void df_fma(dflt& c, dflt a, dflt b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float s = __fadd_rn(c.h, p);
  const float bb = __fsub_rn(s, c.h);
  float t = __fadd_rn(__fsub_rn(c.h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  t = __fadd_rn(t, __fadd_rn(c.l, e));
  const float hs = __fadd_rn(s, t);
  c.l = __fsub_rn(t, __fsub_rn(hs, s));
  c.h = hs;
}

__device__ __forceinline__ dflt df_neg(dflt a) { return {-a.h, -a.l}; }

constexpr int kLrThreads = 256;
constexpr int kLrChunk = 256;      // stored columns per shared-memory chunk of w
// Split over the stored columns: blockIdx.y takes slice y of [0, K) (gridDim.y slices; slice 0
// also starts from the G0 column) and writes its partial columns to part[y]; k_lr_columns_sum adds
// the slices in FP64 in a fixed order, so the result does not depend on scheduling.  One row block
// per CTA alone leaves most of the GPU idle at n ~ 4e4 (145 CTAs).  blockIdx.z takes the step's
// new columns 4 z .. 4 z + 3 (several candidates per step).
__global__ void __launch_bounds__(kLrThreads) k_lr_columns(LrArgs a, int32_t* __restrict__ prof) {
  const LrStep* s = a.step;
  if (prof && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
    *prof = s->skip ? 0 : s->col0 * s->p;
  if (s->skip) return;
  __shared__ float4 sw[kLrChunk * kLrP];       // w[k][u] as (re.h, re.l, im.h, im.l)
  const int u0 = (int)blockIdx.z * kLrP;       // the group's first new column
  if (u0 >= s->p) return;
  const int p = s->p - u0 < kLrP ? s->p - u0 : kLrP;
  const int K = s->col0;
  const int S = (int)gridDim.y, y = (int)blockIdx.y;
  const int gz = (int)blockIdx.z, G = (int)gridDim.z;
  const int Ks = (K + S - 1) / S;
  const int kb = y * Ks < K ? y * Ks : K;
  const int ke = kb + Ks < K ? kb + Ks : K;
  int V[kLrP];
#pragma unroll
  for (int u = 0; u < kLrP; ++u) V[u] = u < p ? s->V[u0 + u] : 0;
  for (int64_t i0 = (int64_t)blockIdx.x * kLrThreads; i0 < a.n; i0 += (int64_t)gridDim.x * kLrThreads) {
    const int64_t i = i0 + threadIdx.x;
    dflt ar[kLrP], ai[kLrP];
#pragma unroll
    for (int u = 0; u < kLrP; ++u) {
      const cplx g = (y == 0 && i < a.n && u < p) ? g0_entry(a, i, V[u]) : mk(0.0, 0.0);
      ar[u] = df_split(g.re);
      ai[u] = df_split(g.im);
    }
    for (int k0 = kb; k0 < ke; k0 += kLrChunk) {
      const int kc = ke - k0 < kLrChunk ? ke - k0 : kLrChunk;
      __syncthreads();
      for (int t = threadIdx.x; t < kc * kLrP; t += kLrThreads) {
        const int uu = t & (kLrP - 1);
        const cplx w = uu < p ? a.w[(int64_t)(k0 + (t >> 2)) * kLrPMax + u0 + uu] : mk(0.0, 0.0);
        const dflt wr = df_split(w.re), wi = df_split(w.im);
        sw[t] = make_float4(wr.h, wr.l, wi.h, wi.l);
      }
      __syncthreads();
      if (i < a.n) {
        for (int k = 0; k < kc; ++k) {
          const cplx uk = a.U[(int64_t)(k0 + k) * a.n + i];
          const dflt ur = df_split(uk.re), ui = df_split(uk.im), nui = df_neg(ui);
#pragma unroll
          for (int u = 0; u < kLrP; ++u) {
            if (u < p) {
              const float4 w4 = sw[k * kLrP + u];
              const dflt wr = {w4.x, w4.y}, wi = {w4.z, w4.w};
              df_fma(ar[u], ur, wr);         // Re: ur wr - ui wi
              df_fma(ar[u], nui, wi);
              df_fma(ai[u], ur, wi);         // Im: ur wi + ui wr
              df_fma(ai[u], ui, wr);
            }
          }
        }
      }
    }
    if (i < a.n) {
#pragma unroll
      for (int u = 0; u < kLrP; ++u)
        if (u < p) a.part[(((int64_t)y * G + gz) * kLrP + u) * a.n + i] = mk(df_to(ar[u]), df_to(ai[u]));
    }
  }
}

// C[:, u] = sum of the slices' partial columns (FP64, slice order), appended to U
__global__ void k_lr_columns_sum(LrArgs a, int S, int G) {
  const LrStep* s = a.step;
  if (s->skip) return;
  const int p = s->p;
  const int K = s->col0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)p * a.n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int u = (int)(t / a.n);
    const int64_t i = t - (int64_t)u * a.n;
    const int g = u / kLrP, uu = u - g * kLrP;
    cplx acc = a.part[((int64_t)g * kLrP + uu) * a.n + i];
    for (int y = 1; y < S; ++y) acc = acc + a.part[(((int64_t)y * G + g) * kLrP + uu) * a.n + i];
    a.U[(int64_t)(K + u) * a.n + i] = acc;
  }
}

// ---- capacitance: A = I - G_VV D from the new columns, y = A^{-1} E_V, M = D A^{-1} (one CTA:
// Gaussian elimination with partial pivoting on [A | I | E_V], one thread picks each pivot (largest
// |a| as in the candidate kernels, first on ties) and forms the rows' multipliers, every element is
// then updated by its own thread; the back substitution runs column by column over all right-hand
// sides at once).  Several candidates: applied jointly only if the joint dFOM is positive, else
// the best candidate alone (its columns lead the new ones).
__global__ void __launch_bounds__(256) k_lr_capacitance(LrArgs a, int32_t* status) {
  LrStep* s = a.step;
  if (s->skip) return;
  __shared__ cplx A[kLrPMax][kLrPMax];
  __shared__ cplx X[kLrPMax][kLrPMax + 1];
  __shared__ cplx F[kLrPMax];
  __shared__ double s_norm;
  __shared__ int s_piv, s_bad, s_p, s_redo;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int K = s->col0;
  if (tid == 0) { s_p = s->p; s_redo = 0; }
  __syncthreads();
  for (int attempt = 0; attempt < 2; ++attempt) {
    const int p = s_p;
    for (int t = tid; t < p * p; t += nt) {
      const int r = t / p, c = t - r * p;
      const cplx g = a.U[(int64_t)(K + c) * a.n + s->V[r]];      // G[v_r, v_c]
      A[r][c] = mk(r == c ? 1.0 : 0.0, 0.0) - s->dchi[c] * g;
      X[r][c] = mk(r == c ? 1.0 : 0.0, 0.0);
    }
    for (int r = tid; r < p; r += nt) X[r][p] = a.E[s->V[r]];
    __syncthreads();
    if (tid == 0) {
      double norm = 0.0;
      for (int r = 0; r < p; ++r) {
        double rs = 0.0;
        for (int c = 0; c < p; ++c) rs += cabs1(A[r][c]);
        norm = fmax(norm, rs);
      }
      s_norm = norm;
      s_bad = 0;
    }
    __syncthreads();
    const double thresh = kSingularRel * s_norm;
    for (int c = 0; c < p; ++c) {
      if (tid == 0) {
        int piv = c;
        double best = cabs1(A[c][c]);
        for (int r = c + 1; r < p; ++r)
          if (cabs1(A[r][c]) > best) { best = cabs1(A[r][c]); piv = r; }
        s_piv = piv;
        if (!(best >= thresh) || !(best > 0.0)) s_bad = 1;
      }
      __syncthreads();
      if (s_bad) break;
      const int piv = s_piv;
      if (piv != c) {
        for (int v = tid; v < p; v += nt) { const cplx t0 = A[c][v]; A[c][v] = A[piv][v]; A[piv][v] = t0; }
        for (int v = tid; v <= p; v += nt) { const cplx t0 = X[c][v]; X[c][v] = X[piv][v]; X[piv][v] = t0; }
      }
      for (int r = c + 1 + tid; r < p; r += nt) F[r] = cdiv(A[r][c], A[c][c]);
      __syncthreads();
      // row r >= c + 1: a_rv -= f_r a_cv (v >= c), x_rv -= f_r x_cv
      const int w = 2 * p + 1 - c;               // columns c..p-1 of A, then 0..p of X
      for (int t = tid; t < (p - 1 - c) * w; t += nt) {
        const int r = c + 1 + t / w, q = t - (t / w) * w;
        const cplx f = F[r];
        if (q < p - c) {
          const int v = c + q;
          A[r][v] = A[r][v] - f * A[c][v];
        } else {
          const int v = q - (p - c);
          X[r][v] = X[r][v] - f * X[c][v];
        }
      }
      __syncthreads();
    }
    if (s_bad) {
      if (tid == 0) {
        *status = GF_ESINGULAR;
        s->skip = 1;
      }
      return;
    }
    // back substitution, column by column from the bottom, every right-hand side at once
    for (int c = p - 1; c >= 0; --c) {
      for (int v = tid; v <= p; v += nt) X[c][v] = cdiv(X[c][v], A[c][c]);
      __syncthreads();
      for (int t = tid; t < c * (p + 1); t += nt) {
        const int r = t / (p + 1), v = t - r * (p + 1);
        X[r][v] = X[r][v] - A[r][c] * X[c][v];
      }
      __syncthreads();
    }
    if (attempt == 0 && s->ncand > 1) {           // the joint decision (Eq. 4 at the monitor)
      if (tid == 0) {
        cplx dE = mk(0.0, 0.0);
        for (int u = 0; u < p; ++u)
          dE = dE + s->dchi[u] * (a.U[(int64_t)(K + u) * a.n + a.N] * X[u][p]);
        const cplx EN = a.E[a.N];
        const double joint = abs2(EN + dE) - abs2(EN);
        if (!(joint > 0.0)) {
          s_p = s->p1;
          s_redo = 1;
        }
      }
      __syncthreads();
      if (s_redo) continue;
    }
    break;
  }
  const int p = s_p;
  const int term = a.count->nterms;
  const int off = a.count->ncoef;
  cplx* M = a.coef + off;
  for (int t = tid; t < p * p; t += nt) {
    const int r = t / p, c = t - r * p;
    const cplx m = s->dchi[r] * X[r][c];
    M[t] = m;
    s->M[t] = m;
  }
  for (int r = tid; r < p; r += nt) {
    s->dy[r] = s->dchi[r] * X[r][p];
    a.colterm[K + r] = (term << 5) | r;
  }
  __syncthreads();
  if (tid == 0) {
    if (s_redo) s->ncand = 1;
    s->p = p;
    a.tcol[term] = K;
    a.tp[term] = p;
    a.tco[term] = off;
    a.count->nterms = term + 1;
    a.count->ncols = K + p;
    a.count->ncoef = off + p * p;
  }
}

// ---- Eq. 10 on the explicit entries (bands, monitor row) and Eq. 4 on E; state, FOM.  PM bounds
// the step's p (4: one candidate, held in registers; kLrPMax: several, M and q_N in shared memory)
template <int PM>
__global__ void __launch_bounds__(256) k_lr_apply(LrArgs a, uint8_t* __restrict__ state, double* __restrict__ fom_out,
                                                  int32_t* __restrict__ applied) {
  const LrStep* s = a.step;
  const bool skip = s->skip != 0;
  const int p = skip ? 0 : s->p;
  const int K = s->col0;
  const cplx* C = a.U + (int64_t)K * a.n;        // the new columns, C[u * n + i]
  __shared__ cplx sM[PM * PM];
  __shared__ cplx sq[PM];
  __shared__ cplx sdy[PM];
  for (int t = threadIdx.x; t < PM * PM; t += blockDim.x) {
    const int r = t / PM, c = t - r * PM;
    sM[t] = (r < p && c < p) ? s->M[r * p + c] : mk(0.0, 0.0);
  }
  for (int c = threadIdx.x; c < PM; c += blockDim.x) sdy[c] = c < p ? s->dy[c] : mk(0.0, 0.0);
  __syncthreads();
  // q_N = C[N, :] M (row vector) for the monitor row
  for (int c = threadIdx.x; c < PM; c += blockDim.x) {
    cplx q = mk(0.0, 0.0);
    for (int r = 0; r < p; ++r) q = cfma(C[(int64_t)r * a.n + a.N], sM[r * PM + c], q);
    sq[c] = q;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    if (p > 0) {
      cplx ri[PM], qi[PM];
#pragma unroll
      for (int u = 0; u < PM; ++u) ri[u] = u < p ? C[(int64_t)u * a.n + i] : mk(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < PM; ++c) {
        qi[c] = mk(0.0, 0.0);
        if (c < p)
#pragma unroll
          for (int r = 0; r < PM; ++r)
            if (r < p) qi[c] = cfma(ri[r], sM[r * PM + c], qi[c]);
      }
      cplx e = a.E[i];
      for (int u = 0; u < p; ++u) e = cfma(ri[u], sdy[u], e);
      a.E[i] = e;
      cplx dm = mk(0.0, 0.0);
      for (int c = 0; c < p; ++c) dm = cfma(sq[c], ri[c], dm);
      a.mon[i] = a.mon[i] + dm;
      if (i < a.N) {
        const int iy = (int)(i / a.nx), ix = (int)(i % a.nx);
        for (int b = 0; b < GF_NBANDS; ++b) {
          int ddx, ddy;
          band_offset(b, ddx, ddy);
          const int jx = ix + ddx, jy = iy + ddy;
          if (jx < 0 || jx >= a.nx || jy < 0 || jy >= a.ny) continue;
          const int64_t j = (int64_t)jy * a.nx + jx;
          cplx d = mk(0.0, 0.0);
#pragma unroll
          for (int c = 0; c < PM; ++c)
            if (c < p) d = cfma(qi[c], C[(int64_t)c * a.n + j], d);
          a.bands[(int64_t)b * a.N + i] = a.bands[(int64_t)b * a.N + i] + d;
        }
      }
    }
    if (i == a.N) {
      *fom_out = abs2(a.E[a.N]);
      if (applied) *applied = p > 0 ? s->ncand : 0;
    }
  }
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t < p; t += blockDim.x) state[s->V[t]] ^= 1;
}

// ---- dense G = G0 + sum_s C_s M_s C_s^T (checks and flushes; O(n^2 K))
__global__ void k_lr_materialize(LrArgs a, double2* __restrict__ G, int64_t ldg) {
  const int K = a.count->ncols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.n * a.n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / a.n, j = t - i * a.n;
    cplx v;
    if (i == a.N && j == a.N) v = mk(0.0, 0.0);
    else if (j == a.N) v = g0_entry(a, j, i);
    else v = g0_entry(a, i, j);
    for (int k = 0; k < K; ++k) {
      const int32_t info = a.colterm[k];
      const int term = info >> 5, row = info & 31;
      const int c0 = a.tcol[term], pt = a.tp[term];
      const cplx* M = a.coef + a.tco[term];
      cplx mj = mk(0.0, 0.0);
      for (int b = 0; b < pt; ++b) mj = cfma(M[row * pt + b], a.U[(int64_t)(c0 + b) * a.n + j], mj);
      v = cfma(a.U[(int64_t)k * a.n + i], mj, v);
    }
    G[i * ldg + j] = make_double2(v.re, v.im);
  }
}

static LrArgs lr_args(const gf_lowrank& lr, char* ws) {
  const LrLayout L = lr_layout(lr.geom, lr.max_cols);
  LrArgs a;
  a.nx = lr.geom.nx;
  a.ny = lr.geom.ny;
  a.N = (int64_t)a.nx * a.ny;
  a.n = a.N + 1;
  a.chi = lr.geom.eps_mat - lr.geom.eps_bg;
  a.max_cols = lr.max_cols;
  a.E = reinterpret_cast<cplx*>(lr.E);
  a.bands = reinterpret_cast<cplx*>(lr.bands);
  a.mon = reinterpret_cast<cplx*>(lr.monrow);
  a.U = reinterpret_cast<cplx*>(lr.U);
  a.table = reinterpret_cast<const cplx*>(ws + L.table);
  a.coef = reinterpret_cast<cplx*>(ws + L.coef);
  a.tcol = reinterpret_cast<int32_t*>(ws + L.tcol);
  a.tp = reinterpret_cast<int32_t*>(ws + L.tp);
  a.tco = reinterpret_cast<int32_t*>(ws + L.tco);
  a.colterm = reinterpret_cast<int32_t*>(ws + L.colterm);
  a.count = reinterpret_cast<LrCount*>(ws + L.count);
  a.step = reinterpret_cast<LrStep*>(ws + L.step);
  a.w = reinterpret_cast<cplx*>(ws + L.w);
  a.part = reinterpret_cast<cplx*>(ws + L.part);
  return a;
}

static int grid_of(int64_t work, int threads, int cap) {
  int64_t b = (work + threads - 1) / threads;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace gf

// ----------------------------------------------------------------------------- C ABI
static gf_status lr_check(gf_handle* h, const gf_lowrank* lr, void* ws, size_t ws_bytes) {
  if (!lr) return gf::api_fail_msg(h, GF_EINVAL, "low-rank problem is NULL");
  gf_problem probe;
  probe.geom = lr->geom;
  probe.G = lr->monrow;          // shape checks only: the monitor row stands in for G
  const int64_t n = (int64_t)lr->geom.nx * lr->geom.ny + 1;
  probe.ldg = n + (n & 1);
  probe.E = lr->E;
  probe.bands = lr->bands;
  gf_status s = gf::api_check_problem(h, &probe, GF_C128);
  if (s) return s;
  if (!lr->U || ((uintptr_t)lr->U & 15u)) return gf::api_fail_msg(h, GF_EINVAL, "U must be non-NULL and 16-byte aligned");
  if (lr->max_cols < 4 || lr->max_cols > (1 << 24)) return gf::api_fail_msg(h, GF_EINVAL, "max_cols must lie in [4, 2^24]");
  if (!ws || ((uintptr_t)ws & 255u)) return gf::api_fail_msg(h, GF_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < gf::lr_layout(lr->geom, lr->max_cols).total) return gf::api_fail_msg(h, GF_ENOMEM, "workspace too small");
  return gf::api_bind_device(h);
}

extern "C" {

size_t gf_lowrank_workspace_size(const gf_geom* geom, int32_t max_cols) {
  if (!geom || geom->nx < 1 || geom->ny < 1 || max_cols < 4 || max_cols > (1 << 24)) return 0;
  return gf::lr_layout(*geom, max_cols).total;
}

gf_status gf_lowrank_init(gf_handle* h, const gf_lowrank* lr, void* ws, size_t ws_bytes, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = lr_check(h, lr, ws, ws_bytes);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  gf::LrArgs a = gf::lr_args(*lr, reinterpret_cast<char*>(ws));
  gf::launch_fill_table(lr->geom, const_cast<gf::cplx*>(a.table), st);
  gf::launch_fill_field(lr->geom, a.E, st);
  gf::k_lr_init<<<gf::grid_of(GF_NBANDS * a.N, 256, 4864), 256, 0, st>>>(a);
  return gf::api_cuda_check(h, "gf_lowrank_init launch");
}

gf_status gf_lowrank_fom(gf_handle* h, const gf_lowrank* lr, double* fom_out, void* stream) {
  if (!h) return GF_EINVAL;
  if (!lr) return gf::api_fail_msg(h, GF_EINVAL, "low-rank problem is NULL");
  if (!lr->E || ((uintptr_t)lr->E & 15u)) return gf::api_fail_msg(h, GF_EINVAL, "E must be non-NULL and 16-byte aligned");
  if (lr->geom.nx < 1 || lr->geom.ny < 1) return gf::api_fail_msg(h, GF_EINVAL, "nx, ny must be >= 1");
  if (!fom_out) return gf::api_fail_msg(h, GF_EINVAL, "fom_out must be non-NULL");
  gf_status s = gf::api_bind_device(h);
  if (s) return s;
  gf::FomArgs a;
  a.nlam = 1;
  a.ncomp = 1;
  a.mrow = (int64_t)lr->geom.nx * lr->geom.ny;
  a.E[0] = reinterpret_cast<const gf::cplx*>(lr->E);
  gf::launch_fom(a, fom_out, (cudaStream_t)stream);
  return gf::api_cuda_check(h, "gf_lowrank_fom launch");
}

gf_status gf_lowrank_eval(gf_handle* h, const gf_lowrank* lr, const uint8_t* state, const gf_cand_spec* spec,
                          double* dfom, void* stream) {
  if (!h) return GF_EINVAL;
  if (!lr) return gf::api_fail_msg(h, GF_EINVAL, "low-rank problem is NULL");
  if (!state || !dfom || !spec) return gf::api_fail_msg(h, GF_EINVAL, "state, spec and dfom must be non-NULL");
  gf_status s = gf::api_check_spec(h, &lr->geom, spec);
  if (s) return s;
  if ((s = gf::api_bind_device(h))) return s;
  // the candidate kernels read bands, E and the monitor row G[N, j]: a one-row "G" with
  // leading dimension 0 makes G[N * 0 + j] the monitor row
  gf::EvalArgs a;
  a.nlam = 1;
  a.dtype = GF_C128;
  a.nx = lr->geom.nx;
  a.ny = lr->geom.ny;
  a.chi = lr->geom.eps_mat - lr->geom.eps_bg;
  a.c_begin = 0;
  a.c_end = -1;
  a.lam[0].G = lr->monrow;
  a.lam[0].ldg = 0;
  a.lam[0].E = reinterpret_cast<const gf::cplx*>(lr->E);
  a.lam[0].bands = reinterpret_cast<const gf::cplx*>(lr->bands);
  gf::launch_eval(a, state, *spec, dfom, (cudaStream_t)stream);
  return gf::api_cuda_check(h, "gf_lowrank_eval launch");
}

gf_status gf_lowrank_update(gf_handle* h, const gf_lowrank* lr, uint8_t* state, const gf_cand_spec* spec,
                            const int32_t* idx, int32_t* status, double* fom_out, int32_t* applied, void* ws,
                            size_t ws_bytes, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = lr_check(h, lr, ws, ws_bytes);
  if (s) return s;
  if (!spec) return gf::api_fail_msg(h, GF_EINVAL, "candidate spec is NULL");
  if ((s = gf::api_check_spec(h, &lr->geom, spec))) return s;
  const int per = spec->kind == GF_KIND_SINGLE ? 1 : gf::kLrP;
  if (spec->k < 1 || spec->k * per > gf::kLrPMax)
    return gf::api_fail_msg(h, GF_EINVAL, "the deferred form applies at most 32 pixels per step (k <= 32 single pixels, k <= 8 brushes)");
  if (!state || !idx || !status || !fom_out) return gf::api_fail_msg(h, GF_EINVAL, "state, idx, status and fom_out must be non-NULL");
  cudaStream_t st = (cudaStream_t)stream;
  gf::LrArgs a = gf::lr_args(*lr, reinterpret_cast<char*>(ws));
  gf::k_lr_pixels<<<1, 32, 0, st>>>(a, spec->kind, spec->dir_mask, state, idx, spec->k, status);
  gf::k_lr_w<<<gf::grid_of(lr->max_cols, 256, 1216), 256, 0, st>>>(a);
  // timed like the dense G update when profiling is armed: the record's rank is K p (columns
  // read x columns written), so the recorded flops 8 (K p) n are the product's
  gf::KernelTimer* tm = gf::api_timer(h);
  const bool rec = tm->on && tm->used < tm->max;
  if (rec) {
    tm->p_host[tm->used] = 0;
    cudaEventRecord(tm->ev0[tm->used], st);
  }
  {
    // slices: enough CTAs for every SM to hold as many as it can at once
    static std::atomic<int> per_sm[64];
    int dev = 0;
    cudaGetDevice(&dev);
    int occ = dev >= 0 && dev < 64 ? per_sm[dev].load() : 0;
    if (occ == 0) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gf::k_lr_columns, gf::kLrThreads, 0) != cudaSuccess ||
          occ < 1)
        occ = 1;
      if (dev >= 0 && dev < 64) per_sm[dev].store(occ);
    }
    // column groups: 4 new columns each, for the step's largest p; slices x groups <= kLrSlices
    const int pmax = spec->k * per;
    const int G = (pmax + gf::kLrP - 1) / gf::kLrP;
    const int64_t rb = (a.n + gf::kLrThreads - 1) / gf::kLrThreads;
    int64_t S = (int64_t)gf::api_sm_count(h) * occ / (rb * G);
    const int64_t smax = gf::kLrSlices / G;
    S = S < 1 ? 1 : (S > smax ? smax : S);
    gf::k_lr_columns<<<dim3((unsigned)(rb < 4864 ? rb : 4864), (unsigned)S, (unsigned)G), gf::kLrThreads, 0, st>>>(
        a, rec ? tm->p_dev + tm->used : nullptr);
    gf::k_lr_columns_sum<<<gf::grid_of((int64_t)pmax * a.n, 256, 4864), 256, 0, st>>>(a, (int)S, G);
  }
  if (rec) {
    cudaEventRecord(tm->ev1[tm->used], st);
    tm->n2[tm->used] = (double)a.n;
    tm->bytes_per_entry[tm->used] = 0;
    tm->used++;
  }
  gf::k_lr_capacitance<<<1, 256, 0, st>>>(a, status);
  if (spec->k * per <= gf::kLrP)
    gf::k_lr_apply<gf::kLrP><<<gf::grid_of(a.n, 256, 4864), 256, 0, st>>>(a, state, fom_out, applied);
  else
    gf::k_lr_apply<gf::kLrPMax><<<gf::grid_of(a.n, 256, 4864), 256, 0, st>>>(a, state, fom_out, applied);
  return gf::api_cuda_check(h, "gf_lowrank_update launch");
}

gf_status gf_lowrank_count(gf_handle* h, const gf_lowrank* lr, void* ws, size_t ws_bytes, int32_t* nterms,
                           int32_t* ncols, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = lr_check(h, lr, ws, ws_bytes);
  if (s) return s;
  gf::LrArgs a = gf::lr_args(*lr, reinterpret_cast<char*>(ws));
  gf::LrCount c{0, 0};
  cudaMemcpyAsync(&c, a.count, sizeof c, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  if (nterms) *nterms = c.nterms;
  if (ncols) *ncols = c.ncols;
  return gf::api_cuda_check(h, "gf_lowrank_count");
}

gf_status gf_lowrank_materialize(gf_handle* h, const gf_lowrank* lr, void* G, int64_t ldg, void* ws, size_t ws_bytes,
                                 void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = lr_check(h, lr, ws, ws_bytes);
  if (s) return s;
  const int64_t n = (int64_t)lr->geom.nx * lr->geom.ny + 1;
  if (!G || ((uintptr_t)G & 15u) || ldg < n) return gf::api_fail_msg(h, GF_EINVAL, "G must be 16-byte aligned with ldg >= n");
  gf::LrArgs a = gf::lr_args(*lr, reinterpret_cast<char*>(ws));
  gf::k_lr_materialize<<<gf::grid_of(n * n, 256, 4864), 256, 0, (cudaStream_t)stream>>>(a, reinterpret_cast<double2*>(G), ldg);
  return gf::api_cuda_check(h, "gf_lowrank_materialize launch");
}

}  // extern "C"
