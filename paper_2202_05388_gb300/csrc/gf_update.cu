// Update of G and E after a selection (Sec. II-B, Eqs. 10-14 and Eq. 4; Sec. III's
// filter + broadcast of the selected rows followed by every partition's update).
//
//   k_capacitance : V and d_chi from the chosen ids, A = I - G_VV D per wavelength, LU with
//                   partial pivoting (FP64), y = A^{-1} E_V, joint dFOM and fallback.
//   k_panels      : snapshots C0 = G[:, V] (n x p) and S = D A^{-1} G[V, :] (p x n), i.e. the
//                   new rows of Eq. 14 scaled by D -- the data the paper broadcasts.
//   k_rank_update : G <- G + C0 S (Eq. 10), every entry read and written once.
//   k_finish      : E <- E + C0 (D y) (Eq. 4), state flip, FOM = sum |E_N|^2.
#include <math.h>

#include <mutex>

#include "gf_internal.cuh"

namespace gf {

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
constexpr double kC128SmallWork = 2.5e6;   // n^2 p_max below which the FP64 FMA update is faster

// sP: shared memory for kLuMaxBlocked x kLuNB entries (the panel, row-major [row][j])
__device__ bool lu_blocked(cplx* __restrict__ A, int p, int32_t* __restrict__ piv, double thresh, cplx* sP) {
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
            const double d = 1.0 / bv;
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
        for (int k = j + 1; k < nb; ++k) sP[r * kLuNB + k] = sP[r * kLuNB + k] - f * sP[j * kLuNB + k];
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
              if (i < j) x[j] = x[j] - sP[j * kLuNB + i] * x[i];
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
            acc = acc - sP[(nb + i) * kLuNB + j] * (sU ? sU[j * w + v] : A[(int64_t)(c0 + j) * p + c0 + nb + v]);
        A[o] = acc;
      }
    }
    __syncthreads();
  }
  return true;
}

// A = I - G_VV D (row-major p x p, Eq. 9) and y = E_V for one wavelength; returns the pivot
// threshold kSingularRel ||A||_inf (every thread).
__device__ double cap_build(const CapArgs& a, const UpdLam& U, int p, const int32_t* __restrict__ V,
                            const double* __restrict__ dchi, cplx* A, cplx* y) {
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
__device__ double cap_tail(const CapArgs& a, const UpdLam& U, int p, const int32_t* __restrict__ V,
                           const double* __restrict__ dchi, const cplx* A, const int32_t* __restrict__ piv, cplx* y,
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
      for (int r = c + 1 + tid; r < p; r += blockDim.x) y[r] = y[r] - A[r * p + c] * yc;
      __syncthreads();
    }
  }
  // upper solve for y (column-oriented: one synchronisation per column)
  for (int c = p - 1; c >= 0; --c) {
    if (tid == 0) y[c] = cdiv(y[c], A[c * p + c]);
    __syncthreads();
    const cplx yc = y[c];
    for (int r = tid; r < c; r += blockDim.x) y[r] = y[r] - A[r * p + c] * yc;
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

// One wavelength of the capacitance solve for the set V (p pixels, contrasts dchi): A = I - G_VV D
// (Eq. 9), its LU with partial pivoting, y = A^{-1} E_V and the dFOM of Eq. 4 at the monitor into
// *df (every thread); the factors, pivots and D y go to the wavelength's workspace slots.  With sA
// (shared memory for kCapSmemP^2 + kCapSmemP entries) a system of p <= kCapSmemP and its
// right-hand side are built, factorised and solved there and copied to the workspace once.
// Returns false (in every thread) when A is singular.
__device__ bool cap_lam(const CapArgs& a, const WsLayout& L, char* ws, int l, int p, const int32_t* __restrict__ V,
                        const double* __restrict__ dchi, cplx* sA, double* df_out) {
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
                                                 const uint8_t* __restrict__ state,
                                                 const int32_t* __restrict__ idx, int32_t* status,
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

__global__ void k_capacitance(CapArgs a, WsLayout L, char* ws, const uint8_t* __restrict__ state,
                              const int32_t* __restrict__ idx, int32_t* status, int pre) {
  extern __shared__ __align__(16) unsigned char cap_smem[];
  capacitance_body(a, L, ws, state, idx, status, L.pmax <= kCapSmemP ? reinterpret_cast<cplx*>(cap_smem) : nullptr,
                   pre != 0);
}

// The first attempt's per-wavelength solves of a multi-wavelength step in parallel, one CTA per
// wavelength (p <= kCapSmemP; each CTA forms the set V again in its shared memory from the same
// ids): each writes its factors, pivots and D y to its workspace slots and its dFOM and singular
// flag to the control block; k_capacitance (pre) reads them, decides and runs any fallback.
__global__ void k_capacitance_lam(CapArgs a, WsLayout L, char* ws, const uint8_t* __restrict__ state,
                                  const int32_t* __restrict__ idx, const int32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char cap_smem[];
  __shared__ int32_t sV[kCapSmemP];
  __shared__ double sD[kCapSmemP];
  __shared__ int s_nv;
  UpdCtl* ctl = reinterpret_cast<UpdCtl*>(ws + L.ctl);
  const int l = blockIdx.x;
  if (threadIdx.x == 0) {
    int nv = 0;
    if (*status == GF_OK)
      for (int c = 0; c < a.k; ++c) {
        const int32_t id = idx[c];
        if (id < 0) break;
        nv += cand_pixels(id, a.kind, a.dir_mask, a.u.nx, a.u.ny, a.u.chi, state, sV + nv, sD + nv, a.u.nz);
      }
    s_nv = nv;
  }
  __syncthreads();
  const int p = s_nv;
  double df = 0.0;
  const bool ok = p > 0 ? cap_lam(a, L, ws, l, p, sV, sD, reinterpret_cast<cplx*>(cap_smem), &df) : true;
  if (threadIdx.x == 0) {
    ctl->lam_df[l] = df;
    ctl->lam_bad[l] = ok ? 0 : 1;
  }
}

// ---- one large system (a single wavelength with p_max > kCapSmemP) factorised by many CTAs.
// One CTA per solve is bound by that SM's FP64 pipe (p = 128: 1.9 ms).  Here the blocked
// right-looking LU of lu_blocked runs as a sequence of launches, with the same operations in the
// same order (so the same factors): per 8-column panel, one CTA factors the panel, applies its row
// interchanges to the other columns and solves U12 = L11^{-1} A12; then a grid of 16 x 16 tiles
// applies A22 -= L21 U12.  No launch waits on another CTA: the stream orders them.
// k_cap_lu_prep forms V, A and y = E_V (and the pivot threshold); k_cap_lu_finish solves for y
// and writes the dFOM and the singular flag where k_capacitance's first attempt reads them.
constexpr int kLuTile = 16;

__global__ void k_cap_lu_prep(CapArgs a, WsLayout L, char* ws, const uint8_t* __restrict__ state,
                              const int32_t* __restrict__ idx, const int32_t* __restrict__ status) {
  __shared__ int s_nv;
  UpdCtl* ctl = reinterpret_cast<UpdCtl*>(ws + L.ctl);
  int32_t* V = reinterpret_cast<int32_t*>(ws + L.V);
  double* dchi = reinterpret_cast<double*>(ws + L.dchi);
  if (threadIdx.x == 0) {
    int nv = 0;
    if (*status == GF_OK)
      for (int c = 0; c < a.k; ++c) {
        const int32_t id = idx[c];
        if (id < 0) break;
        nv += cand_pixels(id, a.kind, a.dir_mask, a.u.nx, a.u.ny, a.u.chi, state, V + nv, dchi + nv, a.u.nz);
      }
    s_nv = nv;
  }
  __syncthreads();
  const int p = s_nv;
  double thresh = 0.0;
  if (p > 0)
    thresh = cap_build(a, a.u.lam[0], p, V, dchi, reinterpret_cast<cplx*>(ws + L.lu), reinterpret_cast<cplx*>(ws + L.yd));
  if (threadIdx.x == 0) {
    ctl->lu_p = p;
    ctl->lu_bad = 0;
    ctl->lu_thresh = thresh;
  }
}

__global__ void k_lu_panel(WsLayout L, char* ws, int q) {
  __shared__ cplx sP[kLuMaxBlocked * kLuNB];
  __shared__ int s_pv[kLuNB];
  __shared__ int s_pr;
  __shared__ cplx s_inv;
  UpdCtl* ctl = reinterpret_cast<UpdCtl*>(ws + L.ctl);
  const int p = ctl->lu_p;
  const int c0 = q * kLuNB;
  if (p <= 0 || c0 >= p || ctl->lu_bad) return;
  cplx* A = reinterpret_cast<cplx*>(ws + L.lu);
  int32_t* piv = reinterpret_cast<int32_t*>(ws + L.piv);
  const double thresh = ctl->lu_thresh;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const int nb = p - c0 < kLuNB ? p - c0 : kLuNB;
  const int m = p - c0;
  for (int t = tid; t < m * nb; t += nt) {
    const int r = t / nb, j = t - r * nb;
    sP[r * kLuNB + j] = A[(int64_t)(c0 + r) * p + c0 + j];
  }
  __syncthreads();
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
          ctl->lu_bad = 1;
          s_pr = -1;
        } else {
          const cplx pv = sP[br * kLuNB + j];
          const double d = 1.0 / bv;
          s_inv = mk(pv.re * d, -pv.im * d);
          s_pr = br;
        }
        s_pv[j] = c0 + br;
        piv[c0 + j] = c0 + br;
      }
    }
    __syncthreads();
    const int pr = s_pr;
    if (pr < 0) return;
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
      for (int k = j + 1; k < nb; ++k) sP[r * kLuNB + k] = sP[r * kLuNB + k] - f * sP[j * kLuNB + k];
    }
    __syncthreads();
  }
  for (int t = tid; t < m * nb; t += nt) {
    const int r = t / nb, j = t - r * nb;
    A[(int64_t)(c0 + r) * p + c0 + j] = sP[r * kLuNB + j];
  }
  // the panel's interchanges on the columns outside it, then U12 (one thread per column)
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
    if (v >= c0 + nb) {
      cplx x[kLuNB];
#pragma unroll
      for (int j = 0; j < kLuNB; ++j)
        if (j < nb) x[j] = A[(int64_t)(c0 + j) * p + v];
#pragma unroll
      for (int j = 1; j < kLuNB; ++j)
        if (j < nb)
#pragma unroll
          for (int i = 0; i < kLuNB; ++i)
            if (i < j) x[j] = x[j] - sP[j * kLuNB + i] * x[i];
#pragma unroll
      for (int j = 1; j < kLuNB; ++j)
        if (j < nb) A[(int64_t)(c0 + j) * p + v] = x[j];
    }
  }
}

// A22 -= L21 U12 on one 16 x 16 tile of the trailing matrix of panel q (blockIdx: column tile, row
// tile), each element with the panel's terms in order.
__global__ void k_lu_trail(WsLayout L, char* ws, int q) {
  __shared__ cplx sL[kLuTile][kLuNB];
  __shared__ cplx sU[kLuNB][kLuTile];
  const UpdCtl* ctl = reinterpret_cast<const UpdCtl*>(ws + L.ctl);
  const int p = ctl->lu_p;
  const int c0 = q * kLuNB;
  if (p <= 0 || c0 >= p || ctl->lu_bad) return;
  const int nb = p - c0 < kLuNB ? p - c0 : kLuNB;
  const int w = p - c0 - nb;
  const int v0 = blockIdx.x * kLuTile, i0 = blockIdx.y * kLuTile;
  if (v0 >= w || i0 >= w) return;
  cplx* A = reinterpret_cast<cplx*>(ws + L.lu);
  const int tid = threadIdx.x;
  for (int t = tid; t < kLuTile * kLuNB; t += blockDim.x) {
    const int r = t / kLuNB, j = t % kLuNB;
    sL[r][j] = (i0 + r < w && j < nb) ? A[(int64_t)(c0 + nb + i0 + r) * p + c0 + j] : mk(0.0, 0.0);
    const int jj = t / kLuTile, c = t % kLuTile;
    sU[jj][c] = (v0 + c < w && jj < nb) ? A[(int64_t)(c0 + jj) * p + c0 + nb + v0 + c] : mk(0.0, 0.0);
  }
  __syncthreads();
  for (int t = tid; t < kLuTile * kLuTile; t += blockDim.x) {
    const int r = t / kLuTile, c = t % kLuTile;
    if (i0 + r >= w || v0 + c >= w) continue;
    const int64_t o = (int64_t)(c0 + nb + i0 + r) * p + c0 + nb + v0 + c;
    cplx acc = A[o];
#pragma unroll
    for (int j = 0; j < kLuNB; ++j)
      if (j < nb) acc = acc - sL[r][j] * sU[j][c];
    A[o] = acc;
  }
}

__global__ void k_cap_lu_finish(CapArgs a, WsLayout L, char* ws) {
  UpdCtl* ctl = reinterpret_cast<UpdCtl*>(ws + L.ctl);
  const int p = ctl->lu_p;
  double df = 0.0;
  bool ok = !ctl->lu_bad;
  if (p > 0 && ok)
    df = cap_tail(a, a.u.lam[0], p, reinterpret_cast<const int32_t*>(ws + L.V),
                  reinterpret_cast<const double*>(ws + L.dchi), reinterpret_cast<const cplx*>(ws + L.lu),
                  reinterpret_cast<const int32_t*>(ws + L.piv), reinterpret_cast<cplx*>(ws + L.yd), false);
  if (threadIdx.x == 0) {
    ctl->lam_df[0] = df;
    ctl->lam_bad[0] = ok ? 0 : 1;
  }
}

// ----------------------------------------------------------------------------- panels
// Column j: R[:, j] = A^{-1} G[V, j] (Eq. 14) and S[:, j] = D R[:, j]; row j of the rows held:
// C0[j, :] = G[j, V].
__device__ __forceinline__ void panels_body(const UpdArgs& a, const WsLayout& L, char* ws, int want_S) {
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
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < jend;
         j += (int64_t)gridDim.x * blockDim.x) {
      if (j < U.rows)
        for (int u = 0; u < p; ++u) C0[j * L.pmax + u] = ldG(U.G, a.dtype, U.ldg, j, V[u]);
      if (!want_S || j >= n) continue;
      if (p <= kMaxPixelsPerCand) {
        cplx x[kMaxPixelsPerCand];
#pragma unroll
        for (int u = 0; u < kMaxPixelsPerCand; ++u)
          if (u < p) x[u] = U.vrows ? ldG(U.vrows, a.dtype, U.ldv, u, j) : ldG(U.G, a.dtype, U.ldg, V[u], j);
        // P A = L U with full-row interchanges: apply all interchanges in order first,
        // then the unit-lower solve, then the upper solve
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
              if (rr < p) x[rr] = x[rr] - A[rr * p + c] * x[c];
          }
        }
#pragma unroll
        for (int c = kMaxPixelsPerCand - 1; c >= 0; --c) {
          if (c < p) {
            cplx acc = x[c];
#pragma unroll
            for (int v = c + 1; v < kMaxPixelsPerCand; ++v)
              if (v < p) acc = acc - A[c * p + v] * x[v];
            x[c] = cdiv(acc, A[c * p + c]);
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

__global__ void k_panels(UpdArgs a, WsLayout L, char* ws, int want_S) { panels_body(a, L, ws, want_S); }

// ----------------------------------------------------------------------------- rank-p (FP64)
constexpr int kUpdThreads = 256;
constexpr int kUpdRows = 16;

// G[i, j] += sum_u C0[i, u] S[u, j] for one wavelength, complex128 storage, native DFMA.
// P > 0: compile-time rank; P == 0: runtime rank p.
template <int P>
__device__ __forceinline__ void rank_update_f64_body(double2* __restrict__ G, int64_t ldg, int64_t n, int64_t rows,
                                                     int pmax, int p, const cplx* __restrict__ C0,
                                                     const cplx* __restrict__ S, int64_t j) {
  cplx s[P > 0 ? P : 1];
  if (P > 0) {
#pragma unroll
    for (int u = 0; u < P; ++u) s[u] = S[(int64_t)u * n + j];
  }
  for (int64_t i0 = (int64_t)blockIdx.y * kUpdRows; i0 < rows; i0 += (int64_t)gridDim.y * kUpdRows) {
    const int64_t iend = i0 + kUpdRows < rows ? i0 + kUpdRows : rows;
    for (int64_t i = i0; i < iend; ++i) {
      double2 g = G[i * ldg + j];
      cplx acc = mk(g.x, g.y);
      if (P > 0) {
#pragma unroll
        for (int u = 0; u < P; ++u) acc = cfma(C0[i * pmax + u], s[u], acc);
      } else {
        for (int u = 0; u < p; ++u) acc = cfma(C0[i * pmax + u], S[(int64_t)u * n + j], acc);
      }
      G[i * ldg + j] = make_double2(acc.re, acc.im);
    }
  }
}

__global__ void __launch_bounds__(kUpdThreads) k_rank_update_f64(double2* __restrict__ G, int64_t ldg,
                                                                 int64_t n, int64_t rows, int pmax,
                                                                 const cplx* __restrict__ C0,
                                                                 const cplx* __restrict__ S,
                                                                 const UpdCtl* __restrict__ ctl,
                                                                 int only_above,
                                                                 int32_t* __restrict__ prof_p) {
  const int p = ctl->skip ? 0 : ctl->nv;
  if (p <= only_above) return;
  if (prof_p && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *prof_p = p;
  const int64_t j = blockIdx.x * (int64_t)kUpdThreads + threadIdx.x;
  if (j >= n) return;
  switch (p) {
    case 1: rank_update_f64_body<1>(G, ldg, n, rows, pmax, p, C0, S, j); break;
    case 2: rank_update_f64_body<2>(G, ldg, n, rows, pmax, p, C0, S, j); break;
    case 3: rank_update_f64_body<3>(G, ldg, n, rows, pmax, p, C0, S, j); break;
    case 4: rank_update_f64_body<4>(G, ldg, n, rows, pmax, p, C0, S, j); break;
    default: rank_update_f64_body<0>(G, ldg, n, rows, pmax, p, C0, S, j); break;
  }
}

// complex64 storage: same update, FP64 arithmetic on the FP64 panels, rounded once on store.
__global__ void __launch_bounds__(kUpdThreads) k_rank_update_c64_ref(float2* __restrict__ G, int64_t ldg,
                                                                     int64_t n, int64_t rows, int pmax,
                                                                     const cplx* __restrict__ C0,
                                                                     const cplx* __restrict__ S,
                                                                     const UpdCtl* __restrict__ ctl,
                                                                     int32_t* __restrict__ prof_p) {
  const int p = ctl->skip ? 0 : ctl->nv;
  if (prof_p && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *prof_p = p;
  if (p == 0) return;
  const int64_t j = blockIdx.x * (int64_t)kUpdThreads + threadIdx.x;
  if (j >= n) return;
  for (int64_t i0 = (int64_t)blockIdx.y * kUpdRows; i0 < rows; i0 += (int64_t)gridDim.y * kUpdRows) {
    const int64_t iend = i0 + kUpdRows < rows ? i0 + kUpdRows : rows;
    for (int64_t i = i0; i < iend; ++i) {
      float2 g = G[i * ldg + j];
      cplx acc = mk(0.0, 0.0);
      for (int u = 0; u < p; ++u) acc = cfma(C0[i * pmax + u], S[(int64_t)u * n + j], acc);
      G[i * ldg + j] = make_float2((float)((double)g.x + acc.re), (float)((double)g.y + acc.im));
    }
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

__device__ __forceinline__ void c64_fp32_tile(float2* __restrict__ G, int64_t ldg, int64_t n, int64_t m, int pmax, int p,
                                              const cplx* __restrict__ C0, const cplx* __restrict__ S,
                                              int64_t rt, int64_t ct, float2 (*sC)[kC64Fp32MaxP]) {
  const int64_t i0 = rt * kF32Rows;
  const int64_t j = ct * kF32Cols + 2 * threadIdx.x;
  __syncthreads();                                   // previous tile done with sC
  for (int t = threadIdx.x; t < kF32Rows * kC64Fp32MaxP; t += kF32Threads) {
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
  const int rows = (int)(m - i0 < kF32Rows ? m - i0 : kF32Rows);
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

__global__ void __launch_bounds__(kF32Threads, 3) k_rank_update_c64_fp32(float2* __restrict__ G, int64_t ldg, int64_t n,
                                                                      int64_t m, int pmax, const cplx* __restrict__ C0,
                                                                      const cplx* __restrict__ S,
                                                                      const UpdCtl* __restrict__ ctl,
                                                                      int32_t* __restrict__ prof_p) {
  __shared__ float2 sC[kF32Rows][kC64Fp32MaxP];
  const int p = ctl->skip ? 0 : ctl->nv;
  if (prof_p && blockIdx.x == 0 && threadIdx.x == 0) *prof_p = p;
  if (p < 1 || p > kC64Fp32MaxP) return;
  const int64_t nrt = (m + kF32Rows - 1) / kF32Rows, nct = (n + kF32Cols - 1) / kF32Cols;
  for (int64_t t = blockIdx.x; t < nrt * nct; t += gridDim.x)
    c64_fp32_tile(G, ldg, n, m, pmax, p, C0, S, t / nct, t % nct, sC);
}

// Batched: the tiles of every problem that applies an update, interleaved over the CTAs.
__global__ void __launch_bounds__(kF32Threads, 3) k_rank_update_c64_fp32_batch(const BatchItem* __restrict__ items,
                                                                            int nprob) {
  __shared__ float2 sC[kF32Rows][kC64Fp32MaxP];
  __shared__ int64_t s_begin[kBatchMax + 1];
  __shared__ int s_p[kBatchMax];
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int b = 0; b < nprob; ++b) {
      s_begin[b] = acc;
      const UpdCtl* c = reinterpret_cast<const UpdCtl*>(items[b].ws + items[b].L.ctl);
      const int p = c->skip ? 0 : c->nv;
      s_p[b] = p;
      const int64_t n = items[b].L.n;
      if (p >= 1 && p <= kC64Fp32MaxP) acc += ((n + kF32Rows - 1) / kF32Rows) * ((n + kF32Cols - 1) / kF32Cols);
    }
    s_begin[nprob] = acc;
  }
  __syncthreads();
  const int64_t T = s_begin[nprob];
  int b = 0;
  for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
    while (t >= s_begin[b + 1]) ++b;
    const BatchItem& it = items[b];
    const int64_t n = it.L.n;
    const int64_t nct = (n + kF32Cols - 1) / kF32Cols;
    const int64_t u = t - s_begin[b];
    c64_fp32_tile(reinterpret_cast<float2*>(it.G), it.ldg, n, n, it.L.pmax, s_p[b],
                  reinterpret_cast<const cplx*>(it.ws + it.L.C0), reinterpret_cast<const cplx*>(it.ws + it.L.S),
                  u / nct, u % nct, sC);
  }
}

void launch_rank_update_c64_fp32(float2* G, int64_t ldg, int64_t n, int64_t rows, int pmax, const cplx* C0, const cplx* S,
                                 const UpdCtl* ctl, int32_t* prof_p, int ctas, cudaStream_t st) {
  k_rank_update_c64_fp32<<<ctas, kF32Threads, 0, st>>>(G, ldg, n, rows, pmax, C0, S, ctl, prof_p);
}

void launch_rank_update_c64_fp32_batch(const BatchItem* items, int nprob, int ctas, cudaStream_t st) {
  k_rank_update_c64_fp32_batch<<<ctas, kF32Threads, 0, st>>>(items, nprob);
}

// ----------------------------------------------------------------------------- field, state, FOM
__device__ __forceinline__ void finish_body(const UpdArgs& a, const WsLayout& L, char* ws, uint8_t* __restrict__ state,
                                            double* __restrict__ fom_out, int32_t* __restrict__ applied) {
  const UpdCtl* ctl = reinterpret_cast<const UpdCtl*>(ws + L.ctl);
  const int64_t n = L.n;
  const int64_t N = n - 1;
  const bool skip = ctl->skip != 0;
  const int p = skip ? 0 : ctl->nv;
  const int32_t* V = reinterpret_cast<const int32_t*>(ws + L.V);
  (void)N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
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
  if (blockIdx.x == 0) {   // one flip per point (the unknowns of a point are consecutive in V)
    for (int t = threadIdx.x; t < p; t += blockDim.x)
      if (V[t] % a.ncomp == 0) state[V[t] / a.ncomp] ^= 1;
  }
}

__global__ void k_finish(UpdArgs a, WsLayout L, char* ws, uint8_t* __restrict__ state,
                         double* __restrict__ fom_out, int32_t* __restrict__ applied) {
  finish_body(a, L, ws, state, fom_out, applied);
}

// ----------------------------------------------------------------------------- batched steps
// blockIdx.y (x for the single-CTA capacitance) selects the problem; the argument blocks are
// rebuilt in shared memory from the device table and the single-problem bodies run unchanged.
__device__ __forceinline__ void batch_shared_args(const BatchItem* items, int b, int dtype, UpdArgs& sa,
                                                  WsLayout& sL) {
  if (threadIdx.x == 0) {
    batch_upd_args(items[b], dtype, sa);
    sL = items[b].L;
  }
  __syncthreads();
}

__global__ void k_capacitance_batch(const BatchItem* __restrict__ items, int dtype, int kind, int dir_mask) {
  __shared__ CapArgs sa;
  __shared__ WsLayout sL;
  if (threadIdx.x == 0) {
    batch_upd_args(items[blockIdx.x], dtype, sa.u);
    sa.kind = kind;
    sa.dir_mask = dir_mask;
    sa.k = 1;
    sa.pmax = items[blockIdx.x].L.pmax;
    sL = items[blockIdx.x].L;
  }
  __syncthreads();
  const BatchItem& it = items[blockIdx.x];
  capacitance_body(sa, sL, it.ws, it.state, it.idx, it.status);
}

__global__ void k_panels_batch(const BatchItem* __restrict__ items, int dtype) {
  __shared__ UpdArgs sa;
  __shared__ WsLayout sL;
  batch_shared_args(items, blockIdx.y, dtype, sa, sL);
  panels_body(sa, sL, items[blockIdx.y].ws, 1);
}

__global__ void k_finish_batch(const BatchItem* __restrict__ items, int dtype) {
  __shared__ UpdArgs sa;
  __shared__ WsLayout sL;
  batch_shared_args(items, blockIdx.y, dtype, sa, sL);
  const BatchItem& it = items[blockIdx.y];
  finish_body(sa, sL, it.ws, it.state, it.fom, it.applied);
}

static dim3 batch_grid(int64_t widest, int nprob) {
  int64_t b = (widest + 255) / 256;
  if (b > 1216) b = 1216;
  return dim3((unsigned)(b < 1 ? 1 : b), (unsigned)nprob);
}

void launch_capacitance_batch(const BatchItem* items, int nprob, int dtype, const gf_cand_spec& spec,
                              cudaStream_t st) {
  k_capacitance_batch<<<nprob, 256, 0, st>>>(items, dtype, spec.kind, spec.dir_mask);
}

void launch_panels_batch(const BatchItem* items, int nprob, int dtype, int64_t widest, cudaStream_t st) {
  k_panels_batch<<<batch_grid(widest, nprob), 256, 0, st>>>(items, dtype);
}

void launch_finish_batch(const BatchItem* items, int nprob, int dtype, int64_t widest, cudaStream_t st) {
  k_finish_batch<<<batch_grid(widest, nprob), 256, 0, st>>>(items, dtype);
}

void launch_update(const UpdArgs& a, const WsLayout& L, char* ws, uint8_t* state,
                   const gf_cand_spec& spec, const int32_t* idx, int32_t* status, double* fom_out,
                   int32_t* applied, cudaStream_t st, KernelTimer* timer) {
  CapArgs ca;
  ca.u = a;
  ca.kind = spec.kind;
  ca.dir_mask = spec.dir_mask;
  ca.k = spec.k < 1 ? 1 : spec.k;
  ca.pmax = L.pmax;
  const size_t cap_smem = L.pmax <= kCapSmemP ? sizeof(cplx) * ((size_t)kCapSmemP * kCapSmemP + kCapSmemP) : 0;
  {
    // once per device: the opt-in above the default (48 KB less the static shared memory)
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || !done[dev]) {
      cudaFuncSetAttribute(k_capacitance, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(cplx) * (kCapSmemP * kCapSmemP + kCapSmemP)));
      cudaFuncSetAttribute(k_capacitance_lam, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(cplx) * (kCapSmemP * kCapSmemP + kCapSmemP)));
      if (dev >= 0 && dev < 64) done[dev] = true;
    }
  }
  // several wavelengths: their joint solves run side by side, one CTA each; one wavelength with
  // a large set: the first attempt's solve factorised by many CTAs
  const bool multi = a.nlam == 1 && L.pmax > kCapSmemP && L.pmax <= kLuMaxBlocked;
  const int pre = (a.nlam > 1 && L.pmax <= kCapSmemP) || multi ? 1 : 0;
  if (multi) {
    k_cap_lu_prep<<<1, 256, 0, st>>>(ca, L, ws, state, idx, status);
    for (int q = 0; q * kLuNB < L.pmax; ++q) {
      k_lu_panel<<<1, 256, 0, st>>>(L, ws, q);
      const int w = L.pmax - q * kLuNB - kLuNB;        // trailing width at p = p_max (smaller p: tiles exit)
      if (w > 0) {
        const unsigned t = (unsigned)((w + kLuTile - 1) / kLuTile);
        k_lu_trail<<<dim3(t, t), 256, 0, st>>>(L, ws, q);
      }
    }
    k_cap_lu_finish<<<1, 256, 0, st>>>(ca, L, ws);
  } else if (pre) {
    k_capacitance_lam<<<a.nlam, 256, cap_smem, st>>>(ca, L, ws, state, idx, status);
  }
  k_capacitance<<<1, 256, cap_smem, st>>>(ca, L, ws, state, idx, status, pre);
  const int64_t n = L.n;
  const int64_t rows = a.lam[0].rows;       // rows of G held (n, or a shard's row block)
  // complex64 on the tensor cores: S is formed from an explicit D A^{-1} by an FP32 GEMM, so
  // the panels kernel only gathers C0
  struct Map128 { alignas(64) unsigned char b[128]; };
  Map128 maps[kMaxLam];
  // rank <= 4 complex64: an FP32 stream on the CUDA cores (HBM-bound); larger ranks: tensor cores
  const bool fast = a.algo != GF_UPDATE_DFMA;
  const bool c64f32 = a.dtype == GF_C64 && fast && L.pmax <= kC64Fp32MaxP;
  bool c64tc = a.dtype == GF_C64 && fast && !c64f32 && L.pmax <= kC64MaxP;
  // complex128, p <= 4: the tensor-core digit products, except where the whole update is small
  // enough (n^2 p_max <= kC128SmallWork, G resident in L2) that the FP64 FMA kernel finishes
  // before the persistent tensor-core pipeline has filled (32x32 single pixel: 19 vs 44 us)
  const bool oz = a.dtype == GF_C128 &&
                  (a.algo == GF_UPDATE_TENSOR || (a.algo == GF_UPDATE_TC && (double)rows * (double)n * L.pmax > kC128SmallWork));
  for (int l = 0; c64tc && l < a.nlam; ++l)
    c64tc = c64_tc_make_map(reinterpret_cast<float2*>(a.lam[l].G), a.lam[l].ldg, n, rows, maps[l].b);
  {
    const int64_t w = rows > n ? rows : n;
    int64_t b = (w + 255) / 256;
    k_panels<<<(int)(b < 4864 ? b : 4864), 256, 0, st>>>(a, L, ws, c64tc ? 0 : 1);
  }
  const UpdCtl* ctl = reinterpret_cast<const UpdCtl*>(ws + L.ctl);
  dim3 grid((unsigned)((n + kUpdThreads - 1) / kUpdThreads),
            (unsigned)(((rows + kUpdRows - 1) / kUpdRows) < 65535 ? (rows + kUpdRows - 1) / kUpdRows : 65535));
  for (int l = 0; l < a.nlam; ++l) {
    const cplx* C0 = reinterpret_cast<const cplx*>(ws + L.C0 + l * L.panel_s);
    const cplx* S = reinterpret_cast<const cplx*>(ws + L.S + l * L.panel_s);
    const bool rec = timer && timer->on && timer->used < timer->max;
    int32_t* prof_p = rec ? timer->p_dev + timer->used : nullptr;
    if (rec) {
      timer->p_host[timer->used] = 0;
      cudaEventRecord(timer->ev0[timer->used], st);
    }
    if (a.dtype == GF_C128) {
      double2* G = reinterpret_cast<double2*>(a.lam[l].G);
      int only_above = 0;
      if (oz) {
        // p <= 4 on the tensor cores; the DFMA kernel below takes p > 4
        // without a tensor map (driver too old) the DFMA kernel below takes every p
        if (launch_rank_update_ozaki(G, a.lam[l].ldg, n, rows, L.pmax, C0, S, ctl,
                                     reinterpret_cast<uint8_t*>(ws + L.ozA), reinterpret_cast<int32_t*>(ws + L.ozE),
                                     reinterpret_cast<uint8_t*>(ws + L.ozB), reinterpret_cast<int32_t*>(ws + L.ozF),
                                     status, prof_p, a.sm_count, st))
          only_above = 4;
      }
      if (!oz || L.pmax > 4 || only_above == 0)
        k_rank_update_f64<<<grid, kUpdThreads, 0, st>>>(G, a.lam[l].ldg, n, rows, L.pmax, C0, S, ctl, only_above,
                                                        prof_p);
    } else if (c64f32) {
      launch_rank_update_c64_fp32(reinterpret_cast<float2*>(a.lam[l].G), a.lam[l].ldg, n, rows, L.pmax, C0, S, ctl,
                                  prof_p, a.sm_count * 3, st);
    } else if (c64tc) {
      launch_rank_update_c64_tc(maps[l].b, reinterpret_cast<float2*>(a.lam[l].G), a.lam[l].ldg, n, rows,
                                a.lam[l].vrows, a.lam[l].ldv, L, ws, l, status, prof_p, a.sm_count, st);
    } else {
      k_rank_update_c64_ref<<<grid, kUpdThreads, 0, st>>>(reinterpret_cast<float2*>(a.lam[l].G),
                                                          a.lam[l].ldg, n, rows, L.pmax, C0, S, ctl, prof_p);
    }
    if (rec) {
      cudaEventRecord(timer->ev1[timer->used], st);
      timer->n2[timer->used] = (double)rows * (double)n;
      timer->bytes_per_entry[timer->used] = a.dtype == GF_C128 ? 32 : 16;
      timer->used++;
    }
  }
  {
    int64_t b = (n + 255) / 256;
    k_finish<<<(int)(b < 4864 ? b : 4864), 256, 0, st>>>(a, L, ws, state, fom_out, applied);
  }
}

}  // namespace gf
