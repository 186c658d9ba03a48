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

#include <cooperative_groups.h>

#include "gf_internal.cuh"
#include "gf_stage_bodies.cuh"

namespace gf {

// ----------------------------------------------------------------------------- capacitance
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

// ---- one large system (a single wavelength with p_max > kCapSmemP), held in the shared memory of
// one cluster of CTAs (distributed shared memory).  One CTA per solve is bound by that SM's FP64
// pipe (p = 128: 1.9 ms).  A = I - G_VV D is built, factorised with partial pivoting and solved
// without leaving the cluster: physical row r (with y as its last entry) lives in CTA r % CN.  Row interchanges
// are kept as a permutation shared by every CTA (logical position i holds physical row phys[i]),
// so a pivot row is only read by the others, never moved, and one cluster barrier per column
// suffices: after it every CTA reads the candidates of the column (double-buffered slots), takes
// the same pivot (largest modulus, lowest position on ties), copies the pivot row from its owner
// and eliminates its own rows.  Every element sees the same operations in the same order as the
// blocked factorisation of lu_blocked (the multiplier a_rj (conj(pv) / |pv|^2), then
// cfms(l, u_jk, a_rk) column after column, y included), and the upper solve runs in blocks of
// kLuNB rows from the bottom as cap_tail does, so the factors, pivots, y and the dFOM are the bits
// one CTA computes.  A pivot's value travels with its candidate, so a column costs one cluster
// barrier and two rounds of distributed-shared-memory loads (candidates, pivot row).
// Outputs: V, dchi, the factors (row-major, logical order), pivots and D y in the workspace, the
// dFOM and singular flag in the control block, where k_capacitance's first attempt reads them.
// CN = 16 CTAs where the device can hold such a cluster (a non-portable size), else 8.
// Candidates are compared as integers: |a|^2 >= 0, and the bit patterns of non-negative doubles
// order as the values do, so the key is the bit pattern (-1 for NaN, which never wins).  The
// comparisons stay off GB300's narrow FP64 pipe, where every one on the per-column critical path
// cost a warp instruction's worth of FP64 issue.
struct CluSlot {                 // a CTA's best candidate of a column: key, position, conj(a) / |a|^2
  cplx inv;
  long long key;
  int pos;
};
__device__ __forceinline__ long long clu_key(double v) {
  const long long b = __double_as_longlong(v);
  return (b & 0x7FFFFFFFFFFFFFFFll) > 0x7FF0000000000000ll ? -1ll : b;
}
__device__ __forceinline__ bool clu_better(long long k, int ps, long long bk, int bps) {
  return k > bk || (k == bk && ps < bps);
}
// conj(a) / |a|^2 with the pivot reciprocal of the one-CTA factorisation (0 for no candidate);
// each warp forms it for its own best candidate, so the reciprocals of a column run side by side
__device__ __forceinline__ cplx clu_inv(long long key, cplx a) {
  if (key <= 0) return mk(0.0, 0.0);
  const double d = rcp_nr(__longlong_as_double(key));
  return mk(a.re * d, -a.im * d);
}
// the CTA's best of its warps' candidates (with their reciprocals) into its slot
__device__ __forceinline__ void clu_publish(const long long* wk, const int* wr, const cplx* wi, int nw, CluSlot& slot) {
  int b = 0;
  for (int w = 1; w < nw; ++w)
    if (clu_better(wk[w], wr[w], wk[b], wr[b])) b = w;
  slot.key = wk[b];
  slot.pos = wr[b];
  slot.inv = wi[b];
}
__host__ __device__ constexpr size_t cap_cluster_smem(int pmax, int cn) {
  // rows (R x (pmax + 1)) | pivot row (pmax + 1) | block of the upper solve (kLuNB x kLuNB + kLuNB)
  // | final y (pmax) | dchi (pmax) | phys, pos, V (pmax each)
  return sizeof(cplx) * ((size_t)((pmax + cn - 1) / cn) * (pmax + 1) + (pmax + 1) + kLuNB * kLuNB + kLuNB + pmax) +
         sizeof(double) * (size_t)pmax + sizeof(int32_t) * 3 * (size_t)pmax;
}

template <int CN>
__global__ void __launch_bounds__(256)
    k_cap_cluster(CapArgs a, WsLayout L, char* ws, const uint8_t* state, const int32_t* idx, const int32_t* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char clu_smem[];
  const int pm = L.pmax;
  const int Rm = (pm + CN - 1) / CN;
  const int W = pm + 1;                                   // row stride: p columns of A, then y
  cplx* rows = reinterpret_cast<cplx*>(clu_smem);
  cplx* prow = rows + (size_t)Rm * W;
  cplx* sU = prow + W;                                    // kLuNB x kLuNB block of U, then its y
  cplx* yfin = sU + kLuNB * kLuNB + kLuNB;
  double* sD = reinterpret_cast<double*>(yfin + pm);
  int32_t* phys = reinterpret_cast<int32_t*>(sD + pm);
  int32_t* pos = phys + pm;
  int32_t* sV = pos + pm;
  __shared__ CluSlot s_slot[2];                           // double-buffered: columns j, j + 1
  __shared__ long long s_wk[8];
  __shared__ int s_wr[8];
  __shared__ cplx s_wa[8];
  __shared__ cplx s_l[kLuMaxBlocked / 8];                 // the column's multipliers, by local row
  __shared__ double s_dv[kLuMaxBlocked / 8];              // 1 / |u_cc|^2 of the CTA's rows (upper solve)
  __shared__ double s_db[kLuNB];                          // CTA 0: those of the current block
  __shared__ double s_thr, s_rmax;
  __shared__ int s_nv, s_pr, s_bad;
  __shared__ cplx s_inv;
  __shared__ double s_red[32], s_bv[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = (int)(blockDim.x >> 5);
  const int rank = (int)cl.block_rank();
  const UpdLam& U = a.u.lam[0];
  UpdCtl* ctl = reinterpret_cast<UpdCtl*>(ws + L.ctl);

  if (tid == 0) {
    int nv = 0;
    if (*status == GF_OK)
      for (int c = 0; c < a.k; ++c) {
        const int32_t id = idx[c];
        if (id < 0) break;
        nv += cand_pixels(id, a.kind, a.dir_mask, a.u.nx, a.u.ny, a.u.chi, state, sV + nv, sD + nv, a.u.nz);
      }
    s_nv = nv;
    s_bad = 0;
  }
  __syncthreads();
  const int p = s_nv;                                     // the same in every CTA
  if (rank == 0) {
    int32_t* V = reinterpret_cast<int32_t*>(ws + L.V);
    double* dchi = reinterpret_cast<double*>(ws + L.dchi);
    for (int t = tid; t < p; t += blockDim.x) {
      V[t] = sV[t];
      dchi[t] = sD[t];
    }
  }
  const int R = p > rank ? (p - rank + CN - 1) / CN : 0;  // physical rows rank + CN lr
  // A = I - G_VV D and y = E_V for the CTA's rows; the row sums |A|_1 a warp per row
  for (int t = tid; t < R * p; t += blockDim.x) {
    const int lr = t / p, c = t - lr * p, r = rank + CN * lr;
    const cplx g = U.vrows ? ldG(U.vrows, a.u.dtype, U.ldv, r, sV[c]) : ldG(U.G, a.u.dtype, U.ldg, sV[r], sV[c]);
    rows[(size_t)lr * W + c] = mk(r == c ? 1.0 : 0.0, 0.0) - sD[c] * g;
  }
  for (int lr = tid; lr < R; lr += blockDim.x) rows[(size_t)lr * W + p] = U.E[sV[rank + CN * lr]];
  for (int i = tid; i < p; i += blockDim.x) {
    phys[i] = i;
    pos[i] = i;
  }
  __syncthreads();
  double rmax = 0.0;
  for (int lr = wid; lr < R; lr += nw) {
    double sum = 0.0;
    for (int c = lane; c < p; c += 32) sum += cabs1(rows[(size_t)lr * W + c]);
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    rmax = fmax(rmax, sum);                               // lane 0 holds the row's sum
  }
  // the candidates of column 0 (every row), a lane per row
  long long bk = -1;
  int bp = 0x7fffffff;
  cplx ba = mk(0.0, 0.0);
  for (int lr = tid; lr < R; lr += blockDim.x) {
    const cplx a0 = rows[(size_t)lr * W];
    const long long k = clu_key(abs2(a0));
    const int ps = rank + CN * lr;
    if (clu_better(k, ps, bk, bp)) { bk = k; bp = ps; ba = a0; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const long long ok = __shfl_down_sync(0xffffffffu, bk, o);
    const int op = __shfl_down_sync(0xffffffffu, bp, o);
    const double ore = __shfl_down_sync(0xffffffffu, ba.re, o), oim = __shfl_down_sync(0xffffffffu, ba.im, o);
    if (clu_better(ok, op, bk, bp)) { bk = ok; bp = op; ba = mk(ore, oim); }
  }
  if (lane == 0) { s_wk[wid] = bk; s_wr[wid] = bp; s_wa[wid] = clu_inv(bk, ba); s_red[wid] = rmax; }
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < nw; ++w) m = fmax(m, s_red[w]);
    s_rmax = m;
    clu_publish(s_wk, s_wr, s_wa, nw, s_slot[0]);
  }
  cl.sync();
  if (wid == 0) {                                         // the pivot threshold kSingularRel ||A||_inf
    double m = lane < CN ? *cl.map_shared_rank(&s_rmax, lane) : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if (lane == 0) s_thr = kSingularRel * m;
  }
  __syncthreads();
  const long long thr2_key = clu_key(s_thr * s_thr);

  // ---- factorisation, one cluster barrier per column
  for (int j = 0; j < p; ++j) {
    const int buf = j & 1;
    if (j > 0) cl.sync();                                 // column j's candidates are published
    if (wid == 0) {                                       // lane q reads CTA q's candidate
      long long k = -1;
      int ps = 0x7fffffff;
      cplx iv = mk(0.0, 0.0);
      if (lane < CN) {
        const CluSlot* sl = cl.map_shared_rank(&s_slot[buf], lane);
        k = sl->key;
        ps = sl->pos;
        iv = sl->inv;
      }
      for (int o = 16; o > 0; o >>= 1) {
        const long long ok = __shfl_down_sync(0xffffffffu, k, o);
        const int op = __shfl_down_sync(0xffffffffu, ps, o);
        const double ore = __shfl_down_sync(0xffffffffu, iv.re, o), oim = __shfl_down_sync(0xffffffffu, iv.im, o);
        if (clu_better(ok, op, k, ps)) { k = ok; ps = op; iv = mk(ore, oim); }
      }
      if (lane == 0) {
        // |pv|^2 >= thresh^2 and > 0 (a NaN key is -1 and fails both)
        if (k < thr2_key || k <= 0) {
          s_bad = 1;
        } else {
          s_pr = ps;
          s_inv = iv;
          if (rank == 0) reinterpret_cast<int32_t*>(ws + L.piv)[j] = ps;
        }
      }
    }
    __syncthreads();
    if (s_bad) break;                                     // the same column in every CTA
    const int pr = s_pr;
    const int rp = phys[pr];                              // the pivot's physical row
    {
      const cplx* src = cl.map_shared_rank(rows, rp % CN) + (size_t)(rp / CN) * W;
      for (int k = j + 1 + tid; k < W; k += blockDim.x) prow[k] = src[k];
    }
    __syncthreads();                                      // every thread has rp and the pivot row
    if (tid == 0) {                                       // the interchange of positions j and pr
      const int rj = phys[j];
      phys[j] = rp;
      phys[pr] = rj;
      pos[rp] = j;
      pos[rj] = pr;
    }
    __syncthreads();
    const cplx inv = s_inv;
    // the multipliers, warp 0 with a lane per row (one FP64 pass for all rows of the CTA)
    if (wid == 0)
      for (int lr = lane; lr < R; lr += 32)
        if (pos[rank + CN * lr] > j) {
          const cplx l = rows[(size_t)lr * W + j] * inv;
          rows[(size_t)lr * W + j] = l;
          s_l[lr] = l;
        }
    __syncthreads();
    if (wid == 0) {
      // column j + 1 of every row first (lane per row), then its candidates and the winner's
      // reciprocal -- the chain to the next barrier -- while warps 1.. eliminate the rest
      bk = -1;
      bp = 0x7fffffff;
      ba = mk(0.0, 0.0);
      for (int lr = lane; lr < R; lr += 32) {
        const int ps = pos[rank + CN * lr];
        if (ps <= j) continue;
        cplx* row = rows + (size_t)lr * W;
        const cplx a1 = cfms(s_l[lr], prow[j + 1], row[j + 1]);
        row[j + 1] = a1;
        if (j + 1 < p) {
          const long long k1 = clu_key(abs2(a1));
          if (clu_better(k1, ps, bk, bp)) { bk = k1; bp = ps; ba = a1; }
        }
      }
      if (j + 1 < p) {
        for (int o = 16; o > 0; o >>= 1) {
          const long long ok = __shfl_down_sync(0xffffffffu, bk, o);
          const int op = __shfl_down_sync(0xffffffffu, bp, o);
          const double ore = __shfl_down_sync(0xffffffffu, ba.re, o), oim = __shfl_down_sync(0xffffffffu, ba.im, o);
          if (clu_better(ok, op, bk, bp)) { bk = ok; bp = op; ba = mk(ore, oim); }
        }
        if (lane == 0) {
          s_slot[buf ^ 1].key = bk;
          s_slot[buf ^ 1].pos = bp;
          s_slot[buf ^ 1].inv = clu_inv(bk, ba);
        }
      }
    } else if (wid & 3) {
      // columns j + 2 .. W - 1 (y included), a row per warp; the warps that share warp 0's
      // scheduler (wid % 4 == 0) stay out, so that its chain does not queue behind them
      const int bw = wid - 1 - (wid >> 2), nb = nw - (nw + 3) / 4;
      for (int lr = bw; lr < R; lr += nb) {
        if (pos[rank + CN * lr] <= j) continue;
        cplx* __restrict__ row = rows + (size_t)lr * W;
        const cplx* __restrict__ pv = prow;
        const cplx l = s_l[lr];
#pragma unroll 4
        for (int k = j + 2 + lane; k < W; k += 32) row[k] = cfms(l, pv[k], row[k]);
      }
    }
    __syncthreads();
  }
  const bool bad = s_bad != 0;
  // ---- upper solve in blocks of kLuNB rows from the bottom (CTA 0 solves each block's triangle)
  if (!bad) {
    // the diagonal's reciprocals 1 / |u_cc|^2, every row at once (as cdiv forms them)
    for (int lr = tid; lr < R; lr += blockDim.x) s_dv[lr] = 1.0 / abs2(rows[(size_t)lr * W + pos[rank + CN * lr]]);
    for (int b1 = p; b1 > 0; b1 -= kLuNB) {
      const int b0 = b1 - kLuNB > 0 ? b1 - kLuNB : 0;
      const int w = b1 - b0;
      cl.sync();                                          // the block's y (and the reciprocals) are final
      if (rank == 0) {
        for (int t = tid; t < w * (w + 2); t += blockDim.x) {
          const int c = t / (w + 2), v = t - c * (w + 2);  // v = w: y, v = w + 1: the reciprocal
          const int rc = phys[b0 + c];
          const cplx* src = cl.map_shared_rank(rows, rc % CN) + (size_t)(rc / CN) * W;
          if (v < w) sU[c * kLuNB + v] = src[b0 + v];
          else if (v == w) sU[kLuNB * kLuNB + c] = src[p];
          else s_db[c] = *cl.map_shared_rank(&s_dv[rc / CN], rc % CN);
        }
        __syncthreads();
        if (tid == 0) {
          cplx* yb = sU + kLuNB * kLuNB;
          for (int c = w - 1; c >= 0; --c) {
            cplx acc = yb[c];
            for (int v = c + 1; v < w; ++v) acc = acc - sU[c * kLuNB + v] * yb[v];
            yb[c] = cdiv_r(acc, sU[c * kLuNB + c], s_db[c]);
            yfin[b0 + c] = yb[c];
          }
        }
      }
      cl.sync();                                          // the block's solution is in CTA 0
      {
        const cplx* yb0 = cl.map_shared_rank(sU, 0) + kLuNB * kLuNB;
        cplx ybl[kLuNB];
#pragma unroll
        for (int v = 0; v < kLuNB; ++v) ybl[v] = v < w ? yb0[v] : mk(0.0, 0.0);
        for (int lr = tid; lr < R; lr += blockDim.x) {
          const int ps = pos[rank + CN * lr];
          if (ps >= b0) continue;
          cplx* row = rows + (size_t)lr * W;
          cplx acc = row[p];
#pragma unroll
          for (int v = 0; v < kLuNB; ++v)
            if (v < w) acc = acc - row[b0 + v] * ybl[v];
          row[p] = acc;
        }
      }
    }
  }
  // ---- outputs: the factors in logical row order; CTA 0: dFOM (Eq. 4 at the monitor) and D y
  if (!bad) {
    cplx* A = reinterpret_cast<cplx*>(ws + L.lu);
    for (int t = tid; t < R * p; t += blockDim.x) {
      const int lr = t / p, c = t - lr * p;
      A[(size_t)pos[rank + CN * lr] * p + c] = rows[(size_t)lr * W + c];
    }
  }
  if (rank == 0) {
    double df = 0.0;
    if (!bad) {
      for (int mc = 0; mc < a.u.mcount; ++mc) {
        const int64_t m = a.u.mrow + mc;
        cplx part = mk(0.0, 0.0);
        for (int u = tid; u < p; u += blockDim.x) {
          const cplx gm = U.vrows ? ldG(U.vrows, a.u.dtype, U.ldv, u, m) : ldG(U.G, a.u.dtype, U.ldg, m, sV[u]);
          part = part + sD[u] * (gm * yfin[u]);
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
      cplx* yd = reinterpret_cast<cplx*>(ws + L.yd);
      for (int u = tid; u < p; u += blockDim.x) yd[u] = sD[u] * yfin[u];
    }
    if (tid == 0) {
      ctl->lam_df[0] = df;
      ctl->lam_bad[0] = bad ? 1 : 0;
    }
  }
  cl.sync();                                              // no CTA leaves while others read its memory
}

// Launch on a cluster of 16 CTAs where the device holds one (checked once per device), else 8.
static void launch_cap_cluster(const CapArgs& ca, const WsLayout& L, char* ws, const uint8_t* state,
                               const int32_t* idx, const int32_t* status, cudaStream_t st) {
  static std::mutex mu;
  static int cn_of[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int cn = 8;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || cn_of[dev] == 0) {
      cudaFuncSetAttribute(k_cap_cluster<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)cap_cluster_smem(kLuMaxBlocked, 8));
      cudaFuncSetAttribute(k_cap_cluster<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)cap_cluster_smem(kLuMaxBlocked, 16));
      int ok16 = 0;
      if (cudaFuncSetAttribute(k_cap_cluster<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = cap_cluster_smem(kLuMaxBlocked, 16);
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, k_cap_cluster<16>, &cfg) == cudaSuccess && nc >= 1) ok16 = 1;
      }
      cudaGetLastError();                                 // a refused size leaves no error behind
      if (dev >= 0 && dev < 64) cn_of[dev] = ok16 ? 16 : 8;
      cn = ok16 ? 16 : 8;
    } else {
      cn = cn_of[dev];
    }
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cn;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)cn);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = cap_cluster_smem(L.pmax, cn);
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cn == 16)
    cudaLaunchKernelEx(&cfg, k_cap_cluster<16>, ca, L, ws, state, idx, status);
  else
    cudaLaunchKernelEx(&cfg, k_cap_cluster<8>, ca, L, ws, state, idx, status);
}

// ----------------------------------------------------------------------------- panels
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
    constexpr int U = 8;                         // eight rows' loads in flight before their arithmetic
    for (int64_t i = i0; i < iend; i += U) {
      double2 g[U];
#pragma unroll
      for (int q = 0; q < U; ++q)
        if (i + q < iend) g[q] = G[(i + q) * ldg + j];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        if (i + q < iend) {
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

// Batched complex128 FP64 FMA update (small problems): blockIdx.z selects the problem.
__global__ void __launch_bounds__(256) k_rank_update_f64_batch(const BatchItem* __restrict__ items) {
  const BatchItem& it = items[blockIdx.z];
  const UpdCtl* ctl = reinterpret_cast<const UpdCtl*>(it.ws + it.L.ctl);
  const int p = ctl->skip ? 0 : ctl->nv;
  const int64_t n = it.L.n;
  if (p < 1 || (int64_t)blockIdx.x * 256 >= n) return;
  for (int64_t rt = blockIdx.y; rt * kF64BatchRows < n; rt += gridDim.y)
    f64_update_tile(reinterpret_cast<double2*>(it.G), it.ldg, n, it.L.pmax, p,
                    reinterpret_cast<const cplx*>(it.ws + it.L.C0), reinterpret_cast<const cplx*>(it.ws + it.L.S), rt,
                    blockIdx.x);
}

void launch_rank_update_f64_batch(const BatchItem* items, int nprob, int64_t widest_n, cudaStream_t st) {
  int64_t rt = (widest_n + kF64BatchRows - 1) / kF64BatchRows;
  if (rt > 65535) rt = 65535;
  k_rank_update_f64_batch<<<dim3((unsigned)((widest_n + 255) / 256), (unsigned)rt, (unsigned)nprob), 256, 0, st>>>(items);
}

void launch_rank_update_c64_fp32_batch(const BatchItem* items, int nprob, int ctas, cudaStream_t st) {
  k_rank_update_c64_fp32_batch<<<ctas, kF32Threads, 0, st>>>(items, nprob);
}

// ----------------------------------------------------------------------------- field, state, FOM
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
    launch_cap_cluster(ca, L, ws, state, idx, status, st);
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
