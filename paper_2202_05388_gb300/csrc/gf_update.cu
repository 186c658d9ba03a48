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
  // p_max <= kMaxPixelsPerCand: every system of the step takes the warp form (no shared matrix)
  const bool smem = L.pmax > kMaxPixelsPerCand && L.pmax <= kCapSmemP;
  capacitance_body(a, L, ws, state, idx, status, smem ? reinterpret_cast<cplx*>(cap_smem) : nullptr, pre != 0);
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
  cplx* sA = L.pmax > kMaxPixelsPerCand ? reinterpret_cast<cplx*>(cap_smem) : nullptr;
  const bool ok = p > 0 ? cap_lam(a, L, ws, l, p, sV, sD, sA, &df) : true;
  if (threadIdx.x == 0) {
    ctl->lam_df[l] = df;
    ctl->lam_bad[l] = ok ? 0 : 1;
  }
}

// ---- one large system per wavelength (p_max > kCapClusterMinP), held in the shared memory of one
// cluster of CTAs per wavelength (distributed shared memory; cluster l of the grid solves
// wavelength l).  One CTA per solve is bound by that SM's FP64
// pipe (p = 128: 1.9 ms).  A = I - G_VV D is built, factorised with partial pivoting and solved
// without leaving the cluster: physical row r (with y as its last entry) lives in CTA r % CN and
// is never moved; the logical order is recorded per row.
//
// GB300's FP64 pipe is shared by the SM's four schedulers (a dependent FP64 operation of one warp
// takes 32 ns; eight warps with dependent chains take 77 ns per operation each), so the per-column
// chain of one warp slows down whenever other warps keep the pipe busy.  A column therefore runs in
// two halves around one split cluster barrier:
//   before the arrive (the chain): warp 0 reads every CTA's candidate (key, physical row,
//   reciprocal, the entry after the pivot column) and takes the pivot (largest modulus, lowest
//   physical row on ties), then forms the multipliers of its CTA's rows, eliminates the next column
//   of every row, and picks the CTA's candidate for the next column, whose reciprocal it forms for
//   every row at once while the keys are reduced.  Meanwhile warps 1-7 copy the pivot row from
//   its owner's published candidate row.  The candidate row is then eliminated in full by warps
//   1-7 and published with its key (a CTA's candidate is the only row others read);
//   after the arrive (the bulk): every warp eliminates the remaining rows, while the barrier
//   gathers the other CTAs' candidates.
// So a column costs one cluster barrier, two rounds of distributed-shared-memory loads and one
// chain of six dependent FP64 operations; the bulk elimination overlaps the barrier.  The
// candidate rows and keys are double-buffered by column parity: a buffer is rewritten two columns
// later, after a barrier that every reader of it has passed.
// Upper solve: the inverses of the 8 x 8 diagonal blocks of U are formed in parallel (a block per
// CTA), after which a block of x costs one barrier: every CTA computes x_b = U_bb^{-1} y_b from the
// owners' y entries (the same bits everywhere) and updates y of its own rows above the block.
// Outputs: V, dchi, the factors (row-major, logical order), pivots (as row interchanges in order)
// and D y in the workspace, the dFOM and singular flag in the control block, where k_capacitance's
// first attempt reads them.  CN = 16 CTAs where the device can hold such a cluster (a non-portable
// size), else 8.  Candidates are compared as integers: |a|^2 >= 0, and the bit patterns of
// non-negative doubles order as the values do, so the key is the bit pattern (-1 for NaN, which
// never wins), off the FP64 pipe.
struct CluSlot {                 // a CTA's candidate for the next pivot
  cplx inv;                      // conj(a) / |a|^2 of its entry a in the pivot column
  cplx un;                       // its entry in the column after the pivot column
  long long key;                 // bit pattern of |a|^2 (-1: no candidate)
  int ph;                        // its physical row (0x7fffffff: none)
};
__device__ __forceinline__ long long clu_key(double v) {
  const long long b = __double_as_longlong(v);
  return (b & 0x7FFFFFFFFFFFFFFFll) > 0x7FF0000000000000ll ? -1ll : b;
}
__device__ __forceinline__ bool clu_better(long long k, int ph, long long bk, int bph) {
  return k > bk || (k == bk && ph < bph);
}
// conj(a) / |a|^2 (without a branch: for no candidate, key <= 0, the value is not used)
__device__ __forceinline__ cplx clu_inv(long long key, cplx a) {
  const double d = rcp_nr_i(__longlong_as_double(key > 0 ? key : 0x3FF0000000000000ll));
  return mk(a.re * d, -a.im * d);
}
// a b and |a|^2 with fused multiply-adds (two dependent FP64 operations each)
__device__ __forceinline__ cplx clu_mul(cplx a, cplx b) {
  return mk(fma(a.re, b.re, -(a.im * b.im)), fma(a.re, b.im, a.im * b.re));
}
__device__ __forceinline__ double clu_abs2(cplx a) { return fma(a.re, a.re, a.im * a.im); }
// the best (key, physical row) over lanes [0, 2 o0) of the warp, in each of those lanes (an
// exchange butterfly, o0 a power of two); the values that go with it are then fetched from the
// winning lane, so the reduction does not wait for them
__device__ __forceinline__ void clu_best(long long& k, int& ph, int o0) {
  for (int o = o0; o > 0; o >>= 1) {
    const long long ok = __shfl_xor_sync(0xffffffffu, k, o);
    const int op = __shfl_xor_sync(0xffffffffu, ph, o);
    if (clu_better(ok, op, k, ph)) {
      k = ok;
      ph = op;
    }
  }
}
__device__ __forceinline__ cplx clu_from(cplx v, int src) {
  return mk(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
}
// the split cluster barrier: each thread arrives (releasing its writes) and later waits
// (acquiring everyone's); every thread of every CTA runs the same sequence
__device__ __forceinline__ void clu_arrive() { asm volatile("barrier.cluster.arrive.release;\n" ::: "memory"); }
__device__ __forceinline__ void clu_wait() { asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory"); }

__host__ __device__ constexpr size_t cap_cluster_smem(int pmax, int cn) {
  // rows (R x W) | candidate rows (2 W) | pivot row (W) | inverted diagonal blocks of U
  // (nb kLuNB^2) | x (pmax) | dchi (pmax) | V, permrow, phys, pos (pmax each) | posof (R)
  return sizeof(cplx) * ((size_t)((pmax + cn - 1) / cn) * (pmax + 1) + 3 * (size_t)(pmax + 1) +
                         (size_t)((pmax + kLuNB - 1) / kLuNB) * kLuNB * kLuNB + pmax) +
         sizeof(double) * (size_t)pmax + sizeof(int32_t) * (4 * (size_t)pmax + (pmax + cn - 1) / cn);
}

template <int CN>
__global__ void __launch_bounds__(256)
    k_cap_cluster(CapArgs a, WsLayout L, char* ws, const uint8_t* state, const int32_t* idx, const int32_t* status) {
  namespace cg = cooperative_groups;
  static_assert(kLuNB == 8, "the upper solve maps 8 x 8 blocks onto groups of 8 lanes");
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char clu_smem[];
  const int pm = L.pmax;
  const int Rm = (pm + CN - 1) / CN;                      // <= 32 (pm <= kLuMaxBlocked, CN >= 8)
  const int W = pm + 1;                                   // row stride: p columns of A, then y
  const int nbm = (pm + kLuNB - 1) / kLuNB;
  cplx* rows = reinterpret_cast<cplx*>(clu_smem);
  cplx* crow = rows + (size_t)Rm * W;                     // candidate rows, by column parity
  cplx* prow = crow + 2 * (size_t)W;
  cplx* Zb = prow + W;                                    // block b: (U_bb)^{-1}, row-major 8 x 8
  cplx* xfin = Zb + (size_t)nbm * kLuNB * kLuNB;
  double* sD = reinterpret_cast<double*>(xfin + pm);
  int32_t* sV = reinterpret_cast<int32_t*>(sD + pm);
  int32_t* permrow = sV + pm;                             // the physical row at each logical position
  int32_t* phys = permrow + pm;                           // CTA 0: the interchanges in order
  int32_t* pos = phys + pm;
  int32_t* posof = pos + pm;                              // a local row's logical position (-1: live)
  __shared__ CluSlot s_cands[2][CN];                      // every CTA's candidate, pushed by its owner
  __shared__ cplx s_l[32];                                // the column's multipliers, by local row
  __shared__ int s_bl[32];                                // the rows of the bulk elimination
  __shared__ cplx s_inv, s_un;
  __shared__ cplx s_T[kLuNB * kLuNB];
  __shared__ double s_dd[kLuNB];
  __shared__ double s_red[8], s_bv[8];
  __shared__ double s_thr, s_rmax;
  __shared__ int s_nv, s_bad, s_ph, s_cand, s_nbulk;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = (int)(blockDim.x >> 5);
  const int rank = (int)cl.block_rank();
  const int lam = (int)(blockIdx.x / CN);                 // cluster l solves wavelength l
  const UpdLam& U = a.u.lam[lam];
  UpdCtl* ctl = reinterpret_cast<UpdCtl*>(ws + L.ctl);
  int32_t* piv_out = reinterpret_cast<int32_t*>(ws + L.piv + lam * L.piv_s);

  // ---- the joint set V: the candidates in order up to the first empty slot, a lane per
  // candidate (pillars, whose pixel count has no small bound: one thread)
  if (a.kind != GF_KIND_PILLAR && a.k <= 32) {
    if (wid == 0) {
      int32_t v4[kMaxPixelsPerCand];
      double d4[kMaxPixelsPerCand];
      const int32_t id = (lane < a.k && *status == GF_OK) ? idx[lane] : -1;
      const unsigned neg = __ballot_sync(0xffffffffu, id < 0);
      const int first = neg ? __ffs(neg) - 1 : 32;
      int cnt = 0;
      if (lane < first) cnt = cand_pixels(id, a.kind, a.dir_mask, a.u.nx, a.u.ny, a.u.chi, state, v4, d4, a.u.nz);
      int off = cnt;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += t;
      }
      const int total = __shfl_sync(0xffffffffu, off, 31);
      off -= cnt;
      for (int u = 0; u < cnt; ++u) {
        sV[off + u] = v4[u];
        sD[off + u] = d4[u];
      }
      if (lane == 0) {
        s_nv = total;
        s_bad = 0;
      }
    }
  } else if (tid == 0) {
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
      if (lam == 0) {                                     // the set, shared by the wavelengths
        V[t] = sV[t];
        dchi[t] = sD[t];
      }
      phys[t] = t;
      pos[t] = t;
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
  for (int lr = tid; lr < Rm; lr += blockDim.x) posof[lr] = -1;
  __syncthreads();
  double rmax = 0.0;
  for (int lr = wid; lr < R; lr += nw) {
    double sum = 0.0;
    for (int c = lane; c < p; c += 32) sum += cabs1(rows[(size_t)lr * W + c]);
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    rmax = fmax(rmax, sum);                               // lane 0 holds the row's sum
  }
  if (lane == 0) s_red[wid] = rmax;
  // the candidates of column 0, a lane per row
  if (wid == 0) {
    long long k = -1;
    int ph = 0x7fffffff;
    cplx iv = mk(0.0, 0.0), un = mk(0.0, 0.0);
    if (lane < R) {
      const cplx a0 = rows[(size_t)lane * W];
      k = clu_key(clu_abs2(a0));
      ph = rank + CN * lane;
      iv = clu_inv(k, a0);
      un = rows[(size_t)lane * W + 1];
    }
    clu_best(k, ph, 16);
    const int src = ph != 0x7fffffff ? ph / CN : 0;
    iv = clu_from(iv, src);
    un = clu_from(un, src);
    if (lane < CN) {                                      // lane q pushes the candidate to CTA q
      CluSlot* d = cl.map_shared_rank(&s_cands[0][rank], lane);
      d->key = k;
      d->ph = ph;
      d->inv = iv;
      d->un = un;
    }
    if (lane == 0) s_cand = ph != 0x7fffffff ? ph / CN : -1;
  }
  __syncthreads();
  if (s_cand >= 0)
    for (int c = tid; c <= p; c += blockDim.x) crow[c] = rows[(size_t)s_cand * W + c];
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < nw; ++w) m = fmax(m, s_red[w]);
    s_rmax = m;
  }
  cl.sync();                                              // column 0's candidates, the row sums
  if (wid == 0) {                                         // the pivot threshold kSingularRel ||A||_inf
    double m = lane < CN ? *cl.map_shared_rank(&s_rmax, lane) : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if (lane == 0) s_thr = kSingularRel * m;
  }
  __syncthreads();
  const long long thr2_key = clu_key(s_thr * s_thr);
  const int rspan = Rm > 16 ? 16 : Rm > 8 ? 8 : Rm > 4 ? 4 : Rm > 2 ? 2 : 1;   // lanes [0, 2 rspan) hold rows

  // ---- factorisation, one split cluster barrier per column
  bool bad = false;
  bool mine = lane < R;                                   // warp 0: this lane's row is not yet pivoted
  for (int j = 0; j < p; ++j) {
    const int buf = j & 1;
    if (j > 0) clu_wait();                                // column j's candidates are published
    if (wid == 0) {                                       // lane q takes CTA q's candidate
      long long k = -1;
      int ph = 0x7fffffff;
      cplx iv = mk(0.0, 0.0), un = mk(0.0, 0.0);
      if (lane < CN) {
        const CluSlot& sl = s_cands[buf][lane];
        k = sl.key;
        ph = sl.ph;
        iv = sl.inv;
        un = sl.un;
      }
      clu_best(k, ph, CN / 2);
      const int src = ph != 0x7fffffff ? ph % CN : 0;
      iv = clu_from(iv, src);
      un = clu_from(un, src);
      if (lane == 0) {
        // |pv|^2 >= thresh^2 and > 0 (a NaN key is -1 and fails both)
        if (k < thr2_key || k <= 0) {
          s_bad = 1;
        } else {
          s_ph = ph;
          s_inv = iv;
          s_un = un;
        }
      }
    }
    __syncthreads();                                      // the pivot; this CTA's bulk of column j - 1 is done
    if (s_bad) {                                          // the same column in every CTA
      bad = true;
      break;
    }
    const int rp = s_ph, w = rp % CN, lw = rp / CN;       // the pivot's physical row, owner, local row
    long long bk = -1;                                    // warp 0: the CTA's candidate for column j + 1
    int bph = 0x7fffffff;
    cplx iv = mk(0.0, 0.0);
    if (wid == 0) {
      const cplx inv = s_inv, un = s_un;
      const bool piv = w == rank && lane == lw;
      const bool live = mine && !piv;
      cplx l = mk(0.0, 0.0), a1 = mk(0.0, 0.0);
      if (live) {
        cplx* row = rows + (size_t)lane * W;
        l = clu_mul(row[j], inv);
        row[j] = l;
        a1 = cfms(l, un, row[j + 1]);
        row[j + 1] = a1;
      }
      if (piv) {
        posof[lane] = j;
        mine = false;
      }
      s_l[lane] = l;
      if (live && j + 1 < p) {
        bk = clu_key(clu_abs2(a1));
        bph = rank + CN * lane;
      }
      // every row's reciprocal is started before the reduction of the keys, which runs on the
      // integer and shuffle units meanwhile; the winner's is taken after the barrier below
      iv = clu_inv(bk, a1);
      clu_best(bk, bph, rspan);
      bk = __shfl_sync(0xffffffffu, bk, 0);
      bph = __shfl_sync(0xffffffffu, bph, 0);
      const int cand = (j + 1 < p && bph != 0x7fffffff) ? bph / CN : -1;
      const bool bulk = live && lane != cand;
      const unsigned bm = __ballot_sync(0xffffffffu, bulk);
      if (bulk) s_bl[__popc(bm & ((1u << lane) - 1u))] = lane;
      if (lane == 0) {
        s_nbulk = __popc(bm);
        s_cand = cand;
      }
    } else {
      const cplx* src = cl.map_shared_rank(crow + (size_t)buf * W, w);
      for (int c = j + 1 + tid - 32; c <= p; c += (int)blockDim.x - 32) prow[c] = src[c];
      if (tid == 32) permrow[j] = rp;
      if (rank == 0 && tid == 64) {                       // the interchange of positions j and pos[rp]
        const int ps = pos[rp], rj = phys[j];
        piv_out[j] = ps;
        phys[j] = rp;
        phys[ps] = rj;
        pos[rp] = j;
        pos[rj] = ps;
      }
    }
    __syncthreads();                                      // pivot row, multipliers, the CTA's candidate
    const int cand = s_cand;
    if (wid == 0) {
      if (j + 1 < p) {
        // the candidate's entry in column j + 2 (every lane forms the same bits; lane 0 stores
        // it), then key, row, reciprocal and that entry: lane q to CTA q
        cplx un2 = mk(0.0, 0.0);
        if (cand >= 0) {
          cplx* row = rows + (size_t)cand * W;
          un2 = cfms(s_l[cand], prow[j + 2], row[j + 2]);
          __syncwarp();
          if (lane == 0) {
            row[j + 2] = un2;
            crow[(size_t)(buf ^ 1) * W + j + 2] = un2;
          }
        }
        const cplx ivw = clu_from(iv, cand >= 0 ? cand : 0);
        if (lane < CN) {
          CluSlot* d = cl.map_shared_rank(&s_cands[buf ^ 1][rank], lane);
          d->key = bk;
          d->ph = bph;
          d->inv = ivw;
          d->un = un2;
        }
      }
    } else if (cand >= 0) {                               // the rest of the candidate row, published
      cplx* row = rows + (size_t)cand * W;
      cplx* dst = crow + (size_t)(buf ^ 1) * W;
      const cplx lc = s_l[cand];
      for (int c = j + 1 + tid - 32; c <= p; c += (int)blockDim.x - 32) {
        if (c == j + 2) continue;                         // warp 0's
        cplx v = row[c];
        if (c > j + 1) {
          v = cfms(lc, prow[c], v);
          row[c] = v;
        }
        dst[c] = v;
      }
    }
    clu_arrive();                                         // column j + 1's candidates are published
    {
      // the bulk: columns j + 2 .. p of the remaining rows, a warp per row
      const int nl = s_nbulk;
      for (int q = wid; q < nl; q += nw) {
        const int lr = s_bl[q];
        cplx* row = rows + (size_t)lr * W;
        const cplx l = s_l[lr];
#pragma unroll 4
        for (int c = j + 2 + lane; c <= p; c += 32) row[c] = cfms(l, prow[c], row[c]);
      }
    }
  }
  if (p > 0 && !bad) clu_wait();                         // the last column's arrive
  // ---- upper solve U x = y
  if (!bad && p > 0) {
    const int nb = (p + kLuNB - 1) / kLuNB;
    // the diagonal blocks inverted, block b by CTA b % CN: column k of T^{-1} by thread k, from
    // the bottom row up (T = U_bb upper triangular, its diagonal bounded away from 0 by the
    // pivot threshold)
    for (int b = rank; b < nb; b += CN) {
      const int b0 = b * kLuNB, wb = p - b0 < kLuNB ? p - b0 : kLuNB;
      if (tid < kLuNB * kLuNB) {
        const int i = tid >> 3, m = tid & 7;
        cplx v = mk(0.0, 0.0);
        if (i < wb && m < wb && m >= i) {
          const int rc = permrow[b0 + i];
          v = cl.map_shared_rank(rows, rc % CN)[(size_t)(rc / CN) * W + b0 + m];
        }
        s_T[tid] = v;
      }
      __syncthreads();
      if (tid < wb) s_dd[tid] = 1.0 / clu_abs2(s_T[tid * kLuNB + tid]);
      __syncthreads();
      cplx* Z = Zb + (size_t)b * kLuNB * kLuNB;
      if (tid < kLuNB) {
        const int k = tid;
        for (int i = kLuNB - 1; i >= 0; --i) {
          cplx z = mk(0.0, 0.0);
          if (k < wb && i <= k) {
            const cplx t = s_T[i * kLuNB + i];
            const cplx ti = mk(t.re * s_dd[i], -t.im * s_dd[i]);   // 1 / T_ii
            if (i == k) {
              z = ti;
            } else {
              cplx s = mk(0.0, 0.0);
              for (int m = i + 1; m <= k; ++m) s = cfma(s_T[i * kLuNB + m], Z[m * kLuNB + k], s);
              z = clu_mul(s, ti);
              z = mk(-z.re, -z.im);
            }
          }
          Z[i * kLuNB + k] = z;
        }
      }
      __syncthreads();
    }
    cl.sync();                                            // every block's inverse is with its CTA
    for (int t = tid; t < nb * kLuNB * kLuNB; t += blockDim.x) {
      const int b = t / (kLuNB * kLuNB);
      if (b % CN != rank) Zb[t] = cl.map_shared_rank(Zb, b % CN)[t];
    }
    __syncthreads();
    // the blocks from the bottom, one barrier each: x_b = U_bb^{-1} y_b in every CTA (the y
    // entries of the block's rows are final once the blocks below have been applied), then
    // y_r -= U_rb x_b for the CTA's rows above the block
    for (int b = nb - 1; b >= 0; --b) {
      const int b0 = b * kLuNB, wb = p - b0 < kLuNB ? p - b0 : kLuNB;
      if (b < nb - 1) clu_wait();                         // the updates of the block below
      if (tid < kLuNB * kLuNB) {                          // warps 0 and 1: lane group i, lane m
        const int i = tid >> 3, m = tid & 7;
        cplx pr = mk(0.0, 0.0);
        if (i < wb && m < wb && m >= i) {
          const int rc = permrow[b0 + m];
          const cplx ym = cl.map_shared_rank(rows, rc % CN)[(size_t)(rc / CN) * W + p];
          pr = clu_mul(Zb[(size_t)b * kLuNB * kLuNB + i * kLuNB + m], ym);
        }
        for (int o = 4; o > 0; o >>= 1) {
          pr.re += __shfl_xor_sync(0xffffffffu, pr.re, o);
          pr.im += __shfl_xor_sync(0xffffffffu, pr.im, o);
        }
        if (m == 0 && i < wb) xfin[b0 + i] = pr;
      }
      __syncthreads();
      {                                                   // thread (local row tid / 8, block column tid % 8)
        const int lr = tid >> 3, m = tid & 7;
        const bool act = lr < R && posof[lr] < b0;
        cplx pr = mk(0.0, 0.0);
        if (act && m < wb) pr = clu_mul(rows[(size_t)lr * W + b0 + m], xfin[b0 + m]);
        for (int o = 4; o > 0; o >>= 1) {
          pr.re += __shfl_xor_sync(0xffffffffu, pr.re, o);
          pr.im += __shfl_xor_sync(0xffffffffu, pr.im, o);
        }
        if (act && m == 0) rows[(size_t)lr * W + p] = rows[(size_t)lr * W + p] - pr;
      }
      if (b > 0) clu_arrive();                            // released to the next block's readers
    }
  }
  // ---- outputs: the factors in logical row order; CTA 0: dFOM (Eq. 4 at the monitor) and D y
  if (!bad) {
    cplx* A = reinterpret_cast<cplx*>(ws + L.lu + lam * L.lu_s);
    for (int t = tid; t < R * p; t += blockDim.x) {
      const int lr = t / p, c = t - lr * p;
      A[(size_t)posof[lr] * p + c] = rows[(size_t)lr * W + c];
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
          part = part + sD[u] * (gm * xfin[u]);
        }
        for (int o = 16; o > 0; o >>= 1) {
          part.re += __shfl_down_sync(0xffffffffu, part.re, o);
          part.im += __shfl_down_sync(0xffffffffu, part.im, o);
        }
        if (lane == 0) {
          s_bv[wid] = part.re;
          s_red[wid] = part.im;
        }
        __syncthreads();
        if (tid == 0) {
          cplx dE = mk(0.0, 0.0);
          for (int w = 0; w < nw; ++w) dE = dE + mk(s_bv[w], s_red[w]);
          const cplx EN = U.E[m];
          df += abs2(EN + dE) - abs2(EN);
        }
        __syncthreads();
      }
      cplx* yd = reinterpret_cast<cplx*>(ws + L.yd + lam * L.yd_s);
      for (int u = tid; u < p; u += blockDim.x) yd[u] = sD[u] * xfin[u];
    }
    if (tid == 0) {
      ctl->lam_df[lam] = df;
      ctl->lam_bad[lam] = bad ? 1 : 0;
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
  cfg.gridDim = dim3((unsigned)(cn * ca.u.nlam));            // one cluster per wavelength
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
  // the shared-memory system for kMaxPixelsPerCand < p_max <= kCapSmemP (a smaller set takes the
  // warp form, which needs none: no carve-out change between the step's kernels)
  const size_t cap_smem = L.pmax > kMaxPixelsPerCand && L.pmax <= kCapSmemP
                              ? sizeof(cplx) * ((size_t)kCapSmemP * kCapSmemP + kCapSmemP) : 0;
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
  // the first attempt's solves: one cluster of CTAs per wavelength for a set above
  // kCapClusterMinP pixels (a 64-pixel system: 0.18 ms against 0.47 ms on one CTA), else one CTA
  // per wavelength side by side (several wavelengths); k_capacitance decides and runs any fallback
  const bool multi = L.pmax > kCapClusterMinP && L.pmax <= kLuMaxBlocked;
  const int pre = (a.nlam > 1 && L.pmax <= kCapSmemP) || multi ? 1 : 0;
  if (multi) {
    launch_cap_cluster(ca, L, ws, state, idx, status, st);
  } else if (pre) {
    k_capacitance_lam<<<a.nlam, 256, cap_smem, st>>>(ca, L, ws, state, idx, status);
  }
  k_capacitance<<<1, 256, cap_smem, st>>>(ca, L, ws, state, idx, status, pre);
  const int64_t n = L.n;
  const int64_t rows = a.lam[0].rows;       // rows of G held (n, or a shard's row block)
  // complex64 on the tensor cores: S is formed from an explicit D A^{-1} by an FP32 GEMM and C0
  // is gathered together with the operand rows, so the panels kernel does not run
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
  if (!c64tc) {         // complex64 on the tensor cores gathers C0 with its operand rows
    const int64_t w = rows > n ? rows : n;
    int64_t b = (w + 255) / 256;
    k_panels<<<(int)(b < 4864 ? b : 4864), 256, 0, st>>>(a, L, ws, 1);
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
