// FP64-accurate rank-p update of a complex128 G on the tensor cores (Eq. 10: G += C0 S with
// C0 = G[:, V] and S = D A^{-1} G[V, :] from Eq. 14).
//
// GB300 executes FP64 FMA at ~1/64 of the FP32 rate, so the plain complex128 update (16 DFMA
// per entry at p = 4) is bound by the FP64 pipe at ~18% of HBM bandwidth.  Here the products
// are formed exactly on the tensor cores instead:
//
//   * The update is written as one real GEMM (the "4M" form): row i of A' is
//     [Re C0[i, 0..4), Im C0[i, 0..4)], and output column 2j (2j+1) of B' holds
//     [Re S[., j], -Im S[., j]] ([Im S[., j], Re S[., j]]), so that A' B' gives Re and Im of
//     (C0 S)[i, j] in adjacent columns.  K = 8.
//   * Each row of A' is scaled by a power of two 2^E_i (each column of B' by 2^F_j) so its
//     entries lie in (-1, 1) and is split into six signed 9-bit integer digits,
//     x = sum_a d_a 2^(-9a) + O(2^-55).  Digits are exact in TF32.
//   * For every digit pair (a, b) with a + b <= 7 one tcgen05.mma (M = 128, N = 32, K = 8)
//     accumulates d_a(A') d_b(B') into the FP32 TMEM accumulator of level L = a + b.  All
//     partial sums are integers below 2^22, so every level is exact.
//   * The epilogue reads the six levels from TMEM, recombines them exactly in int64
//     (sum_L acc_L 2^(9(7-L))), turns the result into a double with integer operations and
//     adds it to G with one FP64 add per real component.
//
// The result equals the FP64 product to about 2^-50 of |C0| |S| per step, inside the 1e-10
// tolerance of the FP64 path, and uses the FP64 pipe for 2 adds per entry instead of 16 FMAs.
#include <math.h>

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <new>

#include "gf_internal.cuh"
#include "gf_stage_bodies.cuh"
#include "gf_tc.cuh"

namespace gf {

__global__ void k_oz_prep_rows(const cplx* __restrict__ C0, int pmax, int64_t n, int64_t nrows_pad,
                               const UpdCtl* __restrict__ ctl, uint8_t* __restrict__ ozA,
                               int32_t* __restrict__ ozE) {
  oz_prep_rows_body(C0, pmax, n, nrows_pad, ctl, ozA, ozE);
}

__global__ void k_oz_prep_cols(const cplx* __restrict__ S, int64_t n, int64_t ncols_pad,
                               const UpdCtl* __restrict__ ctl, uint8_t* __restrict__ ozB) {
  oz_prep_cols_body(S, n, ncols_pad, ctl, ozB);
}

// Batched preparation: blockIdx.y selects the problem; rows and columns of its digit blocks
// come from the panels in its own workspace.
__global__ void k_oz_prep_batch(const BatchItem* __restrict__ items) {
  const BatchItem& it = items[blockIdx.y];
  const int64_t n = it.L.n;
  const UpdCtl* ctl = reinterpret_cast<const UpdCtl*>(it.ws + it.L.ctl);
  const int64_t rows = ((n + kOzM - 1) / kOzM) * kOzM;
  const int64_t cols = ((2 * n + kOzN - 1) / kOzN) * (kOzN / 2);
  oz_prep_rows_body(reinterpret_cast<const cplx*>(it.ws + it.L.C0), it.L.pmax, n, rows, ctl,
                    reinterpret_cast<uint8_t*>(it.ws + it.L.ozA), reinterpret_cast<int32_t*>(it.ws + it.L.ozE));
  oz_prep_cols_body(reinterpret_cast<const cplx*>(it.ws + it.L.S), n, cols, ctl,
                    reinterpret_cast<uint8_t*>(it.ws + it.L.ozB));
}

// ---- epilogue arithmetic --------------------------------------------------------------------
// Exact recombination of the six FP32 levels (each an integer below 2^22 in its own unit
// 2^(-9 (L+2))) into one int64 in units of 2^-59.  Adjacent levels are first joined in int32:
// |acc_L| <= 2^21.8, so |acc_L 2^9 + acc_(L+1)| < 2^31.  The float -> int conversion adds
// 1.5 * 2^23 so that the integer sits in the low mantissa bits.
__device__ __forceinline__ long long oz_combine(const float (&acc)[kOzLv]) {
  constexpr int32_t M = 0x4B400000;            // bit pattern of 1.5 * 2^23
  const int32_t b0 = __float_as_int(acc[0] + 12582912.0f) - M;
  const int32_t b1 = __float_as_int(acc[1] + 12582912.0f) - M;
  const int32_t b2 = __float_as_int(acc[2] + 12582912.0f) - M;
  const int32_t b3 = __float_as_int(acc[3] + 12582912.0f) - M;
  const int32_t b4 = __float_as_int(acc[4] + 12582912.0f) - M;
  const int32_t b5 = __float_as_int(acc[5] + 12582912.0f) - M;
  const int32_t P1 = (b0 << 9) + b1;           // units 2^-27
  const int32_t P2 = (b2 << 9) + b3;           // units 2^-45
  const int32_t P3 = (b4 << 9) + b5;           // units 2^-63
  return ((long long)P1 << 32) + ((long long)P2 << 14) + (long long)((P3 + 8) >> 4);
}

// D * 2^u as a double, built with integer operations (|D| < 2^62; the 53-bit mantissa is
// truncated, an error below 2^-52 of |D 2^u|).
__device__ __forceinline__ double oz_to_double(long long D, int u) {
  const long long sg = D >> 63;                                   // 0 or -1
  unsigned long long M = (unsigned long long)((D ^ sg) - sg);     // |D|
  const int lz = __clzll(M);
  M <<= (lz & 63);
  const unsigned long long mant = M >> 11;                        // leading one at bit 52
  const long long e = 63 - lz + u;
  unsigned long long bits = ((unsigned long long)(e + 1022) << 52) + mant;
  bits |= (unsigned long long)sg & 0x8000000000000000ull;
  return D == 0 ? 0.0 : __longlong_as_double((long long)bits);
}

// ---- the update kernel ----------------------------------------------------------------------
// Persistent, warp-specialised.  Work = the (128-row tile, 16-complex-column tile) grid in
// row-major order, split into equal contiguous ranges, one per CTA.
//   warp 16      producer: TMA copies of the A digit tile when the row tile changes, and per
//                tile the G tile (two 128-row x 128-byte boxes through a tensor map, 128B
//                swizzle) plus the B digit block into a 4-stage shared-memory ring;
//   warp 17      MMA issuer: 21 tcgen05.mma per tile into one of two TMEM buffers;
//   warps 0..15  epilogue: TMEM -> registers, exact recombination, G += delta in shared
//                memory;
//   warp 18      storer: once all epilogue threads have written a tile, TMA-stores its two
//                boxes back to HBM (the tensor map clips ragged edges) and frees the stage
//                when the stores have read shared memory.
// Every wait is bounded (globaltimer) and can be aborted; a timeout sets GF_ETIMEOUT.
constexpr int kOzNS = 4;                          // shared-memory stages
constexpr int kOzBox = kOzM * 128;                // one TMA box: 128 rows x 128 B (8 complex128)
constexpr int kOzGTile = 2 * kOzBox;              // 32768: the tile's two boxes, 128B-swizzled
constexpr int kOzBBlock = kOzTileB + 64;          // digit slices + 16 column exponents
constexpr int kOzStage = 39936;                   // kOzGTile + kOzBBlock, 1024-aligned
constexpr int kOzBarOff = 2 * kOzTileA + kOzNS * kOzStage;
constexpr int kOzSmemV2 = kOzBarOff + 256;
constexpr int kOzEpiThreads = 512;
constexpr int kOzThreadsV2 = 608;
constexpr int kOzTmemColsV2 = 512;                // two accumulator sets of kOzLv * kOzN columns
constexpr int kEpiWarps = kOzEpiThreads / 32;    // 16
constexpr int kWarpProd = kEpiWarps, kWarpMma = kEpiWarps + 1, kWarpStore = kEpiWarps + 2;
constexpr int kOzColsPerThread = 4;               // complex columns per epilogue thread per tile
static_assert(kOzThreadsV2 == 32 * (kEpiWarps + 3), "warp roles");
static_assert(kEpiWarps / 4 * kOzColsPerThread == kOzN / 2, "column split");
static_assert(kOzGTile + kOzBBlock <= kOzStage, "stage layout");
static_assert(kOzLv * kOzN <= 256, "TMEM buffer");

struct OzBars {
  uint64_t full[kOzNS], empty[kOzNS], ebar[kOzNS];
  uint64_t afull[2], aempty[2], tfull[2], tempty[2];
  uint32_t tslot;
  int abort;
};

// Where the tiles come from.  A source enumerates the work as tiles t in [0, total) in raster
// order and maps each to (problem b, row tile rt, column tile ct); row tiles of one problem
// are consecutive so that the A digit tile is reused along the row.
struct OzProb {
  int64_t n, nrt, nct;
  const uint8_t* ozA;
  const int32_t* ozE;
  const uint8_t* ozB;
};

// A role walks its contiguous tile range with a cursor: one division at the start, then
// increments (the epilogue is issue-bound, so no per-tile 64-bit division or search).
struct OzCursor {
  int b;
  int64_t rt, ct;
  int64_t step;             // tiles between this CTA's consecutive tiles in row-major order
};

// One problem.  When a row of tiles holds at least one tile per CTA and its B digit blocks
// fit in kOzInterleaveMaxB, CTA c takes tiles c, c + g, c + 2g, ... (g CTAs): at any moment the
// CTAs stream adjacent column tiles of the same 128 rows, so that HBM sees long contiguous runs
// per row instead of 152 separate row tiles (7.51 -> 7.37 ms at n = 36865); the A digit tile
// then changes about every nct / g tiles (L2-resident, double-buffered).  Every row of tiles
// re-reads all B blocks in this order, which pays only while they stay in L2 against the G
// stream: at n = 102401 (40 MB of blocks) it measured 63.6 ms against 57.4 ms for contiguous
// ranges.  Otherwise each CTA takes a contiguous range.
constexpr int64_t kOzInterleaveMaxB = int64_t(16) << 20;
struct OzSingleSrc {
  const CUtensorMap* map;
  OzProb pr;
  __device__ int64_t total() const { return pr.nrt * pr.nct; }
  __device__ void range(int64_t c, int64_t g, int64_t& tb, int64_t& te, int64_t& ts) const {
    const int64_t T = total();
    if (pr.nct >= g && pr.nct * kOzBBlock <= kOzInterleaveMaxB) {
      tb = c;
      te = T;
      ts = g;
    } else {
      tb = T * c / g;
      te = T * (c + 1) / g;
      ts = 1;
    }
  }
  __device__ void first(int64_t t, int64_t ts, OzCursor& c) const {
    c.b = 0;
    c.rt = t / pr.nct;
    c.ct = t - c.rt * pr.nct;
    c.step = ts;
  }
  __device__ void next(OzCursor& c) const {
    c.ct += c.step;
    while (c.ct >= pr.nct) {
      c.ct -= pr.nct;
      ++c.rt;
    }
  }
  __device__ const OzProb& prob(int) const { return pr; }
  __device__ const CUtensorMap* tmap(int) const { return map; }
};

// Many independent problems in one launch: the tensor maps and descriptors travel in the
// kernel parameters; the tile prefix over the problems that apply an update this step is
// built in shared memory at kernel start (problems that skip contribute no tiles).
struct OzBatchParams {
  CUtensorMap maps[kOzMaxBatch];
  OzProb probs[kOzMaxBatch];
  const UpdCtl* ctl[kOzMaxBatch];
  int32_t* status[kOzMaxBatch];
  int nprob;
};

struct OzBatchSrc {
  const OzBatchParams* P;
  const int64_t* begin;     // shared memory, nprob + 1 entries
  __device__ int64_t total() const { return begin[P->nprob]; }
  __device__ void range(int64_t c, int64_t g, int64_t& tb, int64_t& te, int64_t& ts) const {
    const int64_t T = total();
    tb = T * c / g;
    te = T * (c + 1) / g;
    ts = 1;
  }
  __device__ void first(int64_t t, int64_t, OzCursor& c) const {
    int lo = 0, hi = P->nprob - 1;       // last b with begin[b] <= t: a problem with tiles
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (begin[mid] <= t) lo = mid; else hi = mid - 1;
    }
    c.b = lo;
    const int64_t u = t - begin[lo];
    c.rt = u / P->probs[lo].nct;
    c.ct = u - c.rt * P->probs[lo].nct;
  }
  __device__ void next(OzCursor& c) const {
    if (++c.ct < P->probs[c.b].nct) return;
    c.ct = 0;
    if (++c.rt < P->probs[c.b].nrt) return;
    c.rt = 0;
    do {
      ++c.b;
    } while (c.b < P->nprob && begin[c.b + 1] == begin[c.b]);     // skip problems without tiles
  }
  __device__ const OzProb& prob(int b) const { return P->probs[b]; }
  __device__ const CUtensorMap* tmap(int b) const { return &P->maps[b]; }
};

__device__ __forceinline__ int64_t oz_key(int b, int64_t rt) { return ((int64_t)b << 40) | rt; }

// Returns true (in every thread) when a wait timed out and the tile loop was abandoned.
template <class Src>
__device__ __forceinline__ bool ozaki_body(const Src& src, uint8_t* smem) {
  OzBars* bars = reinterpret_cast<OzBars*>(smem + kOzBarOff);
  uint8_t* Abuf = smem;                                       // 2 x kOzTileA
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile int* abort = &bars->abort;

  if (warp == kWarpMma) {
    tc::tmem_alloc(&bars->tslot, kOzTmemColsV2);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int q = 0; q < kOzNS; ++q) {
      tc::mbar_init(&bars->full[q], 1);
      tc::mbar_init(&bars->empty[q], 2);
      tc::mbar_init(&bars->ebar[q], kOzEpiThreads);
    }
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&bars->afull[q], 1);
      tc::mbar_init(&bars->aempty[q], 1);
      tc::mbar_init(&bars->tfull[q], 1);
      tc::mbar_init(&bars->tempty[q], kOzEpiThreads / 32);
    }
    bars->abort = 0;
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = bars->tslot;

  int64_t tb, te, ts;
  src.range(blockIdx.x, gridDim.x, tb, te, ts);

  if (warp == kWarpProd) {
    // ------------------------------------------------------------------ producer
    // the digit blocks are re-read by every row tile: evict last, so that the G stream does
    // not push them out of L2
    const uint64_t pol_ops = tc::policy_evict_last();
    int64_t cur = -1;
    int64_t aseq = -1;
    int64_t k = 0;
    OzCursor cs;
    if (tb < te) src.first(tb, ts, cs);
    for (int64_t t = tb; t < te; t += ts, ++k, src.next(cs)) {
      const int b = cs.b;
      const int64_t rt = cs.rt, ct = cs.ct;
      const OzProb& pr = src.prob(b);
      bool ok = true;
      if (oz_key(b, rt) != cur) {
        ++aseq;
        const int ab = (int)(aseq & 1);
        if (lane == 0) {
          if (aseq >= 2) ok = tc::mbar_wait_or_abort(&bars->aempty[ab], (uint32_t)((aseq / 2 - 1) & 1), abort, kOzTimeoutNs);
          if (ok) {
            tc::mbar_arrive_expect_tx(&bars->afull[ab], kOzTileA);
            tc::bulk_g2s_hint(Abuf + ab * kOzTileA, pr.ozA + rt * (int64_t)kOzTileA, kOzTileA, &bars->afull[ab],
                              pol_ops);
          }
        }
        cur = oz_key(b, rt);
      }
      const int s = (int)(k % kOzNS);
      if (lane == 0 && ok && k >= kOzNS)
        ok = tc::mbar_wait_or_abort(&bars->empty[s], (uint32_t)((k / kOzNS - 1) & 1), abort, kOzTimeoutNs);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) break;
      uint8_t* stage = smem + 2 * kOzTileA + s * kOzStage;
      if (lane == 0) {
        // x in doubles (2 per complex entry), y in rows; both boxes are always full-size
        const int x = (int)(ct * kOzN), y = (int)(rt * kOzM);
        const bool second = x + 16 < 2 * pr.n;      // the right box holds at least one column
        const CUtensorMap* map = src.tmap(b);
        tc::mbar_arrive_expect_tx(&bars->full[s], (uint32_t)((second ? kOzGTile : kOzBox) + kOzBBlock));
        tc::tma_load_2d(stage, map, x, y, &bars->full[s]);
        if (second) tc::tma_load_2d(stage + kOzBox, map, x + 16, y, &bars->full[s]);
        tc::bulk_g2s_hint(stage + kOzGTile, pr.ozB + ct * (int64_t)kOzBBlock, kOzBBlock, &bars->full[s], pol_ops);
      }
      __syncwarp();
    }
  } else if (warp == kWarpMma) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_tf32(kOzM, kOzN);
      int64_t cur = -1;
      int64_t aseq = -1;
      int64_t k = 0;
      int ab = 0;
      OzCursor cs;
      if (tb < te) src.first(tb, ts, cs);
      for (int64_t t = tb; t < te; t += ts, ++k, src.next(cs)) {
        const int b = cs.b;
        const int64_t rt = cs.rt;
        if (oz_key(b, rt) != cur) {
          if (cur >= 0) tc::mma_commit(&bars->aempty[ab]);         // old A tile free once its MMAs end
          ++aseq;
          ab = (int)(aseq & 1);
          if (!tc::mbar_wait_or_abort(&bars->afull[ab], (uint32_t)((aseq / 2) & 1), abort, kOzTimeoutNs)) break;
          cur = oz_key(b, rt);
        }
        const int s = (int)(k % kOzNS);
        const int bf = (int)(k & 1);
        if (!tc::mbar_wait_or_abort(&bars->full[s], (uint32_t)((k / kOzNS) & 1), abort, kOzTimeoutNs)) break;
        if (k >= 2 && !tc::mbar_wait_or_abort(&bars->tempty[bf], (uint32_t)((k / 2 - 1) & 1), abort, kOzTimeoutNs)) break;
        tc::fence_after_sync();
        const uint32_t sA = tc::smem_u32(Abuf + ab * kOzTileA);
        const uint32_t sB = tc::smem_u32(smem + 2 * kOzTileA + s * kOzStage + kOzGTile);
        bool first[kOzLv];
#pragma unroll
        for (int L = 0; L < kOzLv; ++L) first[L] = true;
#pragma unroll
        for (int a = 0; a < kOzS; ++a) {
#pragma unroll
          for (int bb = 0; bb < kOzS; ++bb) {
            if (a + bb <= kOzLv - 1) {
              const int L = a + bb;
              tc::mma_tf32(tbase + (uint32_t)(bf * 256 + L * kOzN), tc::smem_desc(sA + a * kOzSliceA, 128, 256),
                           tc::smem_desc(sB + bb * kOzSliceB, 128, 256), idesc, first[L] ? 0u : 1u);
              first[L] = false;
            }
          }
        }
        tc::mma_commit(&bars->tfull[bf]);
        tc::mma_commit(&bars->empty[s]);
      }
    }
    __syncwarp();
  } else if (warp < kEpiWarps) {
    // ------------------------------------------------------------------ epilogue
    const int q = warp & 3, h = warp >> 2;     // TMEM lane quarter, column quarter
    const int r = q * 32 + lane;               // tile row
    const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
    int64_t cur = -1;
    int Ei = 0;
    int64_t k = 0;
    OzCursor cs;
    if (tb < te) src.first(tb, ts, cs);
    for (int64_t t = tb; t < te; t += ts, ++k, src.next(cs)) {
      const int b = cs.b;
      const int64_t rt = cs.rt, ct = cs.ct;
      const OzProb& pr = src.prob(b);
      if (oz_key(b, rt) != cur) {
        Ei = pr.ozE[rt * kOzM + r];
        cur = oz_key(b, rt);
      }
      const int s = (int)(k % kOzNS);
      const int bf = (int)(k & 1);
      if (!tc::mbar_wait_or_abort(&bars->tfull[bf], (uint32_t)((k / 2) & 1), abort, kOzTimeoutNs)) break;
      if (!tc::mbar_wait_or_abort(&bars->full[s], (uint32_t)((k / kOzNS) & 1), abort, kOzTimeoutNs)) break;
      tc::fence_after_sync();
      float acc[kOzLv][8];
#pragma unroll
      for (int L = 0; L < kOzLv; ++L)
        tc::tmem_ld8(tbase + lane_addr + (uint32_t)(bf * 256 + L * kOzN + h * 8), acc[L]);
      tc::tmem_ld_wait();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars->tempty[bf]);
      uint8_t* stage = smem + 2 * kOzTileA + s * kOzStage;
      const int32_t* Fj = reinterpret_cast<const int32_t*>(stage + kOzGTile + kOzTileB);
      // complex column jj of row r: box jj/8, 16-byte chunk (jj%8) XOR (r%8) (128B swizzle)
      uint8_t* rowbase = stage + r * 128;
      const int64_t i = rt * kOzM + r;
      const int64_t j0 = ct * (kOzN / 2);
#pragma unroll
      for (int c = 0; c < kOzColsPerThread; ++c) {
        const int jj = h * kOzColsPerThread + c;
        if (i < pr.n && j0 + jj < pr.n) {
          float lr[kOzLv], li[kOzLv];
#pragma unroll
          for (int L = 0; L < kOzLv; ++L) {
            lr[L] = acc[L][2 * c];
            li[L] = acc[L][2 * c + 1];
          }
          const int u = Ei + Fj[jj] - 59;
          double2* gp = reinterpret_cast<double2*>(rowbase + (jj >> 3) * kOzBox + (((jj & 7) ^ (r & 7)) << 4));
          const double2 g = *gp;
          *gp = make_double2(g.x + oz_to_double(oz_combine(lr), u), g.y + oz_to_double(oz_combine(li), u));
        }
      }
      tc::fence_proxy_async_smem();
      tc::mbar_arrive(&bars->ebar[s]);
    }
  }
  if (warp == kWarpStore) {
    // ------------------------------------------------------------------ storer
    int64_t k = 0;
    OzCursor cs;
    if (tb < te) src.first(tb, ts, cs);
    for (int64_t t = tb; t < te; t += ts, ++k, src.next(cs)) {
      const int b = cs.b;
      const int64_t rt = cs.rt, ct = cs.ct;
      const int s = (int)(k % kOzNS);
      bool ok = true;
      if (lane == 0) ok = tc::mbar_wait_or_abort(&bars->ebar[s], (uint32_t)((k / kOzNS) & 1), abort, kOzTimeoutNs);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) break;
      uint8_t* stage = smem + 2 * kOzTileA + s * kOzStage;
      if (lane == 0) {
        const int x = (int)(ct * kOzN), y = (int)(rt * kOzM);
        const CUtensorMap* map = src.tmap(b);
        tc::tma_store_2d(map, x, y, stage);
        if (x + 16 < 2 * src.prob(b).n) tc::tma_store_2d(map, x + 16, y, stage + kOzBox);
      }
      tc::bulk_commit();
      tc::bulk_wait_read0();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars->empty[s]);
    }
    tc::bulk_wait0();
  }
  tc::fence_before_sync();
  __syncthreads();
  const bool aborted = bars->abort != 0;
  tc::fence_after_sync();
  if (warp == kWarpMma) tc::tmem_dealloc(tbase, kOzTmemColsV2);
  return aborted;
}

__global__ void __launch_bounds__(kOzThreadsV2, 1)
k_rank_update_ozaki(const __grid_constant__ CUtensorMap tmapG, int64_t n, int64_t nrt, int64_t nct,
                    const uint8_t* __restrict__ ozA, const int32_t* __restrict__ ozE,
                    const uint8_t* __restrict__ ozB, const UpdCtl* __restrict__ ctl,
                    int32_t* __restrict__ status, int32_t* __restrict__ prof_p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int p = ctl->skip ? 0 : ctl->nv;
  if (prof_p && blockIdx.x == 0 && threadIdx.x == 0 && p >= 1 && p <= 4) *prof_p = p;
  if (p < 1 || p > 4) return;
  OzSingleSrc src;
  src.map = &tmapG;
  src.pr = OzProb{n, nrt, nct, ozA, ozE, ozB};
  if (ozaki_body(src, smem) && threadIdx.x == 0) atomicExch(status, GF_ETIMEOUT);
}

// Batched form: the tiles of every problem that applies a rank-1..4 update this step, one
// persistent launch.  On a timeout every problem's status word receives GF_ETIMEOUT.  The tile
// prefix lives behind the barriers in dynamic shared memory (no static shared memory, so the
// 1024-byte alignment of the swizzled stages holds).
constexpr int kOzSmemBatch = kOzSmemV2 + 8 * (kOzMaxBatch + 1);
__global__ void __launch_bounds__(kOzThreadsV2, 1)
k_rank_update_ozaki_batch(const __grid_constant__ OzBatchParams P) {
  extern __shared__ __align__(1024) uint8_t smem[];
  int64_t* s_begin = reinterpret_cast<int64_t*>(smem + kOzSmemV2);
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int b = 0; b < P.nprob; ++b) {
      s_begin[b] = acc;
      const UpdCtl* c = P.ctl[b];
      const int p = c->skip ? 0 : c->nv;
      if (p >= 1 && p <= 4) acc += P.probs[b].nrt * P.probs[b].nct;
    }
    s_begin[P.nprob] = acc;
  }
  __syncthreads();
  if (s_begin[P.nprob] == 0) return;
  OzBatchSrc src;
  src.P = &P;
  src.begin = s_begin;
  if (ozaki_body(src, smem) && threadIdx.x == 0)
    for (int b = 0; b < P.nprob; ++b) atomicExch(P.status[b], GF_ETIMEOUT);
}

OzLayout oz_layout(int64_t n) {
  OzLayout o;
  o.nrow_tiles = (n + kOzM - 1) / kOzM;
  o.ncol_tiles = (2 * n + kOzN - 1) / kOzN;
  o.bytesA = (size_t)o.nrow_tiles * kOzTileA;
  o.bytesE = (size_t)o.nrow_tiles * kOzM * 4;
  o.bytesB = (size_t)o.ncol_tiles * kOzBBlockG;
  o.bytesF = 0;
  return o;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// G as a 2-D tensor of doubles: 2n columns (re, im interleaved) by n rows, row stride 16 ldg
// bytes; boxes of 16 doubles (128 B) x 128 rows with 128-byte swizzle.
// complex128 G as a 2-D tensor of doubles: 2n columns by `rows` rows (n, or a row block)
static bool make_tmap_G(CUtensorMap* m, double2* G, int64_t ldg, int64_t n, int64_t rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)(2 * n), (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(16 * ldg)};
  cuuint32_t box[2] = {16, (cuuint32_t)kOzM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void*)G, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool launch_rank_update_ozaki(double2* G, int64_t ldg, int64_t n, int64_t grows, int pmax, const cplx* C0,
                              const cplx* S, const UpdCtl* ctl, uint8_t* ozA, int32_t* ozE,
                              uint8_t* ozB, int32_t* ozF, int32_t* status, int32_t* prof_p,
                              int sm_count, cudaStream_t st) {
  (void)ozF;
  CUtensorMap tmap;
  if (!make_tmap_G(&tmap, G, ldg, n, grows)) return false;
  const OzLayout o = oz_layout(n);
  const int64_t nrt = (grows + kOzM - 1) / kOzM;          // row tiles of the rows held
  {
    int64_t rows = nrt * kOzM;
    int64_t b = (rows + 127) / 128;
    k_oz_prep_rows<<<(int)(b < 4864 ? b : 4864), 128, 0, st>>>(C0, pmax, grows, rows, ctl, ozA, ozE);
    int64_t cols = o.ncol_tiles * (kOzN / 2);
    b = (cols + 127) / 128;
    k_oz_prep_cols<<<(int)(b < 4864 ? b : 4864), 128, 0, st>>>(S, n, cols, ctl, ozB);
  }
  {  // once per device
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || !done[dev]) {
      cudaFuncSetAttribute(k_rank_update_ozaki, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmemV2);
      if (dev >= 0 && dev < 64) done[dev] = true;
    }
  }
  const int64_t tiles = nrt * o.ncol_tiles;
  const int grid = (int)(tiles < sm_count ? tiles : sm_count);
  k_rank_update_ozaki<<<grid, kOzThreadsV2, kOzSmemV2, st>>>(tmap, n, nrt, o.ncol_tiles, ozA, ozE, ozB,
                                                            ctl, status, prof_p);
  return true;
}

size_t ozaki_batch_params_bytes() { return sizeof(OzBatchParams); }

// Host: the parameter block of the batched update (one tensor map and descriptor per problem,
// pointing at the problem's G and at the digit buffers in its workspace).
bool ozaki_batch_params(void* out, const BatchItem* it, int nprob) {
  if (nprob < 1 || nprob > kOzMaxBatch) return false;
  OzBatchParams* P = new (out) OzBatchParams();
  P->nprob = nprob;
  for (int b = 0; b < nprob; ++b) {
    const int64_t n = it[b].L.n;
    if (!make_tmap_G(&P->maps[b], reinterpret_cast<double2*>(it[b].G), it[b].ldg, n, n)) return false;
    const OzLayout o = oz_layout(n);
    P->probs[b] = OzProb{n, o.nrow_tiles, o.ncol_tiles, reinterpret_cast<const uint8_t*>(it[b].ws + it[b].L.ozA),
                         reinterpret_cast<const int32_t*>(it[b].ws + it[b].L.ozE),
                         reinterpret_cast<const uint8_t*>(it[b].ws + it[b].L.ozB)};
    P->ctl[b] = reinterpret_cast<const UpdCtl*>(it[b].ws + it[b].L.ctl);
    P->status[b] = it[b].status;
  }
  return true;
}

void launch_oz_prep_batch(const BatchItem* items, int nprob, int64_t widest, cudaStream_t st) {
  int64_t b = (widest + 127) / 128;           // widest: rows (= complex columns) of the largest G
  if (b > 608) b = 608;
  k_oz_prep_batch<<<dim3((unsigned)(b < 1 ? 1 : b), (unsigned)nprob), 128, 0, st>>>(items);
}

void launch_rank_update_ozaki_batch(const void* params, int ctas, cudaStream_t st) {
  {  // once per device
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || !done[dev]) {
      cudaFuncSetAttribute(k_rank_update_ozaki_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmemBatch);
      if (dev >= 0 && dev < 64) done[dev] = true;
    }
  }
  k_rank_update_ozaki_batch<<<ctas, kOzThreadsV2, kOzSmemBatch, st>>>(*reinterpret_cast<const OzBatchParams*>(params));
}

}  // namespace gf
