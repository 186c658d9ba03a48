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

#include "gf_internal.cuh"
#include "gf_tc.cuh"

namespace gf {

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
constexpr int kOzTmemCols = 256;                // >= kOzLv * kOzN, power of two
constexpr int kOzThreads = 128;
constexpr int kOzSmem = 100 * 1024;             // dynamic smem request (limits to 2 CTAs/SM: TMEM)
constexpr uint64_t kOzTimeoutNs = 2000000000ull;

// byte offset of element (r, k) inside one K-major, no-swizzle digit slice (8x16-byte core
// matrices; K-direction core-matrix stride 128 B, row-group stride 256 B)
__host__ __device__ __forceinline__ int oz_off(int r, int k) {
  return (r >> 3) * 256 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

// six signed 9-bit digits of x in (-1, 1): x = sum_a d[a] 2^(-9(a+1)) + r, |r| <= 2^-55
__device__ __forceinline__ void oz_digits(double x, float (&d)[kOzS]) {
  double r = x;
#pragma unroll
  for (int a = 0; a < kOzS; ++a) {
    const double sc = ldexp(1.0, kOzW * (a + 1));
    double t = rint(r * sc);
    d[a] = (float)t;
    r = r - t * ldexp(1.0, -kOzW * (a + 1));
  }
}

__device__ __forceinline__ int oz_exponent(double m) {
  // smallest E with m < 2^E (m > 0); a zero row/column gets digits 0 and any exponent
  return m > 0.0 ? ilogb(m) + 1 : 0;
}

// ---- operand preparation (once per step, O(n p) work) --------------------------------------
__global__ void k_oz_prep_rows(const cplx* __restrict__ C0, int pmax, int64_t n, int64_t nrows_pad,
                               const UpdCtl* __restrict__ ctl, uint8_t* __restrict__ ozA,
                               int32_t* __restrict__ ozE) {
  if (ctl->skip || ctl->nv > 4) return;
  const int p = ctl->nv;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v[kOzK];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      cplx c = (i < n && k < p) ? C0[i * pmax + k] : mk(0.0, 0.0);
      v[k] = c.re;
      v[4 + k] = c.im;
    }
    double m = 0.0;
#pragma unroll
    for (int k = 0; k < kOzK; ++k) m = fmax(m, fabs(v[k]));
    const int E = oz_exponent(m);
    ozE[i] = E;
    uint8_t* tile = ozA + (i / kOzM) * (int64_t)kOzTileA;
    const int r = (int)(i % kOzM);
    float dg[kOzK][kOzS];
#pragma unroll
    for (int k = 0; k < kOzK; ++k) oz_digits(ldexp(v[k], -E), dg[k]);
#pragma unroll
    for (int a = 0; a < kOzS; ++a) {
      float4* q0 = reinterpret_cast<float4*>(tile + a * kOzSliceA + oz_off(r, 0));
      float4* q1 = reinterpret_cast<float4*>(tile + a * kOzSliceA + oz_off(r, 4));
      *q0 = make_float4(dg[0][a], dg[1][a], dg[2][a], dg[3][a]);
      *q1 = make_float4(dg[4][a], dg[5][a], dg[6][a], dg[7][a]);
    }
  }
}

__global__ void k_oz_prep_cols(const cplx* __restrict__ S, int64_t n, int64_t ncols_pad,
                               const UpdCtl* __restrict__ ctl, uint8_t* __restrict__ ozB,
                               int32_t* __restrict__ ozF) {
  if (ctl->skip || ctl->nv > 4) return;
  const int p = ctl->nv;
  // one thread per complex column j; writes real columns 2j and 2j+1
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ncols_pad;
       j += (int64_t)gridDim.x * blockDim.x) {
    double sr[4], si[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      cplx s = (j < n && k < p) ? S[(int64_t)k * n + j] : mk(0.0, 0.0);
      sr[k] = s.re;
      si[k] = s.im;
    }
    double m = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) m = fmax(m, fmax(fabs(sr[k]), fabs(si[k])));
    const int F = oz_exponent(m);
    ozF[j] = F;
    float dr[4][kOzS], di[4][kOzS];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      oz_digits(ldexp(sr[k], -F), dr[k]);
      oz_digits(ldexp(si[k], -F), di[k]);
    }
    const int64_t c_re = 2 * j;
    uint8_t* tile = ozB + (c_re / kOzN) * (int64_t)kOzTileB;
    const int c = (int)(c_re % kOzN);            // even; c + 1 is the imaginary column
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

// ---- epilogue arithmetic --------------------------------------------------------------------
// exact FP32 integer (|x| <= 2^22) -> int32
__device__ __forceinline__ int32_t oz_f2i(float x) {
  return (int32_t)__float_as_uint(x + 12582912.0f) - 0x4B400000;
}

// sum_L acc_L 2^(-9 (L+2)) in units of 2^-59 (levels 2..7)
__device__ __forceinline__ long long oz_combine(const float (&acc)[kOzLv]) {
  long long D = oz_f2i(acc[0]);
#pragma unroll
  for (int L = 1; L < kOzLv - 1; ++L) D = D * 512 + oz_f2i(acc[L]);
  return D * 32 + ((oz_f2i(acc[kOzLv - 1]) + 8) >> 4);
}

// D * 2^u as a double, built with integer operations (|D| < 2^62)
__device__ __forceinline__ double oz_to_double(long long D, int u) {
  if (D == 0) return 0.0;
  const unsigned long long sign = D < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long M = D < 0 ? (unsigned long long)(-D) : (unsigned long long)D;
  const int lz = __clzll(M);
  M <<= lz;                                        // leading one at bit 63
  const unsigned long long mant = (M >> 11) + ((M >> 10) & 1ull);   // 53 bits, rounded
  const long long e = 63 - lz + u;                 // exponent of the leading one
  const unsigned long long bits = ((unsigned long long)(e + 1022) << 52) + mant;
  return __longlong_as_double((long long)(bits | sign));
}

// ---- the update kernel ----------------------------------------------------------------------
// grid.x: 128-row tiles; grid.y: column chunks.  One CTA = 4 warps; thread t owns tile row t
// (= TMEM lane t).  Thread 0 issues the MMAs.
__global__ void __launch_bounds__(kOzThreads, 1)
k_rank_update_ozaki(double2* __restrict__ G, int64_t ldg, int64_t n, int64_t ncol_tiles,
                    const uint8_t* __restrict__ ozA, const int32_t* __restrict__ ozE,
                    const uint8_t* __restrict__ ozB, const int32_t* __restrict__ ozF,
                    const UpdCtl* __restrict__ ctl, int32_t* __restrict__ status,
                    int32_t* __restrict__ prof_p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int p = ctl->skip ? 0 : ctl->nv;
  if (prof_p && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *prof_p = (p >= 1 && p <= 4) ? p : 0;
  if (p < 1 || p > 4) return;

  uint8_t* As = smem;                              // kOzTileA
  uint8_t* Bs = smem + kOzTileA;                   // kOzTileB
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kOzTileA + kOzTileB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kOzTileA + kOzTileB + 8);
  const int t = threadIdx.x, warp = t >> 5;
  const int64_t rt = blockIdx.x;
  const int64_t i = rt * kOzM + t;

  if (warp == 0) {
    tc::tmem_alloc(tslot, kOzTmemCols);
    tc::tmem_relinquish();
  }
  if (t == 0) {
    tc::mbar_init(mbar, 1);
    tc::fence_mbar_init();
  }
  {  // A digit slices of this row tile -> smem
    const uint4* src = reinterpret_cast<const uint4*>(ozA + rt * (int64_t)kOzTileA);
    uint4* dst = reinterpret_cast<uint4*>(As);
    for (int q = t; q < kOzTileA / 16; q += kOzThreads) dst[q] = src[q];
  }
  const int Ei = ozE[rt * kOzM + t];
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t idesc = tc::idesc_tf32(kOzM, kOzN);
  const uint32_t sA = tc::smem_u32(As), sB = tc::smem_u32(Bs);

  // column tiles of this chunk
  const int64_t per = (ncol_tiles + gridDim.y - 1) / gridDim.y;
  const int64_t ct0 = blockIdx.y * per;
  const int64_t ct1 = ct0 + per < ncol_tiles ? ct0 + per : ncol_tiles;
  uint32_t phase = 0;
  bool failed = false;
  for (int64_t ct = ct0; ct < ct1; ++ct) {
    {  // B digit slices of this column tile -> smem
      const uint4* src = reinterpret_cast<const uint4*>(ozB + ct * (int64_t)kOzTileB);
      uint4* dst = reinterpret_cast<uint4*>(Bs);
      for (int q = t; q < kOzTileB / 16; q += kOzThreads) dst[q] = src[q];
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
      int first[kOzLv];
#pragma unroll
      for (int L = 0; L < kOzLv; ++L) first[L] = 1;
#pragma unroll
      for (int a = 0; a < kOzS; ++a) {
#pragma unroll
        for (int b = 0; b < kOzS; ++b) {
          if (a + b <= kOzLv - 1) {
            const int L = a + b;
            const uint64_t da = tc::smem_desc(sA + a * kOzSliceA, 128, 256);
            const uint64_t db = tc::smem_desc(sB + b * kOzSliceB, 128, 256);
            tc::mma_tf32(tbase + (uint32_t)(L * kOzN), da, db, idesc, first[L] ? 0u : 1u);
            first[L] = 0;
          }
        }
      }
      tc::mma_commit(mbar);
    }
    // prefetch this thread's G row segment while the MMAs run
    const int64_t j0 = ct * (kOzN / 2);
    double2 g[kOzN / 2];
    const bool row_ok = i < n;
#pragma unroll
    for (int q = 0; q < kOzN / 2; ++q) {
      const int64_t j = j0 + q;
      g[q] = (row_ok && j < n) ? G[i * ldg + j] : make_double2(0.0, 0.0);
    }
    const bool ok = tc::mbar_wait_bounded(mbar, phase, kOzTimeoutNs);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
#pragma unroll
    for (int cg = 0; cg < kOzN / 8; ++cg) {
      float acc[kOzLv][8];
#pragma unroll
      for (int L = 0; L < kOzLv; ++L)
        tc::tmem_ld8(tbase + lane_base + (uint32_t)(L * kOzN + cg * 8), acc[L]);
      tc::tmem_ld_wait();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int qq = cg * 4 + q;
        const int64_t j = j0 + qq;
        if (!row_ok || j >= n) continue;
        float lr[kOzLv], li[kOzLv];
#pragma unroll
        for (int L = 0; L < kOzLv; ++L) {
          lr[L] = acc[L][2 * q];
          li[L] = acc[L][2 * q + 1];
        }
        const int u = Ei + ozF[j] - 59;
        const double dre = oz_to_double(oz_combine(lr), u);
        const double dim = oz_to_double(oz_combine(li), u);
        G[i * ldg + j] = make_double2(g[qq].x + dre, g[qq].y + dim);
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  if (failed) {
    if (t == 0) atomicExch(status, GF_ETIMEOUT);
    // wait (bounded) for the MMAs of the failed tile before giving the TMEM back
    tc::mbar_wait_bounded(mbar, phase ^ 1u, kOzTimeoutNs);
  }
  tc::fence_after_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, kOzTmemCols);
}

OzLayout oz_layout(int64_t n) {
  OzLayout o;
  o.nrow_tiles = (n + kOzM - 1) / kOzM;
  o.ncol_tiles = (2 * n + kOzN - 1) / kOzN;
  o.bytesA = (size_t)o.nrow_tiles * kOzTileA;
  o.bytesE = (size_t)o.nrow_tiles * kOzM * 4;
  o.bytesB = (size_t)o.ncol_tiles * kOzTileB;
  o.bytesF = (size_t)o.ncol_tiles * (kOzN / 2) * 4;
  return o;
}

void launch_rank_update_ozaki(double2* G, int64_t ldg, int64_t n, int pmax, const cplx* C0,
                              const cplx* S, const UpdCtl* ctl, uint8_t* ozA, int32_t* ozE,
                              uint8_t* ozB, int32_t* ozF, int32_t* status, int32_t* prof_p,
                              int sm_count, cudaStream_t st) {
  const OzLayout o = oz_layout(n);
  {
    int64_t rows = o.nrow_tiles * kOzM;
    int64_t b = (rows + 127) / 128;
    k_oz_prep_rows<<<(int)(b < 4864 ? b : 4864), 128, 0, st>>>(C0, pmax, n, rows, ctl, ozA, ozE);
    int64_t cols = o.ncol_tiles * (kOzN / 2);
    b = (cols + 127) / 128;
    k_oz_prep_cols<<<(int)(b < 4864 ? b : 4864), 128, 0, st>>>(S, n, cols, ctl, ozB, ozF);
  }
  cudaFuncSetAttribute(k_rank_update_ozaki, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
  // about 4 waves of 2 CTAs per SM
  int64_t target = (int64_t)sm_count * 2 * 4;
  int64_t chunks = (target + o.nrow_tiles - 1) / o.nrow_tiles;
  if (chunks < 1) chunks = 1;
  if (chunks > o.ncol_tiles) chunks = o.ncol_tiles;
  if (chunks > 65535) chunks = 65535;
  dim3 grid((unsigned)o.nrow_tiles, (unsigned)chunks);
  k_rank_update_ozaki<<<grid, kOzThreads, kOzSmem, st>>>(G, ldg, n, o.ncol_tiles, ozA, ozE, ozB, ozF,
                                                         ctl, status, prof_p);
}

}  // namespace gf
