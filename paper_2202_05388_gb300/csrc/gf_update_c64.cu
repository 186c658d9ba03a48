// Mixed-precision rank-k p update of a complex64 G (the Woodbury form of Eqs. 10 and 14 for a
// set V of up to 4k pixels accepted together):
//
//   G <- G + C0 S,   C0 = G[:, V],   S = D A^{-1} G[V, :],   A = I - G_VV D.
//
// The p x p capacitance matrix A is factorised in FP64 (k_capacitance); its inverse is formed
// here by p parallel FP64 column solves and scaled by D.  S is an FP32 GEMM of that p x p
// matrix with the p rows G[V, :].  The n x n update runs on the tensor cores as one real GEMM
// in the 4M form (K = 2P, P = p rounded up to 16).  Each row of A' (each column of B') is
// scaled by a power of two into (-2^14, 2^14), x' = 2^(14 - E_i) x (2^(14 - F_j) x), and split
// into two FP16 values, x' = hi + lo with hi = fp16(x') and lo = fp16(x' - hi).  Three products
// per K step, hi*hi + hi*lo + lo*hi, accumulate into one FP32 TMEM accumulator (the dropped
// lo*lo term and the rounding of lo are below 2^-22 of |x'|max |y'|max per product), and the
// epilogue adds 2^(E_i + F_j - 28) times the accumulator to G.  FP16 values cost 2 bytes each
// and run at the FP16 tensor rate.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "gf_internal.cuh"
#include "gf_ra_sched.h"
#include "gf_tc.cuh"

namespace gf {

constexpr int kC64M = 128;                     // rows per tile
constexpr int kC64N = 128;                     // real columns per resident-A tile (64 complex)
constexpr int kC64WN = 256;                    // real columns per streaming tile (128 complex)
constexpr int kC64KC = 16;                     // K per operand chunk
constexpr int kC64Half = kC64M * kC64KC * 2;   // hi (or lo) of a 128-row chunk: 4 KB
constexpr int kC64Block = 2 * kC64Half;        // hi + lo of a 128-row chunk: 8 KB
constexpr int kC64PairBlock = 2 * kC64Block;   // B chunk of a column-tile pair: 16 KB
constexpr int kC64Box = kC64M * 128;           // TMA box: 128 rows x 128 B (16 complex64)
constexpr int kC64GStage = 2 * kC64Box;        // one G stage (two boxes): 32 KB
constexpr int kC64NSG = 4;                     // G stages
constexpr int kC64Ops = 96 * 1024;             // operand area (both forms)
constexpr int kC64BarOff = kC64Ops + kC64NSG * kC64GStage;   // 229376
constexpr int kC64Smem = kC64BarOff + 512;
constexpr int kC64EpiWarps = 16;
constexpr int kC64Threads = 32 * (kC64EpiWarps + 4);   // + G producer, MMA, storer, operand producer
constexpr uint64_t kC64TimeoutNs = 2000000000ull;
constexpr uint64_t kC64DrainNs = 100000000ull;
// streaming raster: groups of 96 row tiles.  The 152 CTAs work on neighbouring tiles of one or
// two column pairs; a group's A chunks (96 x 128 KB at K = 256) stay in L2 and every B chunk is
// fetched from DRAM once per group.  Measured at 320x320, K = 256, ms per update: groups of 8
// 39.7 (B fetched 100 times per launch), 16 37.2, 24 35.9, 32 35.6, 48 33.5, 64 33.0-33.5,
// 96 32.0-32.5, 128 39.5-41.2, 256 40.4-41.2 (every CTA on the same B chunks at once); an L2
// prefetch of the next tile's chunks made every size slower (41-44).
constexpr int kC64Group = 96;
static_assert(kC64Group >= 1, "raster groups hold at least one row tile");
constexpr int kC64Exp = 14;                    // scaled operands lie in (-2^14, 2^14)
constexpr int kC64MinExp = -40;                // smallest scale exponent (keeps 2^(E+F-28) normal)

// byte offset of element (r, k) in the hi (or lo) part of a 128-row x 16-deep FP16 chunk,
// K-major without swizzle: 8-row x 16-byte core matrices, K neighbour at +128 B (LBO), next
// 8-row group at +256 B (SBO); two 128-row parts placed back to back form one 256-row operand
// with the same strides.
__host__ __device__ __forceinline__ int c64_off(int r, int k) {
  return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
constexpr uint32_t kC64Lbo = 128, kC64Sbo = 256;

// x' in (-2^14, 2^14) -> hi + lo, both FP16 (x' - hi is exact in FP32)
__device__ __forceinline__ void f16_split(float x, __half& hi, __half& lo) {
  hi = __float2half_rn(x);
  lo = __float2half_rn(x - __half2float(hi));
}

// E with |x| < 2^E for every x of a row (column) whose largest magnitude is m
__device__ __forceinline__ int scale_exp(float m) {
  const int e = m > 0.f ? ilogbf(m) + 1 : 0;
  return e < kC64MinExp ? kC64MinExp : e;
}

__device__ __forceinline__ void st4h(uint8_t* p, __half a, __half b, __half c, __half d) {
  __half2 x = __halves2half2(a, b), y = __halves2half2(c, d);
  uint2 v;
  v.x = *reinterpret_cast<uint32_t*>(&x);
  v.y = *reinterpret_cast<uint32_t*>(&y);
  *reinterpret_cast<uint2*>(p) = v;
}

// P = p rounded up to 16, so that each of the four u-quarters of k_c64_s_gemm is a multiple
// of 4 and every K chunk holds whole groups of four.
__host__ __device__ int64_t c64_padP(int p) { return (int64_t)((p + 15) / 16) * 16; }

// Operand blocks: A chunk of row tile rt at Aops + (rt nkc + kc) 8 KB = [hi | lo]; B chunk of
// column-tile pair cp at Bops + (cp nkc + kc) 16 KB = [hi(2cp) | hi(2cp+1) | lo(2cp) | lo(2cp+1)],
// so a 256-column streaming tile takes one 16 KB copy per chunk and a 128-column tile two 4 KB
// copies.  Erow: one exponent per row (nrt 128); Fcol: one per complex column (ncp 128).
C64Layout c64_layout(int64_t n, int pmax) {
  C64Layout o;
  o.P = c64_padP(pmax);
  o.K = 2 * o.P;
  o.nkc = o.K / kC64KC;
  o.nrt = (n + kC64M - 1) / kC64M;
  o.nct = (2 * n + kC64N - 1) / kC64N;
  o.ncp = (o.nct + 1) / 2;
  o.bytesA = (size_t)o.nrt * o.nkc * kC64Block;
  o.bytesB = (size_t)o.ncp * o.nkc * kC64PairBlock;
  o.bytesM = (size_t)pmax * pmax * 8;
  o.bytesE = (size_t)o.nrt * kC64M * 4;
  o.bytesF = (size_t)o.ncp * (kC64WN / 2) * 4;
  return o;
}

// ---- D A^{-1} (p x p, FP32) from the FP64 LU: one CTA per column, a thread per row ----------
// The unit vector e_c under the row interchanges in order is e_pos (only the unit's position is
// followed), so the unit-lower solve starts at column pos; the factor columns are staged 16 at a
// time in shared memory (each step would otherwise wait on an L2 load), and the upper solve's
// pivot reciprocals 1 / |u_qq|^2 are formed first, side by side (cdiv_r with them gives cdiv's
// bits), so that a step is one barrier and one dependent complex update per row.
constexpr int kInvCols = 16;
__global__ void __launch_bounds__(128) k_c64_inverse(WsLayout L, char* ws, int lam, float2* __restrict__ Mout) {
  const UpdCtl* ctl = reinterpret_cast<const UpdCtl*>(ws + L.ctl);
  if (ctl->skip) return;
  const int p = ctl->nv;
  const int c = blockIdx.x;
  if (c >= p || p > (int)blockDim.x) return;
  const cplx* A = reinterpret_cast<const cplx*>(ws + L.lu + lam * L.lu_s);
  const int32_t* piv = reinterpret_cast<const int32_t*>(ws + L.piv + lam * L.piv_s);
  const double* dchi = reinterpret_cast<const double*>(ws + L.dchi);
  __shared__ cplx x[kC64MaxP], xs[kC64MaxP];
  __shared__ cplx blk[kInvCols][kC64MaxP];
  __shared__ double dinv[kC64MaxP];
  __shared__ int s_pos;
  const int t = threadIdx.x;
  if (t < p) dinv[t] = 1.0 / abs2(A[t * p + t]);
  if (t == 0) {
    int pos = c;
    for (int q = 0; q < p; ++q) {
      const int r = piv[q];
      if (pos == q) pos = r;
      else if (pos == r) pos = q;
    }
    s_pos = pos;
  }
  __syncthreads();
  const int pos = s_pos;
  if (t < p) x[t] = mk(t == pos ? 1.0 : 0.0, 0.0);
  // unit lower, columns pos .. p - 1
  for (int q0 = pos - pos % kInvCols; q0 < p; q0 += kInvCols) {
    __syncthreads();                                      // the previous block's readers are done
    for (int e = t; e < kInvCols * p; e += blockDim.x) {
      const int qq = e / p, r = e - qq * p;
      if (q0 + qq < p) blk[qq][r] = A[r * p + q0 + qq];
    }
    __syncthreads();
    for (int qq = 0; qq < kInvCols; ++qq) {
      const int q = q0 + qq;
      if (q >= p) break;
      if (q < pos) continue;
      const cplx xq = x[q];
      if (t > q && t < p) x[t] = x[t] - blk[qq][t] * xq;
      __syncthreads();
    }
  }
  // upper, from the bottom; the solved entries go to xs, so that no thread reads an entry that
  // another is overwriting
  for (int q0 = ((p - 1) / kInvCols) * kInvCols; q0 >= 0; q0 -= kInvCols) {
    __syncthreads();
    for (int e = t; e < kInvCols * p; e += blockDim.x) {
      const int qq = e / p, r = e - qq * p;
      if (q0 + qq < p) blk[qq][r] = A[r * p + q0 + qq];
    }
    __syncthreads();
    for (int qq = kInvCols - 1; qq >= 0; --qq) {
      const int q = q0 + qq;
      if (q >= p) continue;
      const cplx xq = cdiv_r(x[q], blk[qq][q], dinv[q]);
      if (t == q) xs[q] = xq;
      if (t < q) x[t] = x[t] - blk[qq][t] * xq;
      __syncthreads();
    }
  }
  // column c of A^{-1}; row u scaled by d_chi[u]
  if (t < p) Mout[t * p + c] = make_float2((float)(dchi[t] * xs[t].re), (float)(dchi[t] * xs[t].im));
}

// ---- S = (D A^{-1}) G[V, :] in FP32, written as scaled split-FP16 B operand blocks ----------
// One CTA per 64 complex columns (one 128-real-column tile, both tiles of the last pair are
// written); thread (u group ug, column group cg): u = 4 ug .. 4 ug + 3 and columns cg + 8 b
// (b < 8), so that per v 12 shared-memory loads (4 of M, 8 of the rows) feed 32 complex FMAs,
// the eight column groups of a warp reading 64 contiguous bytes and the M rows padded to 17
// entries (no bank conflicts).  Chunks of 16 v of M and of the rows are double-buffered in
// shared memory by asynchronous copies (chunk i + 1 arrives while chunk i is summed); the sum
// over v runs in the same order for every entry.
// Row v of the update set is read at R + rowof(v) ldr: from G (rowof = V[v]) or from a panel of the
// set's rows (V == nullptr, rowof = v).
constexpr int kSgMs = 128 * 17, kSgRs = 16 * 64;           // float2 entries per buffer
constexpr size_t kSgSmem = 2 * (kSgMs + kSgRs) * sizeof(float2);
__device__ __forceinline__ void sg_copy8(void* dst, const void* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const int n = valid ? 8 : 0;                              // 0: zero-fill, nothing is read
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__global__ void __launch_bounds__(256) k_c64_s_gemm(const float2* __restrict__ R, int64_t ldr, int64_t n,
                                                    const float2* __restrict__ Mdai, const int32_t* __restrict__ V,
                                                    const UpdCtl* __restrict__ ctl, int nkc,
                                                    uint8_t* __restrict__ Bops, int32_t* __restrict__ Fcol) {
  if (ctl->skip) return;
  const int p = ctl->nv;
  const int P = (int)c64_padP(p);            // this step's P: the blocks beyond K = 2P are not read
  extern __shared__ __align__(16) float2 sg_smem[];
  __shared__ float smax[32][65];
  __shared__ int64_t rowof[kC64MaxP];
  const int t = threadIdx.x;
  const int cg = t & 7, ug = t >> 3;         // columns cg + 8 b, u = 4 ug .. 4 ug + 3
  const int64_t ct = blockIdx.x;
  const int64_t j0 = ct * 64;
  const bool act = 4 * ug < P;
  for (int v = t; v < p; v += blockDim.x) rowof[v] = (int64_t)(V ? V[v] : v) * ldr;
  __syncthreads();
  // the copies of chunk v0 into buffer bf: M[u][v0 .. v0+16) (rows padded to 17), the rows' 64 columns
  auto stage = [&](int v0, int bf) {
    float2* Ms = sg_smem + bf * (kSgMs + kSgRs);
    float2* Rs = Ms + kSgMs;
    for (int e = t; e < 128 * 16; e += 256) {
      const int u = e >> 4, v = v0 + (e & 15);
      const bool ok = u < p && v < p;
      sg_copy8(Ms + u * 17 + (e & 15), ok ? (const void*)(Mdai + u * p + v) : (const void*)Mdai, ok);
    }
    for (int e = t; e < 16 * 64; e += 256) {
      const int vv = e >> 6, jl = e & 63;
      const int64_t j = j0 + jl;
      const bool ok = j < n && v0 + vv < p;
      sg_copy8(Rs + e, ok ? (const void*)(R + rowof[v0 + vv] + j) : (const void*)R, ok);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  float2 acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = make_float2(0.f, 0.f);
  const int nch = (p + 15) / 16;
  if (nch > 0) stage(0, 0);
  for (int ch = 0; ch < nch; ++ch) {
    if (ch + 1 < nch) {
      stage(16 * (ch + 1), (ch + 1) & 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // chunk ch has landed
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    const float2* Ms = sg_smem + (ch & 1) * (kSgMs + kSgRs);
    const float2* Rs = Ms + kSgMs;
    if (act) {
#pragma unroll
      for (int vv = 0; vv < 16; ++vv) {
        float2 m[4], r[8];
#pragma unroll
        for (int a = 0; a < 4; ++a) m[a] = Ms[(4 * ug + a) * 17 + vv];
#pragma unroll
        for (int b = 0; b < 8; ++b) r[b] = Rs[vv * 64 + cg + 8 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) {
            acc[a][b].x = fmaf(m[a].x, r[b].x, fmaf(-m[a].y, r[b].y, acc[a][b].x));
            acc[a][b].y = fmaf(m[a].x, r[b].y, fmaf(m[a].y, r[b].x, acc[a][b].y));
          }
      }
    }
    __syncthreads();                         // buffer ch & 1 is free for chunk ch + 2
  }
  // per-column scale 2^F_j over all u: the largest magnitude of each column over the u groups
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    float m = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) m = fmaxf(m, fmaxf(fabsf(acc[a][b].x), fabsf(acc[a][b].y)));
    smax[ug][cg + 8 * b] = act ? m : 0.f;
  }
  __syncthreads();
  if (!act) return;
  uint8_t* pair = Bops + (ct >> 1) * (int64_t)nkc * kC64PairBlock + (ct & 1) * kC64Half;
  const int u0 = 4 * ug;
  const int kA = u0, kB = P + u0;
  uint8_t* blkA = pair + (kA / kC64KC) * kC64PairBlock;   // hi part; lo part at + kC64Block
  uint8_t* blkB = pair + (kB / kC64KC) * kC64PairBlock;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int jl = cg + 8 * b;
    float mm = 0.f;
    for (int g = 0; g < 32; ++g) mm = fmaxf(mm, smax[g][jl]);
    const int F = scale_exp(mm);
    if (ug == 0) Fcol[j0 + jl] = F;
    const float sc = ldexpf(1.0f, kC64Exp - F);
    // columns 2j (re) and 2j+1 (im) of B':  k < P: (Re S, Im S);  k >= P: (-Im S, Re S)
    const int c_re = 2 * jl, c_im = 2 * jl + 1;
    __half rh[4], rl[4], ih[4], il[4], nh[4], nl[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      f16_split(acc[e][b].x * sc, rh[e], rl[e]);
      f16_split(acc[e][b].y * sc, ih[e], il[e]);
      f16_split(-acc[e][b].y * sc, nh[e], nl[e]);
    }
    const int oRa = c64_off(c_re, kA % kC64KC), oIa = c64_off(c_im, kA % kC64KC);
    const int oRb = c64_off(c_re, kB % kC64KC), oIb = c64_off(c_im, kB % kC64KC);
    st4h(blkA + oRa, rh[0], rh[1], rh[2], rh[3]);
    st4h(blkA + kC64Block + oRa, rl[0], rl[1], rl[2], rl[3]);
    st4h(blkA + oIa, ih[0], ih[1], ih[2], ih[3]);
    st4h(blkA + kC64Block + oIa, il[0], il[1], il[2], il[3]);
    st4h(blkB + oRb, nh[0], nh[1], nh[2], nh[3]);
    st4h(blkB + kC64Block + oRb, nl[0], nl[1], nl[2], nl[3]);
    st4h(blkB + oIb, rh[0], rh[1], rh[2], rh[3]);
    st4h(blkB + kC64Block + oIb, rl[0], rl[1], rl[2], rl[3]);
  }
}

// A float widened to FP64 by integer operations (exact: the FP64 conversion instruction runs on
// GB300's narrow FP64 pipe, which a kernel that widens every entry of C0 would then be bound by).
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  const uint64_t s = (uint64_t)(b >> 31) << 63;
  if (e == 0xFFu) return __longlong_as_double((long long)(s | 0x7FF0000000000000ull | ((uint64_t)m << 29)));
  if (e != 0u) return __longlong_as_double((long long)(s | ((uint64_t)(e + (1023 - 127)) << 52) | ((uint64_t)m << 29)));
  if (m == 0u) return __longlong_as_double((long long)s);
  const int t = 31 - __clz((int)m);                       // subnormal: m 2^-149, leading bit t
  return __longlong_as_double((long long)(s | ((uint64_t)(t - 149 + 1023) << 52) |
                                          (((uint64_t)m << (52 - t)) & 0x000FFFFFFFFFFFFFull)));
}

// ---- C0 = G[:, V] and the A operand blocks from it, a warp per row (lane l: u = 4l .. 4l + 3).
// The rows held are gathered once: C0 (FP64, for the field update) and the row's scaled
// split-FP16 operands, [Re C0[i, :P), Im C0[i, :P)] scaled by 2^(14 - E_i) -- in FP32, which
// gives the bits of the FP64 scaling of C0 (its entries are complex64 values, so the conversion
// is exact, and a power-of-two scaling rounds once either way).  Rows [grows, nrows_pad) are
// zero.  A warp's loads of one row merge where the set's pixels are neighbours (a brush's pairs).
__global__ void __launch_bounds__(256) k_c64_gather_rows(const float2* __restrict__ G, int64_t ldg,
                                                         const int32_t* __restrict__ V, int pmax, int64_t grows,
                                                         int64_t nrows_pad, const UpdCtl* __restrict__ ctl, int nkc,
                                                         cplx* __restrict__ C0, uint8_t* __restrict__ Aops,
                                                         int32_t* __restrict__ Erow) {
  if (ctl->skip) return;
  const int p = ctl->nv;
  const int P = (int)c64_padP(p);
  const int lane = threadIdx.x & 31, u0 = 4 * lane;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t vc[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) vc[e] = u0 + e < p ? V[u0 + e] : -1;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nrows_pad; i += nw) {
    float2 c[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) c[e] = (i < grows && vc[e] >= 0) ? G[i * ldg + vc[e]] : make_float2(0.f, 0.f);
    if (i < grows) {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (vc[e] >= 0) C0[i * pmax + u0 + e] = mk(f2d_bits(c[e].x), f2d_bits(c[e].y));
    }
    float m = 0.f;
#pragma unroll
    for (int e = 0; e < 4; ++e) m = fmaxf(m, fmaxf(fabsf(c[e].x), fabsf(c[e].y)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int E = scale_exp(m);
    if (lane == 0) Erow[i] = E;
    if (u0 < P) {
      const float sc = __int_as_float((127 + kC64Exp - E) << 23);
      __half rh[4], rl[4], ih[4], il[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        f16_split(c[e].x * sc, rh[e], rl[e]);
        f16_split(c[e].y * sc, ih[e], il[e]);
      }
      uint8_t* tile = Aops + (i / kC64M) * (int64_t)nkc * kC64Block;
      const int r = (int)(i % kC64M), kA = u0, kB = P + u0;
      uint8_t* blkA = tile + (kA / kC64KC) * kC64Block;
      uint8_t* blkB = tile + (kB / kC64KC) * kC64Block;
      const int oa = c64_off(r, kA % kC64KC), ob = c64_off(r, kB % kC64KC);
      st4h(blkA + oa, rh[0], rh[1], rh[2], rh[3]);
      st4h(blkA + kC64Half + oa, rl[0], rl[1], rl[2], rl[3]);
      st4h(blkB + ob, ih[0], ih[1], ih[2], ih[3]);
      st4h(blkB + kC64Half + ob, il[0], il[1], il[2], il[3]);
    }
  }
}

// 2^(E + F - 28) as an FP32 bit pattern (E, F >= -40 keep the biased exponent >= 19)
__device__ __forceinline__ float c64_scale(int E, int F) {
  return __int_as_float((E + F - 2 * kC64Exp + 127) << 23);
}

// G += 2^(E + F_j - 28) acc over one 128-byte row of a 128B-swizzled TMA box (16 complex
// columns: chunk ch holds complex columns 2ch, 2ch+1)
__device__ __forceinline__ void c64_epilogue_row(uint8_t* row, int r, int Ei, const int (&Fr)[16], const float (&acc)[32]) {
#pragma unroll
  for (int ch = 0; ch < 8; ++ch) {
    const float s0 = c64_scale(Ei, Fr[2 * ch]);
    const float s1 = c64_scale(Ei, Fr[2 * ch + 1]);
    float4* gp = reinterpret_cast<float4*>(row + ((ch ^ (r & 7)) << 4));
    float4 g = *gp;
    g.x = fmaf(s0, acc[4 * ch + 0], g.x);
    g.y = fmaf(s0, acc[4 * ch + 1], g.y);
    g.z = fmaf(s1, acc[4 * ch + 2], g.z);
    g.w = fmaf(s1, acc[4 * ch + 3], g.w);
    *gp = g;
  }
}

__device__ __forceinline__ void c64_load_f16(const int32_t* __restrict__ Fq, int (&Fr)[16]) {
  const int4* f4 = reinterpret_cast<const int4*>(Fq);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int4 v = f4[e];
    Fr[4 * e] = v.x;
    Fr[4 * e + 1] = v.y;
    Fr[4 * e + 2] = v.z;
    Fr[4 * e + 3] = v.w;
  }
}

// ---- resident-A form: joint rank p <= 48 (K <= 96) ------------------------------------------
// Each CTA owns one row tile at a time and sweeps a run of its column tiles (128 rows x 64
// complex columns).  The row tile's A chunks (nkr x 8 KB, at most 48 KB) are loaded once per run
// and stay in shared memory, so per tile only the B chunks (a ring of 8 KB stages) and the G
// tile move.  Runs: the row tiles are taken in groups of gridDim.x; in a full group CTA b takes
// row tile b of the group across every column tile, all CTAs stepping through the columns
// together (each B chunk is read from L2 by every CTA at about the same time); in the last group
// of R < gridDim.x row tiles each row is split into gridDim.x / R column segments.  Before it
// retires, every role waits (bounded) for the copies and MMAs it issued, so a CTA that gave up on
// a wait leaves nothing in flight.
// A chunks kept resident: K <= 96 (p <= 48).  At eight chunks (64 KB of A) the B ring would be
// too short to cover the L2 latency: p > 48 takes the streaming form below.
constexpr int kRaMaxK = 6;
constexpr int kRaMaxB = kC64Ops / kC64Block - 2;             // B stages when nkr = 2 (K = 32)
constexpr int kRaTmemCols = 256;                             // two buffers x kC64N columns

struct C64RaBars {
  uint64_t bfull[kRaMaxB], bempty[kRaMaxB];
  uint64_t afull, aempty;
  uint64_t gfull[kC64NSG], gempty[kC64NSG], ebar[kC64NSG];
  uint64_t tfull[2], tempty[2];
  uint64_t drain;
  uint32_t tslot;
  int abort;
};
static_assert(sizeof(C64RaBars) <= kC64Smem - kC64BarOff, "barrier block");

__global__ void __launch_bounds__(kC64Threads, 1)
k_rank_update_c64_ra(const __grid_constant__ CUtensorMap tmapG, int64_t n, int64_t nrt, int64_t nct, int nkc,
                     const uint8_t* __restrict__ Aops, const uint8_t* __restrict__ Bops,
                     const int32_t* __restrict__ Erow, const int32_t* __restrict__ Fcol,
                     const UpdCtl* __restrict__ ctl, int32_t* __restrict__ status, int32_t* __restrict__ prof_p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int p = ctl->skip ? 0 : ctl->nv;
  const int nkr = (int)(c64_padP(p) / 8);        // K chunks of this step (K = 2P)
  if (p <= 0 || nkr > kRaMaxK) return;           // uniform over the grid; larger K: streaming form
  if (prof_p && blockIdx.x == 0 && threadIdx.x == 0) *prof_p = p;
  C64RaBars* bars = reinterpret_cast<C64RaBars*>(smem + kC64BarOff);
  uint8_t* As = smem;                            // nkr A chunks of the current row tile
  uint8_t* Bs = smem + nkr * kC64Block;          // B ring
  const int nsb = kC64Ops / kC64Block - nkr;     // 6 .. kRaMaxB stages
  uint8_t* gts = smem + kC64Ops;                 // kC64NSG G half tiles
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile int* abort = &bars->abort;
  constexpr int kWarpGProd = kC64EpiWarps, kWarpMma = kC64EpiWarps + 1, kWarpStore = kC64EpiWarps + 2,
                kWarpOProd = kC64EpiWarps + 3;
  const int64_t G = gridDim.x, me = blockIdx.x;

  if (warp == kWarpMma) {
    tc::tmem_alloc(&bars->tslot, kRaTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int q = 0; q < nsb; ++q) {
      tc::mbar_init(&bars->bfull[q], 1);
      tc::mbar_init(&bars->bempty[q], 1);
    }
    tc::mbar_init(&bars->afull, 1);
    tc::mbar_init(&bars->aempty, 1);
    for (int q = 0; q < kC64NSG; ++q) {
      tc::mbar_init(&bars->gfull[q], 1);
      tc::mbar_init(&bars->gempty[q], 1);
      tc::mbar_init(&bars->ebar[q], 32 * kC64EpiWarps / 2);   // the epilogue warps of that half
    }
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&bars->tfull[q], 1);
      tc::mbar_init(&bars->tempty[q], kC64EpiWarps);
    }
    tc::mbar_init(&bars->drain, 1);
    bars->abort = 0;
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = bars->tslot;

  if (warp == kWarpGProd) {
    if (lane == 0) {
      int64_t k = 0, issued = 0;                 // tiles begun, half-tile uses issued
      bool ok = true;
      RaCursor cur;
      for (bool more = ra_first(cur, nrt, nct, G, me); more && ok; more = ra_next(cur, nrt, nct, G, me), ++k) {
        for (int hh = 0; hh < 2; ++hh) {
          const int64_t u = 2 * k + hh;
          const int s = (int)(u % kC64NSG);
          if (u >= kC64NSG && !tc::mbar_wait_or_abort(&bars->gempty[s], (uint32_t)((u / kC64NSG - 1) & 1), abort, kC64TimeoutNs)) { ok = false; break; }
          const int x0 = (int)(cur.c * kC64N) + 64 * hh, y = (int)(cur.rt * kC64M);     // x in floats
          int nbox = 0;
          for (int bx = 0; bx < 2; ++bx) nbox += (x0 + 32 * bx < 2 * n) ? 1 : 0;
          if (nbox == 0) tc::mbar_arrive(&bars->gfull[s]);
          else {
            tc::mbar_arrive_expect_tx(&bars->gfull[s], (uint32_t)(nbox * kC64Box));
            uint8_t* gt = gts + s * kC64GStage;
            for (int bx = 0; bx < nbox; ++bx) tc::tma_load_2d(gt + bx * kC64Box, &tmapG, x0 + 32 * bx, y, &bars->gfull[s]);
          }
          issued = u + 1;
        }
      }
      // every load issued has landed before the CTA may retire
      for (int64_t q = issued - kC64NSG; q < issued; ++q)
        if (q >= 0) tc::mbar_wait_bounded(&bars->gfull[q % kC64NSG], (uint32_t)((q / kC64NSG) & 1), kC64DrainNs);
    }
    __syncwarp();
  } else if (warp == kWarpOProd) {
    if (lane == 0) {
      const uint64_t pol_ops = tc::policy_evict_last();    // B chunks: read by every row tile
      int64_t c = 0, na = 0;                     // B chunks issued, A loads issued
      bool ok = true;
      RaCursor cur;
      for (bool more = ra_first(cur, nrt, nct, G, me); more && ok; more = ra_next(cur, nrt, nct, G, me)) {
        if (cur.c == cur.cbeg) {                 // a new run: its row tile's A chunks
          if (na >= 1 && !tc::mbar_wait_or_abort(&bars->aempty, (uint32_t)((na - 1) & 1), abort, kC64TimeoutNs)) break;
          tc::mbar_arrive_expect_tx(&bars->afull, (uint32_t)(nkr * kC64Block));
          for (int kc = 0; kc < nkr; ++kc)
            tc::bulk_g2s(As + kc * kC64Block, Aops + (cur.rt * nkc + kc) * (int64_t)kC64Block, kC64Block, &bars->afull);
          ++na;
        }
        // the column tile's half of each pair block: hi at +half 4 KB, lo at +8 KB + half 4 KB
        const uint8_t* bsrc = Bops + (cur.c >> 1) * (int64_t)nkc * kC64PairBlock + (cur.c & 1) * kC64Half;

        for (int kc = 0; kc < nkr; ++kc, ++c) {
          const int s = (int)(c % nsb);
          if (c >= nsb && !tc::mbar_wait_or_abort(&bars->bempty[s], (uint32_t)((c / nsb - 1) & 1), abort, kC64TimeoutNs)) { ok = false; break; }
          tc::mbar_arrive_expect_tx(&bars->bfull[s], (uint32_t)kC64Block);
          const uint8_t* src = bsrc + kc * (int64_t)kC64PairBlock;
          tc::bulk_g2s_hint(Bs + s * kC64Block, src, kC64Half, &bars->bfull[s], pol_ops);
          tc::bulk_g2s_hint(Bs + s * kC64Block + kC64Half, src + kC64Block, kC64Half, &bars->bfull[s], pol_ops);
        }
      }
      // every copy issued has landed before the CTA may retire
      if (na >= 1) tc::mbar_wait_bounded(&bars->afull, (uint32_t)((na - 1) & 1), kC64DrainNs);
      for (int64_t q = c - nsb; q < c; ++q)
        if (q >= 0) tc::mbar_wait_bounded(&bars->bfull[q % nsb], (uint32_t)((q / nsb) & 1), kC64DrainNs);
    }
    __syncwarp();
  } else if (warp == kWarpMma) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_f16(kC64M, kC64N);
      int64_t k = 0, c = 0, na = 0;
      bool ok = true;
      RaCursor cur;
      for (bool more = ra_first(cur, nrt, nct, G, me); more && ok; more = ra_next(cur, nrt, nct, G, me), ++k) {
        if (cur.c == cur.cbeg) {
          if (!tc::mbar_wait_or_abort(&bars->afull, (uint32_t)(na & 1), abort, kC64TimeoutNs)) break;
          ++na;
        }
        const int b = (int)(k & 1);
        if (k >= 2 && !tc::mbar_wait_or_abort(&bars->tempty[b], (uint32_t)((k / 2 - 1) & 1), abort, kC64TimeoutNs)) break;
        tc::fence_after_sync();
        const uint32_t d = tbase + (uint32_t)(b * kC64N);
        for (int kc = 0; kc < nkr; ++kc, ++c) {
          const int s = (int)(c % nsb);
          if (!tc::mbar_wait_or_abort(&bars->bfull[s], (uint32_t)((c / nsb) & 1), abort, kC64TimeoutNs)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t sA = tc::smem_u32(As + kc * kC64Block);
          const uint32_t sB = tc::smem_u32(Bs + s * kC64Block);
          const uint64_t ah = tc::smem_desc(sA, kC64Lbo, kC64Sbo), al = tc::smem_desc(sA + kC64Half, kC64Lbo, kC64Sbo);
          const uint64_t bh = tc::smem_desc(sB, kC64Lbo, kC64Sbo), bl = tc::smem_desc(sB + kC64Half, kC64Lbo, kC64Sbo);
          tc::mma_f16(d, ah, bh, idesc, kc == 0 ? 0u : 1u);
          tc::mma_f16(d, ah, bl, idesc, 1u);
          tc::mma_f16(d, al, bh, idesc, 1u);
          tc::mma_commit(&bars->bempty[s]);
        }
        if (!ok) break;
        tc::mma_commit(&bars->tfull[b]);
        if (cur.c == cur.cend - 1) tc::mma_commit(&bars->aempty);    // last tile of the run
      }
      // every MMA issued has completed before the CTA may release TMEM and retire
      tc::mma_commit(&bars->drain);
      tc::mbar_wait_bounded(&bars->drain, 0u, kC64DrainNs);
    }
    __syncwarp();
  } else if (warp < kC64EpiWarps) {
    const int q = warp & 3, h = warp >> 2;     // TMEM lane quarter, column quarter (32 real columns)
    const int r = q * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
    int64_t k = 0;
    RaCursor cur;
    for (bool more = ra_first(cur, nrt, nct, G, me); more; more = ra_next(cur, nrt, nct, G, me), ++k) {
      const int64_t rt = cur.rt, ct = cur.c;
      const int b = (int)(k & 1);
      const int64_t u = 2 * k + (h >> 1);      // this warp's half of the tile
      const int s = (int)(u % kC64NSG);
      // the scale exponents first: their loads overlap the waits below
      const int Ei = Erow[rt * kC64M + r];
      int Fr[16];
      c64_load_f16(Fcol + ct * (kC64N / 2) + h * 16, Fr);
      if (!tc::mbar_wait_or_abort(&bars->tfull[b], (uint32_t)((k / 2) & 1), abort, kC64TimeoutNs)) break;
      if (!tc::mbar_wait_or_abort(&bars->gfull[s], (uint32_t)((u / kC64NSG) & 1), abort, kC64TimeoutNs)) break;
      tc::fence_after_sync();
      float acc[32];
      {
        float a0[16], a1[16];
        const uint32_t base = tbase + lane_addr + (uint32_t)(b * kC64N + h * 32);
        tc::tmem_ld16(base, a0);
        tc::tmem_ld16(base + 16, a1);
        tc::tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          acc[e] = a0[e];
          acc[16 + e] = a1[e];
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars->tempty[b]);
      // box h & 1 of the half tile holds real columns 32h .. 32h+31 of the tile
      c64_epilogue_row(gts + s * kC64GStage + (h & 1) * kC64Box + r * 128, r, Ei, Fr, acc);
      tc::fence_proxy_async_smem();
      tc::mbar_arrive(&bars->ebar[s]);
    }
  }
  if (warp == kWarpStore) {
    if (lane == 0) {
      int64_t k = 0;
      bool ok = true;
      RaCursor cur;
      for (bool more = ra_first(cur, nrt, nct, G, me); more && ok; more = ra_next(cur, nrt, nct, G, me), ++k) {
        for (int hh = 0; hh < 2; ++hh) {
          const int64_t u = 2 * k + hh;
          const int s = (int)(u % kC64NSG);
          if (!tc::mbar_wait_or_abort(&bars->ebar[s], (uint32_t)((u / kC64NSG) & 1), abort, kC64TimeoutNs)) { ok = false; break; }
          const int x0 = (int)(cur.c * kC64N) + 64 * hh, y = (int)(cur.rt * kC64M);
          uint8_t* gt = gts + s * kC64GStage;
          for (int bx = 0; bx < 2; ++bx)
            if (x0 + 32 * bx < 2 * n) tc::tma_store_2d(&tmapG, x0 + 32 * bx, y, gt + bx * kC64Box);
          tc::bulk_commit();
          tc::bulk_wait_read0();
          tc::mbar_arrive(&bars->gempty[s]);
        }
      }
      tc::bulk_wait0();
    }
    __syncwarp();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0 && bars->abort) atomicExch(status, GF_ETIMEOUT);
  tc::fence_after_sync();
  if (warp == kWarpMma) tc::tmem_dealloc(tbase, kRaTmemCols);
}

// ---- streaming form: joint rank p > 48 (K up to 256) ----------------------------------------
// Persistent, warp-specialised; tiles of 128 rows x 128 complex columns (256 real: one column-
// tile pair of the operand blocks) in a grouped raster order, tile t handled by CTA t mod
// gridDim (neighbouring CTAs share the operand chunks through L2).  Per 16-deep K chunk a CTA
// brings in 8 KB of A and 16 KB of B (a 24 KB stage, four stages), so a 128 KB G tile costs
// 3 operand bytes per G byte; the accumulator is one 128 x 256 FP32 block (256 TMEM columns,
// double-buffered).  G moves as four 32 KB quarter tiles (two TMA boxes each), so a whole tile's
// G is staged while the MMAs of the next tile run.
//   warps 0..15  epilogue (lane quarter q = warp & 3, column quarter h = warp >> 2)
//   warp 16      G producer    warp 17  MMA issuer    warp 18  storer    warp 19  operand producer
// Before it retires, every role waits (bounded) for the copies and MMAs it issued.
constexpr int kWsStage = kC64Block + kC64PairBlock;          // 24 KB
constexpr int kWsNSO = kC64Ops / kWsStage;                   // 4 operand stages
constexpr int kWsTmemCols = 512;                             // two buffers x kC64WN columns
static_assert(kWsStage % 1024 == 0 && kWsNSO == 4, "operand stages");

struct C64WBars {
  uint64_t ofull[kWsNSO], oempty[kWsNSO];
  uint64_t gfull[kC64NSG], gempty[kC64NSG], ebar[kC64NSG];
  uint64_t tfull[2], tempty[2];
  uint64_t drain;
  uint32_t tslot;
  int abort;
};
static_assert(sizeof(C64WBars) <= kC64Smem - kC64BarOff, "barrier block");

__device__ __forceinline__ void c64_tile_coords(int64_t t, int64_t nrt, int64_t ncol, int64_t& rt, int64_t& ct) {
  const int64_t per_group = (int64_t)kC64Group * ncol;
  const int64_t g = t / per_group;
  const int64_t rem = t - g * per_group;
  const int64_t rows_in_group = (nrt - g * kC64Group) < kC64Group ? (nrt - g * kC64Group) : kC64Group;
  rt = g * kC64Group + rem % rows_in_group;
  ct = rem / rows_in_group;
}

__global__ void __launch_bounds__(kC64Threads, 1)
k_rank_update_c64_wide(const __grid_constant__ CUtensorMap tmapG, int64_t n, int64_t nrt, int64_t ncp, int nkc,
                       const uint8_t* __restrict__ Aops, const uint8_t* __restrict__ Bops,
                       const int32_t* __restrict__ Erow, const int32_t* __restrict__ Fcol,
                       const UpdCtl* __restrict__ ctl, int32_t* __restrict__ status, int32_t* __restrict__ prof_p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int p = ctl->skip ? 0 : ctl->nv;
  const int nkr = (int)(c64_padP(p) / 8);        // K chunks of this step (K = 2P); nkc is the block stride
  if (p <= 0 || nkr <= kRaMaxK) return;          // uniform over the grid; the resident-A form took it
  if (prof_p && blockIdx.x == 0 && threadIdx.x == 0) *prof_p = p;
  C64WBars* bars = reinterpret_cast<C64WBars*>(smem + kC64BarOff);
  uint8_t* ops = smem;                           // kWsNSO x (A chunk, B pair chunk)
  uint8_t* gts = smem + kC64Ops;                 // kC64NSG G quarter tiles
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile int* abort = &bars->abort;
  constexpr int kWarpGProd = kC64EpiWarps, kWarpMma = kC64EpiWarps + 1, kWarpStore = kC64EpiWarps + 2,
                kWarpOProd = kC64EpiWarps + 3;
  const int64_t cid = blockIdx.x, ncl = gridDim.x;
  const int64_t T = nrt * ncp;

  if (warp == kWarpMma) {
    tc::tmem_alloc(&bars->tslot, kWsTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int q = 0; q < kWsNSO; ++q) {
      tc::mbar_init(&bars->ofull[q], 1);
      tc::mbar_init(&bars->oempty[q], 1);
    }
    for (int q = 0; q < kC64NSG; ++q) {
      tc::mbar_init(&bars->gfull[q], 1);
      tc::mbar_init(&bars->gempty[q], 1);
      tc::mbar_init(&bars->ebar[q], 32 * kC64EpiWarps / 4);   // the four epilogue warps of that quarter
    }
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&bars->tfull[q], 1);
      tc::mbar_init(&bars->tempty[q], kC64EpiWarps);
    }
    tc::mbar_init(&bars->drain, 1);
    bars->abort = 0;
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = bars->tslot;

  if (warp == kWarpGProd) {
    if (lane == 0) {
      int64_t k = 0;                             // tiles begun (every tile uses all four stages once)
      int64_t fills[kC64NSG] = {0, 0, 0, 0};     // loads issued into each stage
      bool ok = true;
      for (int64_t t = cid; t < T && ok; t += ncl, ++k) {
        int64_t rt, cp;
        c64_tile_coords(t, nrt, ncp, rt, cp);
        for (int s = 0; s < kC64NSG; ++s) {      // quarter s of the tile goes to stage s
          if (k >= 1 && !tc::mbar_wait_or_abort(&bars->gempty[s], (uint32_t)((k - 1) & 1), abort, kC64TimeoutNs)) { ok = false; break; }
          const int x0 = (int)(cp * kC64WN) + 64 * s, y = (int)(rt * kC64M);      // x in floats
          int nbox = 0;
          for (int bx = 0; bx < 2; ++bx) nbox += (x0 + 32 * bx < 2 * n) ? 1 : 0;
          if (nbox == 0) tc::mbar_arrive(&bars->gfull[s]);
          else {
            tc::mbar_arrive_expect_tx(&bars->gfull[s], (uint32_t)(nbox * kC64Box));
            uint8_t* gt = gts + s * kC64GStage;
            for (int bx = 0; bx < nbox; ++bx) tc::tma_load_2d(gt + bx * kC64Box, &tmapG, x0 + 32 * bx, y, &bars->gfull[s]);
          }
          ++fills[s];
        }
      }
      // every load issued has landed before the CTA may retire
      for (int s = 0; s < kC64NSG; ++s)
        if (fills[s] >= 1) tc::mbar_wait_bounded(&bars->gfull[s], (uint32_t)((fills[s] - 1) & 1), kC64DrainNs);
    }
    __syncwarp();
  } else if (warp == kWarpOProd) {
    if (lane == 0) {
      const uint64_t pol_ops = tc::policy_evict_last();    // operand chunks: re-read by many tiles
      int64_t c = 0;
      bool ok = true;
      for (int64_t t = cid; t < T && ok; t += ncl) {
        int64_t rt, cp;
        c64_tile_coords(t, nrt, ncp, rt, cp);
        for (int kc = 0; kc < nkr; ++kc, ++c) {
          const int s = (int)(c % kWsNSO);
          if (c >= kWsNSO && !tc::mbar_wait_or_abort(&bars->oempty[s], (uint32_t)((c / kWsNSO - 1) & 1), abort, kC64TimeoutNs)) { ok = false; break; }
          uint8_t* st = ops + s * kWsStage;
          tc::mbar_arrive_expect_tx(&bars->ofull[s], (uint32_t)kWsStage);
          tc::bulk_g2s_hint(st, Aops + (rt * nkc + kc) * (int64_t)kC64Block, kC64Block, &bars->ofull[s], pol_ops);
          tc::bulk_g2s_hint(st + kC64Block, Bops + (cp * nkc + kc) * (int64_t)kC64PairBlock, kC64PairBlock,
                            &bars->ofull[s], pol_ops);
        }
      }
      // every copy issued has landed before the CTA may retire
      for (int64_t q = c - kWsNSO; q < c; ++q)
        if (q >= 0) tc::mbar_wait_bounded(&bars->ofull[q % kWsNSO], (uint32_t)((q / kWsNSO) & 1), kC64DrainNs);
    }
    __syncwarp();
  } else if (warp == kWarpMma) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_f16(kC64M, kC64WN);
      int64_t k = 0, c = 0;
      bool ok = true;
      for (int64_t t = cid; t < T && ok; t += ncl, ++k) {
        const int b = (int)(k & 1);
        if (k >= 2 && !tc::mbar_wait_or_abort(&bars->tempty[b], (uint32_t)((k / 2 - 1) & 1), abort, kC64TimeoutNs)) break;
        tc::fence_after_sync();
        const uint32_t d = tbase + (uint32_t)(b * kC64WN);
        for (int kc = 0; kc < nkr; ++kc, ++c) {
          const int s = (int)(c % kWsNSO);
          if (!tc::mbar_wait_or_abort(&bars->ofull[s], (uint32_t)((c / kWsNSO) & 1), abort, kC64TimeoutNs)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t sA = tc::smem_u32(ops + s * kWsStage);
          const uint32_t sB = sA + kC64Block;    // 256 rows: hi at +0 (8 KB), lo at +8 KB
          const uint64_t ah = tc::smem_desc(sA, kC64Lbo, kC64Sbo), al = tc::smem_desc(sA + kC64Half, kC64Lbo, kC64Sbo);
          const uint64_t bh = tc::smem_desc(sB, kC64Lbo, kC64Sbo), bl = tc::smem_desc(sB + kC64Block, kC64Lbo, kC64Sbo);
          tc::mma_f16(d, ah, bh, idesc, kc == 0 ? 0u : 1u);
          tc::mma_f16(d, ah, bl, idesc, 1u);
          tc::mma_f16(d, al, bh, idesc, 1u);
          tc::mma_commit(&bars->oempty[s]);
        }
        if (ok) tc::mma_commit(&bars->tfull[b]);
      }
      // every MMA issued has completed before the CTA may release TMEM and retire
      tc::mma_commit(&bars->drain);
      tc::mbar_wait_bounded(&bars->drain, 0u, kC64DrainNs);
    }
    __syncwarp();
  } else if (warp < kC64EpiWarps) {
    const int q = warp & 3, h = warp >> 2;     // TMEM lane quarter, column quarter (32 complex columns)
    const int r = q * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
    int64_t k = 0;
    for (int64_t t = cid; t < T; t += ncl, ++k) {
      int64_t rt, cp;
      c64_tile_coords(t, nrt, ncp, rt, cp);
      const int b = (int)(k & 1);
      const int Ei = Erow[rt * kC64M + r];
      if (!tc::mbar_wait_or_abort(&bars->tfull[b], (uint32_t)((k / 2) & 1), abort, kC64TimeoutNs)) break;
      if (!tc::mbar_wait_or_abort(&bars->gfull[h], (uint32_t)(k & 1), abort, kC64TimeoutNs)) break;
      tc::fence_after_sync();
      for (int bx = 0; bx < 2; ++bx) {         // box bx of quarter h: real columns 64h + 32bx .. +31
        int Fr[16];
        c64_load_f16(Fcol + cp * (kC64WN / 2) + h * 32 + bx * 16, Fr);
        float acc[32];
        {
          float a0[16], a1[16];
          const uint32_t base = tbase + lane_addr + (uint32_t)(b * kC64WN + h * 64 + bx * 32);
          tc::tmem_ld16(base, a0);
          tc::tmem_ld16(base + 16, a1);
          tc::tmem_ld_wait();
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            acc[e] = a0[e];
            acc[16 + e] = a1[e];
          }
        }
        c64_epilogue_row(gts + h * kC64GStage + bx * kC64Box + r * 128, r, Ei, Fr, acc);
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars->tempty[b]);
      tc::fence_proxy_async_smem();
      tc::mbar_arrive(&bars->ebar[h]);
    }
  }
  if (warp == kWarpStore) {
    if (lane == 0) {
      int64_t k = 0;
      bool ok = true;
      for (int64_t t = cid; t < T && ok; t += ncl, ++k) {
        int64_t rt, cp;
        c64_tile_coords(t, nrt, ncp, rt, cp);
        for (int s = 0; s < kC64NSG; ++s) {
          if (!tc::mbar_wait_or_abort(&bars->ebar[s], (uint32_t)(k & 1), abort, kC64TimeoutNs)) { ok = false; break; }
          const int x0 = (int)(cp * kC64WN) + 64 * s, y = (int)(rt * kC64M);
          uint8_t* gt = gts + s * kC64GStage;
          for (int bx = 0; bx < 2; ++bx)
            if (x0 + 32 * bx < 2 * n) tc::tma_store_2d(&tmapG, x0 + 32 * bx, y, gt + bx * kC64Box);
          tc::bulk_commit();
          tc::bulk_wait_read0();
          tc::mbar_arrive(&bars->gempty[s]);
        }
      }
      tc::bulk_wait0();
    }
    __syncwarp();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0 && bars->abort) atomicExch(status, GF_ETIMEOUT);
  tc::fence_after_sync();
  if (warp == kWarpMma) tc::tmem_dealloc(tbase, kWsTmemCols);
}

static PFN_cuTensorMapEncodeTiled_v12000 c64_encode_fn() {
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

// complex64 G as a 2-D tensor of floats: 2n columns by `rows` rows (n, or a row block), row
// stride 8 ldg bytes; boxes of 32 floats (128 B) x 128 rows, 128-byte swizzle.
static bool make_tmap_G64(CUtensorMap* m, float2* G, int64_t ldg, int64_t n, int64_t rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = c64_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)(2 * n), (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(8 * ldg)};
  cuuint32_t box[2] = {32, (cuuint32_t)kC64M};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)G, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool c64_tc_make_map(float2* G, int64_t ldg, int64_t n, int64_t rows, void* map128) {
  return make_tmap_G64(reinterpret_cast<CUtensorMap*>(map128), G, ldg, n, rows);
}

void launch_rank_update_c64_tc(const void* map128, float2* G, int64_t ldg, int64_t n, int64_t grows,
                               const void* vrows, int64_t ldv, const WsLayout& L, char* ws, int lam,
                               int32_t* status, int32_t* prof_p, int sm_count, cudaStream_t st) {
  const CUtensorMap& tmap = *reinterpret_cast<const CUtensorMap*>(map128);
  C64Layout o = c64_layout(n, L.pmax);
  o.nrt = (grows + kC64M - 1) / kC64M;       // row tiles of the rows held (n, or a row block)
  const UpdCtl* ctl = reinterpret_cast<const UpdCtl*>(ws + L.ctl);
  float2* Mdai = reinterpret_cast<float2*>(ws + L.c64M);
  uint8_t* Aops = reinterpret_cast<uint8_t*>(ws + L.c64A);
  uint8_t* Bops = reinterpret_cast<uint8_t*>(ws + L.c64B);
  const cplx* C0 = reinterpret_cast<const cplx*>(ws + L.C0 + lam * L.panel_s);
  // once per device: shared-memory opt-in of both update forms and of the S GEMM's buffers
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || !done[dev]) {
      cudaFuncSetAttribute(k_rank_update_c64_ra, cudaFuncAttributeMaxDynamicSharedMemorySize, kC64Smem);
      cudaFuncSetAttribute(k_rank_update_c64_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, kC64Smem);
      cudaFuncSetAttribute(k_c64_s_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSgSmem);
      if (dev >= 0 && dev < 64) done[dev] = true;
    }
  }
  k_c64_inverse<<<L.pmax, 128, 0, st>>>(L, ws, lam, Mdai);
  int32_t* Erow = reinterpret_cast<int32_t*>(ws + L.c64E);
  int32_t* Fcol = reinterpret_cast<int32_t*>(ws + L.c64F);
  if (vrows)      // the rows G[V, :] from the caller's panel (a shard of G does not hold them)
    k_c64_s_gemm<<<(unsigned)(2 * o.ncp), 256, kSgSmem, st>>>(reinterpret_cast<const float2*>(vrows), ldv, n, Mdai,
                                                               nullptr, ctl, (int)o.nkc, Bops, Fcol);
  else
    k_c64_s_gemm<<<(unsigned)(2 * o.ncp), 256, kSgSmem, st>>>(G, ldg, n, Mdai,
                                                               reinterpret_cast<const int32_t*>(ws + L.V), ctl,
                                                               (int)o.nkc, Bops, Fcol);
  {
    const int64_t rows = o.nrt * kC64M;
    const int64_t b = (rows + 7) / 8;                       // eight rows (warps) per CTA
    k_c64_gather_rows<<<(int)(b < 4864 ? b : 4864), 256, 0, st>>>(G, ldg, reinterpret_cast<const int32_t*>(ws + L.V),
                                                                   L.pmax, grows, rows, ctl, (int)o.nkc,
                                                                   const_cast<cplx*>(C0), Aops, Erow);
  }
  // joint rank p <= 48 (decided on the device): the resident-A form; larger p: the streaming
  // form, launched only where the workspace allows p > 48 (each returns at once when the other
  // applies)
  {
    const int64_t tiles = o.nrt * o.nct;
    const int grid = (int)(tiles < sm_count ? tiles : sm_count);
    k_rank_update_c64_ra<<<grid, kC64Threads, kC64Smem, st>>>(tmap, n, o.nrt, o.nct, (int)o.nkc, Aops, Bops, Erow,
                                                               Fcol, ctl, status, prof_p);
    if (o.nkc <= kRaMaxK) return;
  }
  const int64_t tiles = o.nrt * o.ncp;
  const int grid = (int)(tiles < sm_count ? tiles : sm_count);
  k_rank_update_c64_wide<<<grid, kC64Threads, kC64Smem, st>>>(tmap, n, o.nrt, o.ncp, (int)o.nkc, Aops, Bops, Erow,
                                                               Fcol, ctl, status, prof_p);
}

}  // namespace gf
