// The optimizer in 3-D (the paper's Sec. II with 3x3 dyadic blocks, Sec. IV's pillar updates):
// the fill of the 3n x 3n background matrix, the dFOM of every pillar candidate and the entry
// points; selection and the update reuse the 2-D kernels on the 3 (N + 1) unknowns.
//
//   G0(R) = e^{ikR} / (4 pi R) [A(kR) I + B(kR) R^ R^],  A = 1 + (i kR - 1)/(kR)^2,
//           B = (3 - 3 i kR - (kR)^2)/(kR)^2,  folded with k^2 dV;
//   voxel self block = [(2/3)((1 - i k a) e^{ika} - 1) - 1/3] I  (principal volume over the
//           equal-volume sphere, radius a, with the depolarisation I/3).
#include <math.h>

#include <mutex>

#include "gf_internal.cuh"

namespace gf {

constexpr int kEv3Threads = 128;
constexpr int kEv3MaxP = 96;            // 12 nz unknowns per pillar, nz <= 8

struct Geo3 {
  int nx, ny, nz;
  int64_t N;          // voxels
  int64_t n;          // unknowns 3 (N + 1)
  double dx, k, chi;
  double mx, my, mz;
};

static Geo3 geo3(const gf_geom3d& g) {
  Geo3 o;
  o.nx = g.nx;
  o.ny = g.ny;
  o.nz = g.nz;
  o.N = (int64_t)g.nx * g.ny * g.nz;
  o.n = 3 * (o.N + 1);
  o.dx = g.dx;
  o.k = 2.0 * M_PI / g.wavelength;
  o.chi = g.eps_mat - g.eps_bg;
  o.mx = g.mon_x;
  o.my = g.mon_y;
  o.mz = g.mon_z;
  return o;
}

// k^2 dV e^{ikR}/(4 pi R) times A and times B / R^2 (so that B R^_a R^_b = that * R_a R_b)
__device__ __forceinline__ void dyadic_parts(const Geo3& g, double R, cplx& fA, cplx& fB) {
  const double kr = g.k * R;
  double sn, cs;
  sincos(kr, &sn, &cs);
  const double c = g.k * g.k * g.dx * g.dx * g.dx / (4.0 * M_PI * R);
  const cplx ph = mk(c * cs, c * sn);
  const double ikr2 = 1.0 / (kr * kr);
  const cplx A = mk(1.0 - ikr2, kr * ikr2);                     // 1 + (i kr - 1)/kr^2
  const cplx Bc = mk(3.0 * ikr2 - 1.0, -3.0 * kr * ikr2);       // (3 - 3 i kr - kr^2)/kr^2
  fA = ph * A;
  fB = (1.0 / (R * R)) * (ph * Bc);
}

__device__ __forceinline__ cplx self_block(const Geo3& g) {
  const double a = cbrt(3.0 * g.dx * g.dx * g.dx / (4.0 * M_PI));
  const double ka = g.k * a;
  double sn, cs;
  sincos(ka, &sn, &cs);
  const cplx e = mk(cs, sn);
  const cplx t = mk(1.0, -ka) * e;                                // (1 - i ka) e^{ika}
  return mk((2.0 / 3.0) * (t.re - 1.0) - 1.0 / 3.0, (2.0 / 3.0) * t.im);
}

// table over lattice offsets (|dx|, |dy|, |dz|): entry 2 t = fA, 2 t + 1 = fB / dx^2-scaled so that
// the block is fA I + fB' d d^T with integer offsets d
__global__ void k_fill3_table(Geo3 g, cplx* __restrict__ table, float4* __restrict__ table32) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.N; t += (int64_t)gridDim.x * blockDim.x) {
    const int dz = (int)(t / ((int64_t)g.nx * g.ny));
    const int64_t r = t - (int64_t)dz * g.nx * g.ny;
    const int dy = (int)(r / g.nx), dxi = (int)(r - (int64_t)dy * g.nx);
    cplx fA, fB;
    if (t == 0) {
      fA = self_block(g);
      fB = mk(0.0, 0.0);
    } else {
      const double d2 = (double)dxi * dxi + (double)dy * dy + (double)dz * dz;
      dyadic_parts(g, g.dx * sqrt(d2), fA, fB);
      fB = (g.dx * g.dx) * fB;                                      // times integer d_a d_b
    }
    table[2 * t] = fA;
    table[2 * t + 1] = fB;
    table32[t] = make_float4((float)fA.re, (float)fA.im, (float)fB.re, (float)fB.im);
  }
}

// complex64 storage: the same assembly in FP32 from the FP32 copy of the table (the stored
// value is FP32 anyway; the FP64 form of this loop is bound by the FP64 pipe)
__global__ void __launch_bounds__(256) k_fill3_expand_f32(Geo3 g, int64_t ldg, const float4* __restrict__ table32,
                                                          float2* __restrict__ G) {
  const int64_t nxy = (int64_t)g.nx * g.ny;
  for (int64_t u = blockIdx.x; u < 3 * g.N; u += gridDim.x) {
    const int64_t i = u / 3;
    const int a = (int)(u - 3 * i);
    const int iz = (int)(i / nxy);
    const int64_t ri = i - iz * nxy;
    const int iy = (int)(ri / g.nx), ix = (int)(ri - (int64_t)iy * g.nx);
    float2* row = G + u * ldg;
    int64_t j = threadIdx.x;
    int jz = (int)(j / nxy);
    int64_t rj = j - jz * nxy;
    int jy = (int)(rj / g.nx), jx = (int)(rj - (int64_t)jy * g.nx);
    for (; j < g.N; j += blockDim.x) {
      const int d[3] = {ix - jx, iy - jy, iz - jz};
      const int ax = d[0] < 0 ? -d[0] : d[0], ay = d[1] < 0 ? -d[1] : d[1], az = d[2] < 0 ? -d[2] : d[2];
      const float4 tv = table32[((int64_t)az * g.ny + ay) * g.nx + ax];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float w = (float)(d[a] * d[b]);
        float2 v = make_float2(tv.z * w, tv.w * w);
        if (a == b) {
          v.x += tv.x;
          v.y += tv.y;
        }
        row[3 * j + b] = v;
      }
      jx += blockDim.x;
      while (jx >= g.nx) {
        jx -= g.nx;
        if (++jy >= g.ny) { jy = 0; ++jz; }
      }
    }
    for (int64_t c = g.n + threadIdx.x; c < ldg; c += blockDim.x) row[c] = make_float2(0.f, 0.f);
  }
}

template <typename T>
__device__ __forceinline__ void st3(T* p, cplx v);
template <>
__device__ __forceinline__ void st3<double2>(double2* p, cplx v) { *p = make_double2(v.re, v.im); }
template <>
__device__ __forceinline__ void st3<float2>(float2* p, cplx v) { *p = make_float2((float)v.re, (float)v.im); }

// voxel rows: row u = 3 i + a, columns 3 j + b of voxel j (a thread per voxel, coordinates
// advanced incrementally); also zeroes the padding columns
template <typename T>
__global__ void __launch_bounds__(256) k_fill3_expand(Geo3 g, int64_t ldg, const cplx* __restrict__ table,
                                                      T* __restrict__ G) {
  const int64_t nxy = (int64_t)g.nx * g.ny;
  for (int64_t u = blockIdx.x; u < 3 * g.N; u += gridDim.x) {
    const int64_t i = u / 3;
    const int a = (int)(u - 3 * i);
    const int iz = (int)(i / nxy);
    const int64_t ri = i - iz * nxy;
    const int iy = (int)(ri / g.nx), ix = (int)(ri - (int64_t)iy * g.nx);
    T* row = G + u * ldg;
    int64_t j = threadIdx.x;
    int jz = (int)(j / nxy);
    int64_t rj = j - jz * nxy;
    int jy = (int)(rj / g.nx), jx = (int)(rj - (int64_t)jy * g.nx);
    for (; j < g.N; j += blockDim.x) {
      const int d[3] = {ix - jx, iy - jy, iz - jz};
      const int ax = d[0] < 0 ? -d[0] : d[0], ay = d[1] < 0 ? -d[1] : d[1], az = d[2] < 0 ? -d[2] : d[2];
      const int64_t t = ((int64_t)az * g.ny + ay) * g.nx + ax;
      const cplx fA = table[2 * t], fB = table[2 * t + 1];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        cplx v = (double)(d[a] * d[b]) * fB;
        if (a == b) v = v + fA;
        st3<T>(row + 3 * j + b, v);
      }
      jx += blockDim.x;
      while (jx >= g.nx) {
        jx -= g.nx;
        if (++jy >= g.ny) { jy = 0; ++jz; }
      }
    }
    for (int64_t c = g.n + threadIdx.x; c < ldg; c += blockDim.x) st3<T>(row + c, mk(0.0, 0.0));
  }
}

// monitor blocks (row and column of every voxel), the monitor rows' own block and padding, E_inc
template <typename T>
__global__ void k_fill3_monitor(Geo3 g, int64_t ldg, T* __restrict__ G, cplx* __restrict__ E) {
  const int64_t nxy = (int64_t)g.nx * g.ny;
  const int64_t m0 = 3 * g.N;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= g.N; j += (int64_t)gridDim.x * blockDim.x) {
    double zj;
    if (j < g.N) {
      const int jz = (int)(j / nxy);
      const int64_t rj = j - jz * nxy;
      const int jy = (int)(rj / g.nx), jx = (int)(rj - (int64_t)jy * g.nx);
      const double R[3] = {(jx + 0.5) * g.dx - g.mx, (jy + 0.5) * g.dx - g.my, (jz + 0.5) * g.dx - g.mz};
      const double r = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
      cplx fA, fB;
      dyadic_parts(g, r, fA, fB);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          cplx v = (R[a] * R[b]) * fB;
          if (a == b) v = v + fA;
          st3<T>(G + (3 * j + a) * ldg + m0 + b, v);        // column of the monitor
          st3<T>(G + (m0 + a) * ldg + 3 * j + b, v);        // row of the monitor (G0 is even, symmetric)
        }
      zj = (jz + 0.5) * g.dx;
    } else {
      for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) st3<T>(G + (m0 + a) * ldg + m0 + b, mk(0.0, 0.0));
        for (int64_t c = g.n; c < ldg; ++c) st3<T>(G + (m0 + a) * ldg + c, mk(0.0, 0.0));
      }
      zj = g.mz;
    }
    double sn, cs;
    sincos(g.k * zj, &sn, &cs);
    E[3 * j] = mk(cs, sn);
    E[3 * j + 1] = mk(0.0, 0.0);
    E[3 * j + 2] = mk(0.0, 0.0);
  }
}

// ---- dFOM of every pillar: one CTA per candidate, its 3p x 3p system in shared memory
struct Ev3Args {
  Geo3 g;
  int dtype;
  const void* G;
  int64_t ldg;
  const cplx* E;
};

__device__ __forceinline__ void block_argmax(double& v, int& idx, double* sv, int* si) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, v, o);
    const int oi = __shfl_down_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if (lane == 0) { sv[w] = v; si[w] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < nw; ++q)
      if (sv[q] > sv[0] || (sv[q] == sv[0] && si[q] < si[0])) { sv[0] = sv[q]; si[0] = si[q]; }
  }
  __syncthreads();
  v = sv[0];
  idx = si[0];
  __syncthreads();
}

__device__ __forceinline__ cplx block_sum(cplx v, cplx* sc) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    v.re += __shfl_down_sync(0xffffffffu, v.re, o);
    v.im += __shfl_down_sync(0xffffffffu, v.im, o);
  }
  if (lane == 0) sc[w] = v;
  __syncthreads();
  cplx t = mk(0.0, 0.0);
  for (int q = 0; q < nw; ++q) t = t + sc[q];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kEv3Threads) k_eval_pillar(Ev3Args a, const uint8_t* __restrict__ state,
                                                             int dir_mask, int aligned, int64_t ncand,
                                                             double* __restrict__ dfom) {
  extern __shared__ __align__(16) unsigned char ev3_smem[];
  cplx* A = reinterpret_cast<cplx*>(ev3_smem);                   // p x p, row-major
  __shared__ cplx y[kEv3MaxP];
  __shared__ int32_t V[kEv3MaxP];
  __shared__ double D[kEv3MaxP];
  __shared__ int s_p;
  __shared__ double s_v[kEv3Threads / 32];
  __shared__ int s_i[kEv3Threads / 32];
  __shared__ cplx s_c[kEv3Threads / 32];
  __shared__ int s_bad;
  const Geo3& g = a.g;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int64_t c = blockIdx.x; c < ncand; c += gridDim.x) {
    if (tid == 0) {
      const int64_t an = c % ((int64_t)(g.nx - 1) * (g.ny - 1));
      const int ay = (int)(an / (g.nx - 1)), ax = (int)(an - (int64_t)ay * (g.nx - 1));
      s_p = (aligned && ((ax | ay) & 1)) ? 0
                                         : cand_pixels(c, GF_KIND_PILLAR, dir_mask, g.nx, g.ny, g.chi, state, V, D, g.nz);
      s_bad = 0;
    }
    __syncthreads();
    const int p = s_p;
    if (p == 0) {
      if (tid == 0) dfom[c] = -INFINITY;
      __syncthreads();
      continue;
    }
    for (int t = tid; t < p * p; t += nt) {
      const int r = t / p, q = t - r * p;
      const cplx gv = ldG(a.G, a.dtype, a.ldg, V[r], V[q]);
      A[t] = mk(r == q ? 1.0 : 0.0, 0.0) - D[q] * gv;
    }
    for (int t = tid; t < p; t += nt) y[t] = a.E[V[t]];
    __syncthreads();
    double rs = 0.0;
    for (int r = tid; r < p; r += nt) {
      double s = 0.0;
      for (int q = 0; q < p; ++q) s += cabs1(A[r * p + q]);
      rs = fmax(rs, s);
    }
    int dummy = 0;
    block_argmax(rs, dummy, s_v, s_i);
    const double thresh = kSingularRel * rs;
    // LU with partial pivoting (largest modulus, lowest row on ties), y eliminated alongside
    for (int cc = 0; cc < p; ++cc) {
      double bv = -1.0;
      int br = 0x7fffffff;
      for (int r = cc + tid; r < p; r += nt) {
        const double m = cabs1(A[r * p + cc]);
        if (m > bv) { bv = m; br = r; }
      }
      block_argmax(bv, br, s_v, s_i);
      if (!(bv >= thresh) || !(bv > 0.0)) {
        if (tid == 0) s_bad = 1;
        break;
      }
      if (br != cc) {
        for (int q = tid; q < p; q += nt) {
          const cplx t0 = A[cc * p + q];
          A[cc * p + q] = A[br * p + q];
          A[br * p + q] = t0;
        }
        if (tid == 0) { const cplx t0 = y[cc]; y[cc] = y[br]; y[br] = t0; }
      }
      __syncthreads();
      const cplx pv = A[cc * p + cc];
      const int w = p - cc - 1;
      for (int r = cc + 1 + tid; r < p; r += nt) A[r * p + cc] = cdiv(A[r * p + cc], pv);
      __syncthreads();
      for (int e = tid; e < w * w; e += nt) {
        const int r = cc + 1 + e / w, q = cc + 1 + e % w;
        A[r * p + q] = A[r * p + q] - A[r * p + cc] * A[cc * p + q];
      }
      if (tid == 0)
        for (int r = cc + 1; r < p; ++r) y[r] = y[r] - A[r * p + cc] * y[cc];
      __syncthreads();
    }
    __syncthreads();
    if (s_bad) {
      if (tid == 0) dfom[c] = -INFINITY;
      __syncthreads();
      continue;
    }
    for (int cc = p - 1; cc >= 0; --cc) {            // upper solve, column-oriented
      if (tid == 0) y[cc] = cdiv(y[cc], A[cc * p + cc]);
      __syncthreads();
      const cplx yc = y[cc];
      for (int r = tid; r < cc; r += nt) y[r] = y[r] - A[r * p + cc] * yc;
      __syncthreads();
    }
    double df = 0.0;
    for (int mc = 0; mc < 3; ++mc) {                 // Eq. 4 at the monitor, |E|^2 over components
      const int64_t m = 3 * g.N + mc;
      cplx part = mk(0.0, 0.0);
      for (int u = tid; u < p; u += nt) part = part + D[u] * (ldG(a.G, a.dtype, a.ldg, m, V[u]) * y[u]);
      const cplx dE = block_sum(part, s_c);
      const cplx Em = a.E[m];
      df += abs2(Em + dE) - abs2(Em);
    }
    if (tid == 0) dfom[c] = df;
    __syncthreads();
  }
}

// ---- dFOM of every pillar for complex64 G --------------------------------------------------
// The stored G is FP32, so the p x p system of Eqs. 6-9 is factorised in FP32 (LU with partial
// pivoting, largest modulus, lowest row on ties) and the solution is refined once with the
// residual b - A y formed in FP64 from the stored entries (classical iterative refinement):
// y then has the accuracy of an FP64 solve of the same system, at the FP32 rate for the O(p^3)
// part.  Eq. 4 at the monitor in FP64.  Singular: a pivot below kSingularRel of the largest row
// sum, or a refinement correction above 2^-10 of the solution (the FP32 factors do not resolve
// the system: condition number around 10^4 or more).  Shared memory: the factors, row stride
// p + 1 (column walks free of bank conflicts).
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 crecipf(float2 b) {
  const float s = 1.0f / fmaf(b.x, b.x, b.y * b.y);
  return make_float2(b.x * s, -b.y * s);
}

// block-wide (max value, lowest index on ties) in FP32 (the pivot search of the FP32 factors)
__device__ __forceinline__ void block_argmax_f(float& v, int& idx, float* sv, int* si) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_down_sync(0xffffffffu, v, o);
    const int oi = __shfl_down_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if (lane == 0) { sv[w] = v; si[w] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < nw; ++q)
      if (sv[q] > sv[0] || (sv[q] == sv[0] && si[q] < si[0])) { sv[0] = sv[q]; si[0] = si[q]; }
  }
  __syncthreads();
  v = sv[0];
  idx = si[0];
  __syncthreads();
}

// w <- U^{-1} L^{-1} P w for the factors in A (row stride lda, unit lower L below the
// diagonal, row interchanges piv); one warp, row-oriented dot products
__device__ __forceinline__ void lu32_solve_warp(const float2* A, int lda, const int* piv, int p, float2* w) {
  const int lane = threadIdx.x & 31;
  if (lane == 0)
    for (int c = 0; c < p; ++c) {
      const int r = piv[c];
      if (r != c) { const float2 t = w[c]; w[c] = w[r]; w[r] = t; }
    }
  __syncwarp();
  for (int r = 1; r < p; ++r) {
    float sx = 0.f, sy = 0.f;
    for (int q = lane; q < r; q += 32) {
      const float2 t = cmulf(A[r * lda + q], w[q]);
      sx += t.x;
      sy += t.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) w[r] = make_float2(w[r].x - sx, w[r].y - sy);
    __syncwarp();
  }
  for (int r = p - 1; r >= 0; --r) {
    float sx = 0.f, sy = 0.f;
    for (int q = r + 1 + lane; q < p; q += 32) {
      const float2 t = cmulf(A[r * lda + q], w[q]);
      sx += t.x;
      sy += t.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) w[r] = cmulf(make_float2(w[r].x - sx, w[r].y - sy), crecipf(A[r * lda + r]));
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kEv3Threads) k_eval_pillar_f32(Ev3Args a, const uint8_t* __restrict__ state,
                                                                 int dir_mask, int aligned, int64_t ncand,
                                                                 double* __restrict__ dfom) {
  extern __shared__ __align__(16) unsigned char ev3_smem[];
  float2* A = reinterpret_cast<float2*>(ev3_smem);              // p x p, row stride p + 1
  __shared__ cplx b[kEv3MaxP], y[kEv3MaxP], rv[kEv3MaxP];
  __shared__ float2 w[kEv3MaxP];
  __shared__ int32_t V[kEv3MaxP];
  __shared__ int piv[kEv3MaxP];
  __shared__ double D[kEv3MaxP];
  __shared__ int s_p;
  __shared__ float s_v[kEv3Threads / 32];
  __shared__ int s_i[kEv3Threads / 32];
  __shared__ cplx s_c[kEv3Threads / 32];
  __shared__ int s_bad;
  const Geo3& g = a.g;
  const float2* G = reinterpret_cast<const float2*>(a.G);
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int64_t c = blockIdx.x; c < ncand; c += gridDim.x) {
    if (tid == 0) {
      const int64_t an = c % ((int64_t)(g.nx - 1) * (g.ny - 1));
      const int ay = (int)(an / (g.nx - 1)), ax = (int)(an - (int64_t)ay * (g.nx - 1));
      s_p = (aligned && ((ax | ay) & 1)) ? 0
                                         : cand_pixels(c, GF_KIND_PILLAR, dir_mask, g.nx, g.ny, g.chi, state, V, D, g.nz);
      s_bad = 0;
    }
    __syncthreads();
    const int p = s_p, lda = p + 1;
    if (p == 0) {
      if (tid == 0) dfom[c] = -INFINITY;
      __syncthreads();
      continue;
    }
    // A = I - G_VV D in FP32 (only the factors use it; the refinement residual below forms
    // its entries again in FP64)
    for (int r = warp; r < p; r += nw) {
      const float2* Grow = G + (int64_t)V[r] * a.ldg;
      for (int q = lane; q < p; q += 32) {
        const float2 gv = Grow[V[q]];
        const float dq = (float)D[q];
        A[r * lda + q] = make_float2(fmaf(-dq, gv.x, r == q ? 1.f : 0.f), -dq * gv.y);
      }
    }
    for (int t = tid; t < p; t += nt) b[t] = a.E[V[t]];
    __syncthreads();
    float rs = 0.f;
    for (int r = tid; r < p; r += nt) {
      float s = 0.f;
      for (int q = 0; q < p; ++q) {
        const float2 e = A[r * lda + q];
        s += sqrtf(fmaf(e.x, e.x, e.y * e.y));
      }
      rs = fmaxf(rs, s);
    }
    int dummy = 0;
    block_argmax_f(rs, dummy, s_v, s_i);
    const float thresh = (float)kSingularRel * rs;
    for (int cc = 0; cc < p; ++cc) {
      float bv = -1.f;
      int br = 0x7fffffff;
      for (int r = cc + tid; r < p; r += nt) {
        const float2 e = A[r * lda + cc];
        const float m = sqrtf(fmaf(e.x, e.x, e.y * e.y));
        if (m > bv) { bv = m; br = r; }
      }
      block_argmax_f(bv, br, s_v, s_i);
      if (!(bv >= thresh) || !(bv > 0.f)) {
        if (tid == 0) s_bad = 1;
        break;
      }
      if (tid == 0) piv[cc] = br;
      if (br != cc)
        for (int q = tid; q < p; q += nt) {
          const float2 t0 = A[cc * lda + q];
          A[cc * lda + q] = A[br * lda + q];
          A[br * lda + q] = t0;
        }
      __syncthreads();
      const float2 rp = crecipf(A[cc * lda + cc]);
      for (int r = cc + 1 + tid; r < p; r += nt) A[r * lda + cc] = cmulf(A[r * lda + cc], rp);
      __syncthreads();
      // trailing update: warps over rows, lanes over columns (the pivot row's entries in registers)
      float2 u[kEv3MaxP / 32];
#pragma unroll
      for (int j = 0; j < kEv3MaxP / 32; ++j) {
        const int q = cc + 1 + lane + 32 * j;
        u[j] = q < p ? A[cc * lda + q] : make_float2(0.f, 0.f);
      }
      for (int r = cc + 1 + warp; r < p; r += nw) {
        const float2 l = A[r * lda + cc];
#pragma unroll
        for (int j = 0; j < kEv3MaxP / 32; ++j) {
          const int q = cc + 1 + lane + 32 * j;
          if (q < p) {
            float2 e = A[r * lda + q];
            e.x = fmaf(-l.x, u[j].x, fmaf(l.y, u[j].y, e.x));
            e.y = fmaf(-l.x, u[j].y, fmaf(-l.y, u[j].x, e.y));
            A[r * lda + q] = e;
          }
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (s_bad) {
      if (tid == 0) dfom[c] = -INFINITY;
      __syncthreads();
      continue;
    }
    // y0 = A^{-1} b with the FP32 factors
    if (warp == 0) {
      for (int t = lane; t < p; t += 32) w[t] = make_float2((float)b[t].re, (float)b[t].im);
      __syncwarp();
      lu32_solve_warp(A, lda, piv, p, w);
      for (int t = lane; t < p; t += 32) y[t] = mk((double)w[t].x, (double)w[t].y);
    }
    __syncthreads();
    // refinement: rv = b - A y in FP64 (A y = y - G_VV D y), then y += A^{-1} rv
    for (int r = warp; r < p; r += nw) {
      const float2* Grow = G + (int64_t)V[r] * a.ldg;
      double sx = 0.0, sy = 0.0;
      for (int q = lane; q < p; q += 32) {
        const float2 gv = Grow[V[q]];
        const double gx = D[q] * (double)gv.x, gy = D[q] * (double)gv.y;
        sx = fma(gx, y[q].re, fma(-gy, y[q].im, sx));
        sy = fma(gx, y[q].im, fma(gy, y[q].re, sy));
      }
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
      }
      if (lane == 0) rv[r] = mk(b[r].re - y[r].re + sx, b[r].im - y[r].im + sy);
    }
    __syncthreads();
    if (warp == 0) {
      for (int t = lane; t < p; t += 32) w[t] = make_float2((float)rv[t].re, (float)rv[t].im);
      __syncwarp();
      lu32_solve_warp(A, lda, piv, p, w);
      double dmax = 0.0, ymax = 0.0;
      for (int t = lane; t < p; t += 32) {
        const cplx yn = mk(y[t].re + (double)w[t].x, y[t].im + (double)w[t].y);
        y[t] = yn;
        dmax = fmax(dmax, fmax(fabs((double)w[t].x), fabs((double)w[t].y)));
        ymax = fmax(ymax, fmax(fabs(yn.re), fabs(yn.im)));
      }
      for (int o = 16; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        ymax = fmax(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
      }
      if (lane == 0 && !(dmax <= 0x1p-10 * ymax)) s_bad = 1;
    }
    __syncthreads();
    if (s_bad) {
      if (tid == 0) dfom[c] = -INFINITY;
      __syncthreads();
      continue;
    }
    double df = 0.0;
    for (int mc = 0; mc < 3; ++mc) {                 // Eq. 4 at the monitor, |E|^2 over components
      const int64_t m = 3 * g.N + mc;
      cplx part = mk(0.0, 0.0);
      for (int u = tid; u < p; u += nt) part = part + D[u] * (ldG(a.G, a.dtype, a.ldg, m, V[u]) * y[u]);
      const cplx dE = block_sum(part, s_c);
      const cplx Em = a.E[m];
      df += abs2(Em + dE) - abs2(Em);
    }
    if (tid == 0) dfom[c] = df;
    __syncthreads();
  }
}

static gf_status check3(gf_handle* h, const gf_geom3d* g) {
  if (!g) return api_fail_msg(h, GF_EINVAL, "geometry is NULL");
  if (g->nx < 2 || g->ny < 2 || g->nz < 1 || g->nz > 8)
    return api_fail_msg(h, GF_EINVAL, "3-D geometry needs nx, ny >= 2 and 1 <= nz <= 8");
  const int64_t n = 3 * ((int64_t)g->nx * g->ny * g->nz + 1);
  if (n > (int64_t)INT32_MAX) return api_fail_msg(h, GF_EINVAL, "3 (N + 1) exceeds int32");
  if (!(g->dx > 0.0) || !isfinite(g->dx) || !(g->wavelength > 0.0) || !isfinite(g->wavelength))
    return api_fail_msg(h, GF_EINVAL, "dx and wavelength must be positive and finite");
  if (g->eps_bg != 1.0) return api_fail_msg(h, GF_EINVAL, "eps_bg must be 1 (vacuum background G0)");
  if (!isfinite(g->eps_mat) || g->eps_mat == g->eps_bg) return api_fail_msg(h, GF_EINVAL, "eps_mat must differ from eps_bg");
  const double X = g->nx * g->dx, Y = g->ny * g->dx, Z = g->nz * g->dx;
  if (!isfinite(g->mon_x) || !isfinite(g->mon_y) || !isfinite(g->mon_z))
    return api_fail_msg(h, GF_EINVAL, "monitor position not finite");
  if (g->mon_x >= 0.0 && g->mon_x <= X && g->mon_y >= 0.0 && g->mon_y <= Y && g->mon_z >= 0.0 && g->mon_z <= Z)
    return api_fail_msg(h, GF_EINVAL, "the monitor lies inside the design slab");
  return GF_OK;
}

static gf_status check3_spec(gf_handle* h, const gf_geom3d* g, const gf_cand_spec* s) {
  if (!s) return api_fail_msg(h, GF_EINVAL, "candidate spec is NULL");
  if (s->kind != GF_KIND_PILLAR) return api_fail_msg(h, GF_EINVAL, "3-D problems take GF_KIND_PILLAR candidates");
  if (s->dir_mask < 1 || s->dir_mask > 3) return api_fail_msg(h, GF_EINVAL, "dir_mask must be 1, 2 or 3");
  if (s->k < 1 || 12 * g->nz * s->k > 1024) return api_fail_msg(h, GF_EINVAL, "k must keep 12 nz k <= 1024");
  if (s->excl_radius < 0 || !(s->tie_rel >= 0.0)) return api_fail_msg(h, GF_EINVAL, "bad exclusion radius or tie_rel");
  return GF_OK;
}

static gf_status check3_problem(gf_handle* h, const gf_problem3d* p, int dtype) {
  if (!p) return api_fail_msg(h, GF_EINVAL, "problem is NULL");
  gf_status s = check3(h, &p->geom);
  if (s) return s;
  if (dtype != GF_C128 && dtype != GF_C64) return api_fail_msg(h, GF_EINVAL, "unknown dtype");
  const int64_t n = 3 * ((int64_t)p->geom.nx * p->geom.ny * p->geom.nz + 1);
  if (!p->G || !p->E || ((uintptr_t)p->G & 15u) || ((uintptr_t)p->E & 15u))
    return api_fail_msg(h, GF_EINVAL, "G and E must be non-NULL and 16-byte aligned");
  if (p->ldg < n || (p->ldg & 1)) return api_fail_msg(h, GF_EINVAL, "ldg must be even and >= n");
  return GF_OK;
}

static WsLayout ws3(const gf_geom3d& g, int dtype, const gf_cand_spec& spec) {
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  return ws_layout_n(3 * (N + 1), 3 * N, 12 * g.nz * (spec.k < 1 ? 1 : spec.k), 1, dtype);
}

}  // namespace gf

extern "C" {

int64_t gf3_num_unknowns(const gf_geom3d* g) {
  if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1) return 0;
  return 3 * ((int64_t)g->nx * g->ny * g->nz + 1);
}

int64_t gf3_num_candidates(const gf_geom3d* g) {
  if (!g || g->nx < 2 || g->ny < 2) return 0;
  return 2 * (int64_t)(g->nx - 1) * (g->ny - 1);
}

size_t gf3_workspace_size(const gf_geom3d* g, int32_t dtype, const gf_cand_spec* s) {
  if (!g || !s || g->nx < 2 || g->ny < 2 || g->nz < 1 || g->nz > 8) return 0;
  if (dtype != GF_C128 && dtype != GF_C64) return 0;
  return gf::ws3(*g, dtype, *s).total;
}

gf_status gf3_fill_g0(gf_handle* h, const gf_problem3d* prob, int32_t dtype, void* ws, size_t ws_bytes, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = gf::check3_problem(h, prob, dtype);
  if (s) return s;
  const gf::Geo3 g = gf::geo3(prob->geom);
  if (!ws || ((uintptr_t)ws & 255u)) return gf::api_fail_msg(h, GF_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < sizeof(gf::cplx) * (size_t)(3 * g.N)) return gf::api_fail_msg(h, GF_ENOMEM, "workspace too small for the fill table");
  if ((s = gf::api_bind_device(h))) return s;
  cudaStream_t st = (cudaStream_t)stream;
  gf::cplx* table = reinterpret_cast<gf::cplx*>(ws);
  float4* table32 = reinterpret_cast<float4*>(table + 2 * g.N);
  int64_t b = (g.N + 255) / 256;
  gf::k_fill3_table<<<(int)(b < 4864 ? b : 4864), 256, 0, st>>>(g, table, table32);
  const int rows = (int)(3 * g.N < 152 * 16 ? 3 * g.N : 152 * 16);
  if (dtype == GF_C128) {
    gf::k_fill3_expand<double2><<<rows, 256, 0, st>>>(g, prob->ldg, table, reinterpret_cast<double2*>(prob->G));
    gf::k_fill3_monitor<double2><<<(int)(b < 4864 ? b + 1 : 4864), 256, 0, st>>>(g, prob->ldg, reinterpret_cast<double2*>(prob->G),
                                                                                 reinterpret_cast<gf::cplx*>(prob->E));
  } else {
    gf::k_fill3_expand_f32<<<rows, 256, 0, st>>>(g, prob->ldg, table32, reinterpret_cast<float2*>(prob->G));
    gf::k_fill3_monitor<float2><<<(int)(b < 4864 ? b + 1 : 4864), 256, 0, st>>>(g, prob->ldg, reinterpret_cast<float2*>(prob->G),
                                                                                reinterpret_cast<gf::cplx*>(prob->E));
  }
  return gf::api_cuda_check(h, "gf3_fill_g0 launch");
}

gf_status gf3_fom(gf_handle* h, const gf_problem3d* prob, int32_t dtype, double* fom_out, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = gf::check3_problem(h, prob, dtype);
  if (s) return s;
  if (!fom_out) return gf::api_fail_msg(h, GF_EINVAL, "fom_out must be non-NULL");
  if ((s = gf::api_bind_device(h))) return s;
  gf::FomArgs a;
  a.nlam = 1;
  a.ncomp = 3;
  a.mrow = 3 * (int64_t)prob->geom.nx * prob->geom.ny * prob->geom.nz;
  a.E[0] = reinterpret_cast<const gf::cplx*>(prob->E);
  gf::launch_fom(a, fom_out, (cudaStream_t)stream);
  return gf::api_cuda_check(h, "gf3_fom launch");
}

gf_status gf3_eval_candidates(gf_handle* h, const gf_problem3d* prob, int32_t dtype, const uint8_t* state,
                              const gf_cand_spec* spec, double* dfom, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = gf::check3_problem(h, prob, dtype);
  if (s) return s;
  if ((s = gf::check3_spec(h, &prob->geom, spec))) return s;
  if (!state || !dfom) return gf::api_fail_msg(h, GF_EINVAL, "state and dfom must be non-NULL");
  if ((s = gf::api_bind_device(h))) return s;
  gf::Ev3Args a;
  a.g = gf::geo3(prob->geom);
  a.dtype = dtype;
  a.G = prob->G;
  a.ldg = prob->ldg;
  a.E = reinterpret_cast<const gf::cplx*>(prob->E);
  const int p = 12 * prob->geom.nz;
  const bool f32 = dtype == GF_C64 && gf::api_update_algo(h) != GF_UPDATE_DFMA;
  const size_t smem = f32 ? sizeof(float2) * (size_t)p * (p + 1) : sizeof(gf::cplx) * (size_t)p * p;
  {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || !done[dev]) {
      cudaFuncSetAttribute(gf::k_eval_pillar, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(gf::cplx) * gf::kEv3MaxP * gf::kEv3MaxP));
      cudaFuncSetAttribute(gf::k_eval_pillar_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(float2) * gf::kEv3MaxP * (gf::kEv3MaxP + 1)));
      if (dev >= 0 && dev < 64) done[dev] = true;
    }
  }
  const int64_t ncand = gf3_num_candidates(&prob->geom);
  int per_sm = 8;
  if (f32 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gf::k_eval_pillar_f32, gf::kEv3Threads, smem) !=
                  cudaSuccess ||
              per_sm < 1)) {
    cudaGetLastError();
    per_sm = 4;
  }
  const int64_t cap = (int64_t)gf::api_sm_count(h) * per_sm;
  const int grid = (int)(ncand < cap ? ncand : cap);
  if (f32)
    gf::k_eval_pillar_f32<<<grid, gf::kEv3Threads, smem, (cudaStream_t)stream>>>(a, state, spec->dir_mask,
                                                                                 spec->aligned, ncand, dfom);
  else
    gf::k_eval_pillar<<<grid, gf::kEv3Threads, smem, (cudaStream_t)stream>>>(a, state, spec->dir_mask, spec->aligned,
                                                                             ncand, dfom);
  return gf::api_cuda_check(h, "gf3_eval_candidates launch");
}

gf_status gf3_select_topk(gf_handle* h, const gf_geom3d* geom, const gf_cand_spec* spec, const double* dfom,
                          int64_t ncand, int32_t* idx, double* val, int32_t* status, void* ws, size_t ws_bytes,
                          void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = gf::check3(h, geom);
  if (s) return s;
  if ((s = gf::check3_spec(h, geom, spec))) return s;
  if (ncand != gf3_num_candidates(geom)) return gf::api_fail_msg(h, GF_EINVAL, "ncand does not match the pillar family");
  if (!dfom || !idx || !val || !status) return gf::api_fail_msg(h, GF_EINVAL, "dfom, idx, val and status must be non-NULL");
  if ((s = gf::api_bind_device(h))) return s;
  // pillars share the 2-D brushes' id layout and anchors
  gf_geom g2 = {};
  g2.nx = geom->nx;
  g2.ny = geom->ny;
  void* sel = nullptr;
  if (ws && spec->k > 1) {
    const gf::WsLayout L = gf::ws3(*geom, GF_C128, *spec);
    if (((uintptr_t)ws & 255u) == 0 && ws_bytes >= L.sel + gf::topk_scratch_bytes()) sel = (char*)ws + L.sel;
  }
  gf::launch_select(g2, *spec, dfom, ncand, idx, val, status, sel, (cudaStream_t)stream);
  return gf::api_cuda_check(h, "gf3_select_topk launch");
}

gf_status gf3_apply_update(gf_handle* h, const gf_problem3d* prob, int32_t dtype, uint8_t* state,
                           const gf_cand_spec* spec, const int32_t* idx, int32_t* status, double* fom_out,
                           int32_t* applied, void* ws, size_t ws_bytes, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = gf::check3_problem(h, prob, dtype);
  if (s) return s;
  if ((s = gf::check3_spec(h, &prob->geom, spec))) return s;
  if (!state || !idx || !status || !fom_out) return gf::api_fail_msg(h, GF_EINVAL, "state, idx, status and fom_out must be non-NULL");
  const gf::WsLayout L = gf::ws3(prob->geom, dtype, *spec);
  if (!ws || ((uintptr_t)ws & 255u)) return gf::api_fail_msg(h, GF_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < L.total) return gf::api_fail_msg(h, GF_ENOMEM, "workspace too small");
  if ((s = gf::api_bind_device(h))) return s;
  const gf::Geo3 g = gf::geo3(prob->geom);
  gf::UpdArgs a;
  a.nlam = 1;
  a.dtype = dtype;
  a.nx = prob->geom.nx;
  a.ny = prob->geom.ny;
  a.chi = g.chi;
  a.pmax = L.pmax;
  a.algo = gf::api_update_algo(h);
  a.sm_count = gf::api_sm_count(h);
  a.nz = prob->geom.nz;
  a.ncomp = 3;
  a.mrow = 3 * g.N;
  a.mcount = 3;
  a.lam[0].G = prob->G;
  a.lam[0].ldg = prob->ldg;
  a.lam[0].E = reinterpret_cast<gf::cplx*>(prob->E);
  a.lam[0].bands = nullptr;
  a.lam[0].vrows = nullptr;
  a.lam[0].ldv = 0;
  a.lam[0].rows = 3 * (g.N + 1);
  gf::launch_update(a, L, reinterpret_cast<char*>(ws), state, *spec, idx, status, fom_out, applied,
                    (cudaStream_t)stream, gf::api_timer(h));
  return gf::api_cuda_check(h, "gf3_apply_update launch");
}

}  // extern "C"
