// Background Green's matrix G0 of a vacuum design region (Sec. II-B / Sec. IV: the initial
// Green's function of a vacuum background is known analytically), incident field, and the
// neighbour bands that candidate evaluation gathers (the G_VV blocks of Eq. 8).
//
// G0 depends on the pixel offset (|dix|, |diy|) only, so the Hankel functions are evaluated
// once per offset into a table of nx*ny values (plus N monitor values) and the n x n matrix
// is written by an expansion kernel that is bound by HBM write bandwidth.
#include <math.h>

#include "gf_internal.cuh"
#include "gf_stage_bodies.cuh"

namespace gf {

// (i/4) k^2 dx^2 H0(k r) = (k^2 dx^2 / 4) (i J0 - Y0)
__device__ __forceinline__ cplx g0_offdiag(double k, double dx, double r) {
  double c = 0.25 * k * k * dx * dx;
  double x = k * r;
  return {-c * y0(x), c * j0(x)};
}

// (i pi/2) k a H1(k a) - 1 with a = dx/sqrt(pi): k^2 times the integral of (i/4) H0(k r)
// over a disk with the pixel's area.
__device__ __forceinline__ cplx g0_self(double k, double dx) {
  double a = dx * 0.56418958354775628695;   // 1/sqrt(pi)
  double x = k * a;
  double c = 0.5 * M_PI * x;
  return {-c * y1(x) - 1.0, c * j1(x)};
}

__global__ void k_fill_table(int nx, int ny, double dx, double k, double mx, double my,
                             cplx* __restrict__ table) {
  const int64_t ntab = (int64_t)nx * ny;
  const int64_t N = ntab;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntab + N;
       t += (int64_t)gridDim.x * blockDim.x) {
    cplx v;
    if (t < ntab) {
      int ddy = (int)(t / nx), ddx = (int)(t % nx);
      if (ddx == 0 && ddy == 0) {
        v = g0_self(k, dx);
      } else {
        double r = dx * sqrt((double)ddx * ddx + (double)ddy * ddy);
        v = g0_offdiag(k, dx, r);
      }
    } else {
      int64_t j = t - ntab;
      int iy = (int)(j / nx), ix = (int)(j % nx);
      double px = (ix + 0.5) * dx - mx, py = (iy + 0.5) * dx - my;
      v = g0_offdiag(k, dx, sqrt(px * px + py * py));
    }
    table[t] = v;
  }
}

template <typename T>
__device__ __forceinline__ void st_entry(void* G, int64_t off, cplx v);
template <>
__device__ __forceinline__ void st_entry<double2>(void* G, int64_t off, cplx v) {
  reinterpret_cast<double2*>(G)[off] = make_double2(v.re, v.im);
}
template <>
__device__ __forceinline__ void st_entry<float2>(void* G, int64_t off, cplx v) {
  reinterpret_cast<float2*>(G)[off] = make_float2((float)v.re, (float)v.im);
}

// One block per row (grid-stride over rows); threads sweep the row's ldg columns.
template <typename T>
__global__ void k_fill_expand(int nx, int ny, int64_t ldg, const cplx* __restrict__ table,
                              void* __restrict__ G) {
  const int64_t N = (int64_t)nx * ny;
  const cplx* mon = table + N;
  for (int64_t i = blockIdx.x; i <= N; i += gridDim.x) {
    const int64_t row = i * ldg;
    if (i < N) {
      const int iy = (int)(i / nx), ix = (int)(i % nx);
      for (int64_t j = threadIdx.x; j < ldg; j += blockDim.x) {
        cplx v;
        if (j < N) {
          int jy = (int)(j / nx), jx = (int)(j - (int64_t)jy * nx);
          int ay = iy > jy ? iy - jy : jy - iy;
          int ax = ix > jx ? ix - jx : jx - ix;
          v = table[(int64_t)ay * nx + ax];
        } else if (j == N) {
          v = mon[i];
        } else {
          v = mk(0.0, 0.0);
        }
        st_entry<T>(G, row + j, v);
      }
    } else {
      for (int64_t j = threadIdx.x; j < ldg; j += blockDim.x) {
        cplx v = j < N ? mon[j] : mk(0.0, 0.0);
        st_entry<T>(G, row + j, v);
      }
    }
  }
}

// Pixel-row-pair blocks: for image rows (iy, jy) the nx x nx sub-block G[iy*nx + ix, jy*nx + jx]
// equals table row |iy - jy| at offset |ix - jx| (G0 depends on the offset only).  One CTA stages
// that table row in shared memory (in the storage precision) and writes the sub-block row by
// row with coalesced stores, so the table is read nx times less often than per entry and the
// fill is bound by the stores.  The monitor row and column and the padding columns follow in
// k_fill_edges.  Used for nx <= kFillMaxNx.
constexpr int kFillMaxNx = 2048;

template <typename T>
__device__ __forceinline__ T to_store(cplx v);
template <>
__device__ __forceinline__ double2 to_store<double2>(cplx v) { return make_double2(v.re, v.im); }
template <>
__device__ __forceinline__ float2 to_store<float2>(cplx v) { return make_float2((float)v.re, (float)v.im); }

template <typename T>
__global__ void __launch_bounds__(256) k_fill_blocks(int nx, int ny, int64_t ldg, const cplx* __restrict__ table,
                                                     T* __restrict__ G) {
  extern __shared__ __align__(16) unsigned char fill_smem[];
  T* trow = reinterpret_cast<T*>(fill_smem);
  const int64_t pairs = (int64_t)ny * ny;
  for (int64_t q = blockIdx.x; q < pairs; q += gridDim.x) {
    const int iy = (int)(q / ny), jy = (int)(q - (int64_t)iy * ny);
    const int ay = iy > jy ? iy - jy : jy - iy;
    __syncthreads();                               // previous pair done with trow
    for (int x = threadIdx.x; x < nx; x += blockDim.x) trow[x] = to_store<T>(table[(int64_t)ay * nx + x]);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    for (int ix = warp; ix < nx; ix += nwarp) {          // a warp per row, lanes along it
      T* row = G + ((int64_t)iy * nx + ix) * ldg + (int64_t)jy * nx;
      for (int jx = lane; jx < nx; jx += 32) row[jx] = trow[ix > jx ? ix - jx : jx - ix];
    }
  }
}

// monitor column (rows 0..N-1), monitor row (G_NN = 0) and padding columns (zero)
template <typename T>
__global__ void k_fill_edges(int nx, int ny, int64_t ldg, const cplx* __restrict__ table, T* __restrict__ G) {
  const int64_t N = (int64_t)nx * ny;
  const cplx* mon = table + N;
  const int64_t pad = ldg - N;                     // columns N .. ldg-1 of every row
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N * pad; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / pad, c = t - i * pad;
    G[i * ldg + N + c] = to_store<T>(c == 0 ? mon[i] : mk(0.0, 0.0));
  }
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ldg; j += (int64_t)gridDim.x * blockDim.x)
    G[N * ldg + j] = to_store<T>(j < N ? mon[j] : mk(0.0, 0.0));
}

__global__ void k_fill_field(int nx, int ny, double dx, double k, double my, cplx* __restrict__ E) {
  const int64_t N = (int64_t)nx * ny;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= N;
       j += (int64_t)gridDim.x * blockDim.x) {
    double y = j < N ? ((double)(j / nx) + 0.5) * dx : my;
    double s, c;
    sincos(k * y, &s, &c);
    E[j] = mk(c, s);
  }
}

__global__ void k_bands(int nx, int ny, int dtype, const void* __restrict__ G, int64_t ldg,
                        cplx* __restrict__ bands) {
  bands_body(nx, ny, dtype, G, ldg, bands);
}

// Batched band extraction: blockIdx.y selects the problem of the device table.
__global__ void k_bands_batch(const BatchItem* __restrict__ items, int dtype) {
  const BatchItem& it = items[blockIdx.y];
  bands_body(it.nx, it.ny, dtype, it.G, it.ldg, it.bands);
}

void launch_bands_batch(const BatchItem* items, int nprob, int dtype, int64_t widest, cudaStream_t st) {
  int64_t b = (widest + 255) / 256;                  // widest: pixels of the largest problem
  if (b > 1216) b = 1216;
  k_bands_batch<<<dim3((unsigned)(b < 1 ? 1 : b), (unsigned)nprob), 256, 0, st>>>(items, dtype);
}

static int grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

void launch_fill_table(const gf_geom& g, cplx* table, cudaStream_t st) {
  const int64_t N = (int64_t)g.nx * g.ny;
  const double k = 2.0 * M_PI / g.wavelength;
  k_fill_table<<<grid_for(2 * N, 256), 256, 0, st>>>(g.nx, g.ny, g.dx, k, g.mon_x, g.mon_y, table);
}

void launch_fill_expand(const gf_geom& g, int dtype, void* G, int64_t ldg, const cplx* table,
                        cplx* E, cudaStream_t st) {
  const int64_t N = (int64_t)g.nx * g.ny;
  const double k = 2.0 * M_PI / g.wavelength;
  int blocks = (int)(N + 1 < 152 * 16 ? N + 1 : 152 * 16);
  if (g.nx <= kFillMaxNx) {
    const int64_t pairs = (int64_t)g.ny * g.ny;
    const int fb = (int)(pairs < 152 * 8 ? pairs : 152 * 8);
    const int eb = grid_for(N + 1, 256);
    if (dtype == GF_C128) {
      k_fill_blocks<double2><<<fb, 256, (size_t)g.nx * sizeof(double2), st>>>(g.nx, g.ny, ldg, table,
                                                                              reinterpret_cast<double2*>(G));
      k_fill_edges<double2><<<eb, 256, 0, st>>>(g.nx, g.ny, ldg, table, reinterpret_cast<double2*>(G));
    } else {
      k_fill_blocks<float2><<<fb, 256, (size_t)g.nx * sizeof(float2), st>>>(g.nx, g.ny, ldg, table,
                                                                            reinterpret_cast<float2*>(G));
      k_fill_edges<float2><<<eb, 256, 0, st>>>(g.nx, g.ny, ldg, table, reinterpret_cast<float2*>(G));
    }
  } else if (dtype == GF_C128) {
    k_fill_expand<double2><<<blocks, 256, 0, st>>>(g.nx, g.ny, ldg, table, G);
  } else {
    k_fill_expand<float2><<<blocks, 256, 0, st>>>(g.nx, g.ny, ldg, table, G);
  }
  k_fill_field<<<grid_for(N + 1, 256), 256, 0, st>>>(g.nx, g.ny, g.dx, k, g.mon_y, E);
}

void launch_fill_field(const gf_geom& g, cplx* E, cudaStream_t st) {
  const int64_t N = (int64_t)g.nx * g.ny;
  const double k = 2.0 * M_PI / g.wavelength;
  k_fill_field<<<grid_for(N + 1, 256), 256, 0, st>>>(g.nx, g.ny, g.dx, k, g.mon_y, E);
}

void launch_bands(const gf_geom& g, int dtype, const void* G, int64_t ldg, cplx* bands,
                  cudaStream_t st) {
  const int64_t N = (int64_t)g.nx * g.ny;
  k_bands<<<grid_for(N, 256), 256, 0, st>>>(g.nx, g.ny, dtype, G, ldg, bands);
}

}  // namespace gf
