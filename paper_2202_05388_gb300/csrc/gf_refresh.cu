// Drift refresh: checks of the accumulated state against the discrete Lippmann-Schwinger and
// Dyson equations (Eqs. 3 and 2), which the step-by-step updates satisfy only up to rounding.
//
//   resid[0]     = ||E - E_inc - G0 X E||_2 / ||E||_2                      (Eq. 3 residual)
//   resid[1 + s] = ||G[:, c_s] - g_s||_2 / ||g_s||_2,  (I - G0 X) g_s = G0[:, c_s]   (Eq. 2)
//
// g_s is found by restarted GMRES started from the stored column.  The background G0 depends
// on pixel offsets only, so G0 X v restricted to the pixels is a 2-D convolution: it is
// computed by circulant embedding on an Ly x Lx power-of-two grid (Lx >= 2 nx - 1,
// Ly >= 2 ny - 1) with radix-2 FFTs in FP64; the monitor row of G0 X v is a dot product.
// X is zero at the monitor, so the monitor column of G0 never enters.
#include <math.h>

#include <vector>

#include "gf_internal.cuh"

namespace gf {

static int64_t pow2_at_least(int64_t v) {
  int64_t L = 1;
  while (L < v) L <<= 1;
  return L;
}

struct RefLayout {
  int64_t Lx, Ly, n, N;
  int m;
  size_t table, khat, grid, V, w, x, b, r, dots, twx, twy, part, total;
};

// Reductions over the n unknowns run on the whole GPU in two stages: kRefParts slices (or the
// CTAs of a grid-stride kernel) write partial sums, one warp per result adds them in a fixed
// order -- deterministic, unlike atomics.
constexpr int kRefParts = 128;
constexpr int kRefBlocks = 152 * 4;          // CTAs of the grid-stride vector kernels

static size_t up256r(size_t x) { return (x + 255) & ~(size_t)255; }

RefLayout ref_layout(const gf_geom& g, int restart) {
  RefLayout L;
  L.N = (int64_t)g.nx * g.ny;
  L.n = L.N + 1;
  L.Lx = pow2_at_least(2 * (int64_t)g.nx - 1);
  L.Ly = pow2_at_least(2 * (int64_t)g.ny - 1);
  L.m = restart;
  const size_t c = sizeof(cplx);
  size_t o = 0;
  L.table = o; o = up256r(o + c * (size_t)(2 * L.N));
  L.khat = o; o = up256r(o + c * (size_t)(L.Lx * L.Ly));
  L.grid = o; o = up256r(o + c * (size_t)(L.Lx * L.Ly));
  L.V = o; o = up256r(o + c * (size_t)L.n * (L.m + 1));
  L.w = o; o = up256r(o + c * (size_t)L.n);
  L.x = o; o = up256r(o + c * (size_t)L.n);
  L.b = o; o = up256r(o + c * (size_t)L.n);
  L.r = o; o = up256r(o + c * (size_t)L.n);
  L.dots = o; o = up256r(o + c * (size_t)(L.m + 2));
  L.twx = o; o = up256r(o + c * (size_t)(L.Lx / 2 + 1));
  L.twy = o; o = up256r(o + c * (size_t)(L.Ly / 2 + 1));
  const size_t nparts = (size_t)(L.m + 1) * kRefParts > (size_t)kRefBlocks ? (size_t)(L.m + 1) * kRefParts
                                                                              : (size_t)kRefBlocks;
  L.part = o; o = up256r(o + c * nparts);
  L.total = o;
  return L;
}

// ---- FFT: one CTA per line, radix-2 decimation in time in shared memory ----------------------
// Twiddles from a table tw[t] = exp(-2 pi i t / L), t < L / 2, made once per refresh (computing
// them per butterfly cost an FP64 sincospi each: 21 million per GMRES iteration at L = 1024);
// the stage with butterflies of span 2h uses tw[kk L / (2 h)], conjugated for sign = +1.
__global__ void k_twiddles(cplx* __restrict__ tw, int L) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L / 2; t += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(-(double)t / (double)(L / 2), &sn, &cs);
    tw[t] = mk(cs, sn);
  }
}

__global__ void k_fft_lines(cplx* __restrict__ data, int L, int logL, int64_t stride, int64_t line_stride,
                            double sign, const cplx* __restrict__ tw) {
  extern __shared__ cplx sh[];
  cplx* stw = sh + L;                                  // the twiddle table, L / 2 entries
  cplx* base = data + blockIdx.x * line_stride;
  for (int e = threadIdx.x; e < L; e += blockDim.x) {
    const int rev = (int)(__brev((unsigned)e) >> (32 - logL));
    sh[rev] = base[(int64_t)e * stride];
  }
  for (int t = threadIdx.x; t < L / 2; t += blockDim.x) stw[t] = tw[t];
  __syncthreads();
  for (int s = 1; s <= logL; ++s) {
    const int half = 1 << (s - 1);
    const int step = L >> s;                           // L / (2 half)
    for (int t = threadIdx.x; t < L / 2; t += blockDim.x) {
      const int kk = t & (half - 1);
      const int i = ((t >> (s - 1)) << s) + kk;
      const int j = i + half;
      cplx wv = stw[kk * step];
      if (sign > 0.0) wv.im = -wv.im;
      const cplx tv = wv * sh[j];
      sh[j] = sh[i] - tv;
      sh[i] = sh[i] + tv;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < L; e += blockDim.x) base[(int64_t)e * stride] = sh[e];
}

static void fft2(cplx* grid, int64_t Lx, int64_t Ly, double sign, const cplx* twx, const cplx* twy, cudaStream_t st) {
  int lx = 0, ly = 0;
  while ((1LL << lx) < Lx) ++lx;
  while ((1LL << ly) < Ly) ++ly;
  if (Lx > 1) {
    int th = (int)(Lx / 2 < 512 ? Lx / 2 : 512);
    k_fft_lines<<<(unsigned)Ly, th, sizeof(cplx) * (Lx + Lx / 2), st>>>(grid, (int)Lx, lx, 1, Lx, sign, twx);
  }
  if (Ly > 1) {
    int th = (int)(Ly / 2 < 512 ? Ly / 2 : 512);
    k_fft_lines<<<(unsigned)Lx, th, sizeof(cplx) * (Ly + Ly / 2), st>>>(grid, (int)Ly, ly, Lx, 1, sign, twy);
  }
}

// ---- circulant embedding of the G0 pixel kernel ---------------------------------------------
__global__ void k_embed(const cplx* __restrict__ table, int nx, int ny, int64_t Lx, int64_t Ly, cplx* __restrict__ K) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Lx * Ly; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = e / Lx, x = e - y * Lx;
    const int64_t dy = y < ny ? y : (y > Ly - ny ? Ly - y : -1);
    const int64_t dx = x < nx ? x : (x > Lx - nx ? Lx - x : -1);
    K[e] = (dy >= 0 && dx >= 0) ? table[dy * nx + dx] : mk(0.0, 0.0);
  }
}

__global__ void k_mul(cplx* __restrict__ a, const cplx* __restrict__ b, int64_t cnt, double scale) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
    a[e] = scale * (a[e] * b[e]);
}

// grid <- chi v on the pixels (zero padded)
__global__ void k_scatter(const cplx* __restrict__ v, const uint8_t* __restrict__ state, double chi, int nx, int ny,
                          int64_t Lx, int64_t Ly, cplx* __restrict__ grid) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Lx * Ly; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = e / Lx, x = e - y * Lx;
    cplx u = mk(0.0, 0.0);
    if (x < nx && y < ny) {
      const int64_t j = y * nx + x;
      if (state[j]) u = chi * v[j];
    }
    grid[e] = u;
  }
}

// out = alpha * v + beta * (G0 X v) on the pixels from the convolution grid; the monitor entry is
// the dot product of the monitor row with X v, whose per-CTA partial sums go to part[blockIdx.x]
// (k_mon_finish adds them)
__global__ void k_gather_combine(const cplx* __restrict__ v, const cplx* __restrict__ grid, const cplx* __restrict__ mon,
                                 const uint8_t* __restrict__ state, double chi, int nx, int ny, int64_t Lx,
                                 double alpha, double beta, cplx* __restrict__ out, cplx* __restrict__ part) {
  __shared__ double sr[32], si[32];
  const int64_t N = (int64_t)nx * ny;
  double ar = 0.0, ai = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / nx, x = i - y * nx;
    out[i] = alpha * v[i] + beta * grid[y * Lx + x];
    if (state[i]) {
      const cplx t = mon[i] * (chi * v[i]);
      ar += t.re;
      ai += t.im;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar += __shfl_down_sync(0xffffffffu, ar, o);
    ai += __shfl_down_sync(0xffffffffu, ai, o);
  }
  if ((threadIdx.x & 31) == 0) { sr[threadIdx.x >> 5] = ar; si[threadIdx.x >> 5] = ai; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tr += sr[w]; ti += si[w]; }
    part[blockIdx.x] = mk(tr, ti);
  }
}

// one warp: s = the nparts partial sums in a fixed order
__device__ __forceinline__ cplx warp_sum_parts(const cplx* __restrict__ part, int nparts) {
  const int lane = threadIdx.x & 31;
  double ar = 0.0, ai = 0.0;
  for (int p = lane; p < nparts; p += 32) {
    ar += part[p].re;
    ai += part[p].im;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar += __shfl_down_sync(0xffffffffu, ar, o);
    ai += __shfl_down_sync(0xffffffffu, ai, o);
  }
  return mk(ar, ai);
}

__global__ void k_mon_finish(const cplx* __restrict__ part, int nparts, const cplx* __restrict__ v, int64_t N,
                             double alpha, double beta, cplx* __restrict__ out) {
  const cplx s = warp_sum_parts(part, nparts);
  if (threadIdx.x == 0) out[N] = alpha * v[N] + beta * s;
}

// ---- vectors ----------------------------------------------------------------------------------
__device__ void block_sum2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) { sa[threadIdx.x >> 5] = a; sb[threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { ta += sa[w]; tb += sb[w]; }
    a = ta;
    b = tb;
  }
}

// part[q][p] = sum over slice p of conj(V_q) w  (grid kRefParts x nvec)
__global__ void k_dots_part(const cplx* __restrict__ V, int64_t n, const cplx* __restrict__ w, cplx* __restrict__ part) {
  const int q = blockIdx.y, p = blockIdx.x;
  const int64_t lo = n * p / kRefParts, hi = n * (p + 1) / kRefParts;
  const cplx* vq = V + (int64_t)q * n;
  double ar = 0.0, ai = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const cplx a = vq[i], b = w[i];
    ar += a.re * b.re + a.im * b.im;
    ai += a.re * b.im - a.im * b.re;
  }
  block_sum2(ar, ai);
  if (threadIdx.x == 0) part[q * kRefParts + p] = mk(ar, ai);
}

// h[q] = sum of part[q][*] (one warp per vector)
__global__ void k_parts_sum(const cplx* __restrict__ part, cplx* __restrict__ h) {
  const cplx s = warp_sum_parts(part + (int64_t)blockIdx.x * kRefParts, kRefParts);
  if (threadIdx.x == 0) h[blockIdx.x] = s;
}

// w -= sum_q h[q] V_q
__global__ void k_sub_combo(cplx* __restrict__ w, const cplx* __restrict__ V, int64_t n, int nvec,
                            const cplx* __restrict__ h) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    cplx acc = w[i];
    for (int q = 0; q < nvec; ++q) acc = acc - h[q] * V[(int64_t)q * n + i];
    w[i] = acc;
  }
}

// part[p] = ||a restricted to slice p||^2 (as the real part; grid kRefParts)
__global__ void k_norm2_part(const cplx* __restrict__ a, int64_t n, cplx* __restrict__ part) {
  const int p = blockIdx.x;
  const int64_t lo = n * p / kRefParts, hi = n * (p + 1) / kRefParts;
  double s = 0.0, z = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += abs2(a[i]);
  block_sum2(s, z);
  if (threadIdx.x == 0) part[p] = mk(s, 0.0);
}

// out[0] = the sum of the kRefParts partial squares
__global__ void k_norm2_finish(const cplx* __restrict__ part, double* __restrict__ out) {
  const cplx s = warp_sum_parts(part, kRefParts);
  if (threadIdx.x == 0) *out = s.re;
}

// y = a * x   (a real)
__global__ void k_scale(cplx* __restrict__ y, const cplx* __restrict__ x, int64_t n, double a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// y = x - z
__global__ void k_diff(cplx* __restrict__ y, const cplx* __restrict__ x, const cplx* __restrict__ z, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] - z[i];
}

// x += sum_q c[q] V_q  (c on the device)
__global__ void k_add_combo(cplx* __restrict__ x, const cplx* __restrict__ V, int64_t n, int nvec,
                            const cplx* __restrict__ c) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    cplx acc = x[i];
    for (int q = 0; q < nvec; ++q) acc = acc + c[q] * V[(int64_t)q * n + i];
    x[i] = acc;
  }
}

// E_inc at the n points
__global__ void k_einc(int nx, int ny, double dx, double k, double my, cplx* __restrict__ out) {
  const int64_t N = (int64_t)nx * ny;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= N; j += (int64_t)gridDim.x * blockDim.x) {
    const double y = j < N ? ((double)(j / nx) + 0.5) * dx : my;
    double s, c;
    sincos(k * y, &s, &c);
    out[j] = mk(c, s);
  }
}

// b = G0[:, c] from the table (column c of the background matrix), x = stored G[:, c]
__global__ void k_column_rhs(const cplx* __restrict__ table, int nx, int ny, int64_t c, const void* G, int dtype,
                             int64_t ldg, cplx* __restrict__ b, cplx* __restrict__ x) {
  const int64_t N = (int64_t)nx * ny;
  const cplx* mon = table + N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= N; i += (int64_t)gridDim.x * blockDim.x) {
    cplx v;
    if (c == N) {
      v = i < N ? mon[i] : mk(0.0, 0.0);
    } else if (i == N) {
      v = mon[c];
    } else {
      const int64_t iy = i / nx, ix = i - iy * nx, cy = c / nx, cx = c - cy * nx;
      const int64_t ay = iy > cy ? iy - cy : cy - iy, ax = ix > cx ? ix - cx : cx - ix;
      v = table[ay * nx + ax];
    }
    b[i] = v;
    x[i] = ldG(G, dtype, ldg, i, c);
  }
}

struct RefCtx {
  const gf_geom* g;
  RefLayout L;
  char* ws;
  const uint8_t* state;
  double chi;
  cudaStream_t st;
  int blocks;
};

static cplx* P(const RefCtx& c, size_t off) { return reinterpret_cast<cplx*>(c.ws + off); }

// out = v - G0 X v  (alpha = 1, beta = -1) or out = G0 X v (alpha = 0, beta = 1)
static void apply(const RefCtx& c, const cplx* v, cplx* out, double alpha, double beta) {
  const RefLayout& L = c.L;
  cplx* grid = P(c, L.grid);
  k_scatter<<<c.blocks, 256, 0, c.st>>>(v, c.state, c.chi, c.g->nx, c.g->ny, L.Lx, L.Ly, grid);
  fft2(grid, L.Lx, L.Ly, -1.0, P(c, L.twx), P(c, L.twy), c.st);
  k_mul<<<c.blocks, 256, 0, c.st>>>(grid, P(c, L.khat), L.Lx * L.Ly, 1.0 / (double)(L.Lx * L.Ly));
  fft2(grid, L.Lx, L.Ly, +1.0, P(c, L.twx), P(c, L.twy), c.st);
  k_gather_combine<<<kRefBlocks, 256, 0, c.st>>>(v, grid, P(c, L.table) + L.N, c.state, c.chi, c.g->nx, c.g->ny, L.Lx,
                                                alpha, beta, out, P(c, L.part));
  k_mon_finish<<<1, 32, 0, c.st>>>(P(c, L.part), kRefBlocks, v, L.N, alpha, beta, out);
}

static double norm2_host(const RefCtx& c, const cplx* a) {
  double* d = reinterpret_cast<double*>(P(c, c.L.dots));
  k_norm2_part<<<kRefParts, 256, 0, c.st>>>(a, c.L.n, P(c, c.L.part));
  k_norm2_finish<<<1, 32, 0, c.st>>>(P(c, c.L.part), d);
  double h = 0.0;
  cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, c.st);
  cudaStreamSynchronize(c.st);
  return sqrt(h);
}

// GMRES(m) on (I - G0 X) x = b from the initial x.  Returns iterations used.
static int gmres(const RefCtx& c, int max_iter, double tol) {
  const RefLayout& L = c.L;
  const int64_t n = L.n;
  cplx *V = P(c, L.V), *w = P(c, L.w), *x = P(c, L.x), *b = P(c, L.b), *r = P(c, L.r);
  cplx* hd = P(c, L.dots);
  const double bnorm = norm2_host(c, b);
  if (!(bnorm > 0.0)) return 0;
  const int m = L.m;
  std::vector<cplx> H((size_t)(m + 1) * m), cs(m), sn(m), gvec(m + 1), hcol(m + 2);
  int it = 0;
  while (it < max_iter) {
    apply(c, x, w, 1.0, -1.0);                        // w = A x
    k_diff<<<c.blocks, 256, 0, c.st>>>(r, b, w, n);    // r = b - A x
    const double beta = norm2_host(c, r);
    if (!(beta > tol * bnorm)) break;
    k_scale<<<c.blocks, 256, 0, c.st>>>(V, r, n, 1.0 / beta);
    for (auto& z : gvec) z = mk(0.0, 0.0);
    gvec[0] = mk(beta, 0.0);
    int k = 0;
    bool converged = false;
    for (; k < m && it < max_iter; ++k, ++it) {
      apply(c, V + (int64_t)k * n, w, 1.0, -1.0);     // w = A v_k
      // classical Gram-Schmidt, twice
      std::vector<cplx> hsum(k + 1, mk(0.0, 0.0));
      for (int pass = 0; pass < 2; ++pass) {
        k_dots_part<<<dim3(kRefParts, (unsigned)(k + 1)), 256, 0, c.st>>>(V, n, w, P(c, L.part));
        k_parts_sum<<<k + 1, 32, 0, c.st>>>(P(c, L.part), hd);
        k_sub_combo<<<c.blocks, 256, 0, c.st>>>(w, V, n, k + 1, hd);
        cudaMemcpyAsync(hcol.data(), hd, sizeof(cplx) * (k + 1), cudaMemcpyDeviceToHost, c.st);
        cudaStreamSynchronize(c.st);
        for (int q = 0; q <= k; ++q) hsum[q] = hsum[q] + hcol[q];
      }
      const double hn = norm2_host(c, w);
      for (int q = 0; q <= k; ++q) H[(size_t)q * m + k] = hsum[q];
      H[(size_t)(k + 1) * m + k] = mk(hn, 0.0);
      if (hn > 0.0) k_scale<<<c.blocks, 256, 0, c.st>>>(V + (int64_t)(k + 1) * n, w, n, 1.0 / hn);
      // apply the previous Givens rotations, then a new one zeroing H[k+1][k]
      for (int q = 0; q < k; ++q) {
        const cplx a = H[(size_t)q * m + k], bq = H[(size_t)(q + 1) * m + k];
        const cplx cq = cs[q], sq = sn[q];
        H[(size_t)q * m + k] = cq * a + sq * bq;
        H[(size_t)(q + 1) * m + k] = mk(-sq.re, sq.im) * a + mk(cq.re, -cq.im) * bq;   // -conj(s) a + conj(c) b
      }
      {
        const cplx a = H[(size_t)k * m + k], bb = H[(size_t)(k + 1) * m + k];
        const double den = sqrt(abs2(a) + abs2(bb));
        cplx ck, sk;
        if (den == 0.0) { ck = mk(1.0, 0.0); sk = mk(0.0, 0.0); }
        else { ck = mk(a.re / den, -a.im / den); sk = mk(bb.re / den, -bb.im / den); }   // conj(a)/den, conj(b)/den
        cs[k] = ck;
        sn[k] = sk;
        H[(size_t)k * m + k] = ck * a + sk * bb;
        H[(size_t)(k + 1) * m + k] = mk(0.0, 0.0);
        const cplx gk = gvec[k];
        gvec[k] = ck * gk;
        gvec[k + 1] = mk(-sk.re, sk.im) * gk;
      }
      if (!(cabs1(gvec[k + 1]) > tol * bnorm) || hn == 0.0) { ++k; ++it; converged = true; break; }
    }
    // back substitution H y = g (k x k upper triangular), x += V y
    std::vector<cplx> y(k);
    for (int q = k - 1; q >= 0; --q) {
      cplx acc = gvec[q];
      for (int v = q + 1; v < k; ++v) acc = acc - H[(size_t)q * m + v] * y[v];
      y[q] = cdiv(acc, H[(size_t)q * m + q]);
    }
    if (k > 0) {
      cudaMemcpyAsync(hd, y.data(), sizeof(cplx) * k, cudaMemcpyHostToDevice, c.st);
      k_add_combo<<<c.blocks, 256, 0, c.st>>>(x, V, n, k, hd);
    }
    if (converged) break;
  }
  cudaStreamSynchronize(c.st);
  return it;
}

size_t refresh_workspace_size(const gf_geom& g, int restart) { return ref_layout(g, restart).total; }

// Twiddles, the background table and the FFT of the embedded Toeplitz kernel: the set-up every
// G0 X v product of a refresh call needs.
static void ref_setup(RefCtx& c, const gf_geom& g, const uint8_t* state, int restart, char* ws, cudaStream_t st) {
  c.g = &g;
  c.L = ref_layout(g, restart);
  c.ws = ws;
  c.state = state;
  c.chi = g.eps_mat - g.eps_bg;
  c.st = st;
  c.blocks = kRefBlocks;
  const RefLayout& L = c.L;
  cudaFuncSetAttribute(k_fft_lines, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(cplx) * (8192 + 4096)));
  if (L.Lx > 1) k_twiddles<<<(unsigned)((L.Lx / 2 + 255) / 256), 256, 0, st>>>(P(c, L.twx), (int)L.Lx);
  if (L.Ly > 1) k_twiddles<<<(unsigned)((L.Ly / 2 + 255) / 256), 256, 0, st>>>(P(c, L.twy), (int)L.Ly);
  launch_fill_table(g, P(c, L.table), st);
  k_embed<<<c.blocks, 256, 0, st>>>(P(c, L.table), g.nx, g.ny, L.Lx, L.Ly, P(c, L.khat));
  fft2(P(c, L.khat), L.Lx, L.Ly, -1.0, P(c, L.twx), P(c, L.twy), st);
}

// ||b - (I - G0 X) x|| / ||b||, using w and r as scratch
static double rel_residual(const RefCtx& c, const cplx* x, const cplx* b) {
  const RefLayout& L = c.L;
  apply(c, x, P(c, L.w), 1.0, -1.0);
  k_diff<<<c.blocks, 256, 0, c.st>>>(P(c, L.r), b, P(c, L.w), L.n);
  return norm2_host(c, P(c, L.r)) / norm2_host(c, b);
}

gf_status refresh(const gf_problem& prob, int dtype, const uint8_t* state, int nsample, const int32_t* cols,
                  int restart, int max_iter, double tol, double* resid, int32_t* iters, double* colres, char* ws,
                  cudaStream_t st) {
  const gf_geom& g = prob.geom;
  RefCtx c;
  ref_setup(c, g, state, restart, ws, st);
  const RefLayout& L = c.L;
  // Eq. 3 residual of E: r = E - E_inc - G0 X E
  const cplx* E = reinterpret_cast<const cplx*>(prob.E);
  const double k0 = 2.0 * M_PI / g.wavelength;
  k_einc<<<c.blocks, 256, 0, st>>>(g.nx, g.ny, g.dx, k0, g.mon_y, P(c, L.b));
  apply(c, E, P(c, L.w), 0.0, 1.0);                               // w = G0 X E
  k_diff<<<c.blocks, 256, 0, st>>>(P(c, L.r), E, P(c, L.b), L.n);   // r = E - E_inc
  k_diff<<<c.blocks, 256, 0, st>>>(P(c, L.r), P(c, L.r), P(c, L.w), L.n);
  resid[0] = norm2_host(c, P(c, L.r)) / norm2_host(c, E);
  for (int s = 0; s < nsample; ++s) {
    k_column_rhs<<<c.blocks, 256, 0, st>>>(P(c, L.table), g.nx, g.ny, cols[s], prob.G, dtype, prob.ldg, P(c, L.b),
                                           P(c, L.x));
    // backward error of the stored column (Eq. 2): ||G0[:, c] - (I - G0 X) G[:, c]|| / ||G0[:, c]||
    if (colres) colres[s] = rel_residual(c, P(c, L.x), P(c, L.b));
    const int its = gmres(c, max_iter, tol);     // x: stored column -> refined solution
    if (iters) iters[s] = its;
    k_column_rhs<<<c.blocks, 256, 0, st>>>(P(c, L.table), g.nx, g.ny, cols[s], prob.G, dtype, prob.ldg, P(c, L.b),
                                           P(c, L.w));                 // w = stored column again
    k_diff<<<c.blocks, 256, 0, st>>>(P(c, L.r), P(c, L.w), P(c, L.x), L.n);
    resid[1 + s] = norm2_host(c, P(c, L.r)) / norm2_host(c, P(c, L.x));
  }
  cudaStreamSynchronize(st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GF_OK : GF_ECUDA;
}

gf_status refresh_field(const gf_problem& prob, const uint8_t* state, double e_tol, int restart, int max_iter,
                        double tol, gf_refresh_report* rep, char* ws, cudaStream_t st) {
  const gf_geom& g = prob.geom;
  RefCtx c;
  ref_setup(c, g, state, restart, ws, st);
  const RefLayout& L = c.L;
  cplx* E = reinterpret_cast<cplx*>(prob.E);
  const double k0 = 2.0 * M_PI / g.wavelength;
  k_einc<<<c.blocks, 256, 0, st>>>(g.nx, g.ny, g.dx, k0, g.mon_y, P(c, L.b));   // b = E_inc
  const double r0 = rel_residual(c, E, P(c, L.b));               // ||E_inc - (I - G0 X) E|| / ||E_inc||
  rep->e_residual = r0;
  rep->e_residual_after = r0;
  rep->e_iters = 0;
  rep->e_replaced = 0;
  if (r0 > e_tol) {
    k_scale<<<c.blocks, 256, 0, st>>>(P(c, L.x), E, L.n, 1.0);    // x = E, the initial guess
    rep->e_iters = gmres(c, max_iter, tol);
    const double r1 = rel_residual(c, P(c, L.x), P(c, L.b));
    if (r1 < r0) {
      k_scale<<<c.blocks, 256, 0, st>>>(E, P(c, L.x), L.n, 1.0);
      rep->e_residual_after = r1;
      rep->e_replaced = 1;
    }
  }
  cudaStreamSynchronize(st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GF_OK : GF_ECUDA;
}

}  // namespace gf
