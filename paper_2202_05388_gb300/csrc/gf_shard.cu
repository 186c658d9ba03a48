// Row-block shards of G: the partitioned form of the method (Sec. III).  The paper splits the
// rows of G over partitions; each partition evaluates the dFOM of the candidates it holds, the
// results are combined globally, the rows of the chosen pixels are broadcast to every partition
// and each partition updates its own rows (Eqs. 10, 14).
//
// Here a shard holds the rows of G of pixel rows [y0, y1) (the shard with y1 = ny also holds the
// monitor row).  What evaluation reads -- the bands and the monitor entries G[N, j] = G[j, N]
// (reciprocity) of the shard's pixels and of one halo pixel row y1 -- comes from its own rows
// and from the next shard (the halo, exchanged by the caller); the field E and the design state
// are kept whole and identical on every shard.  A step per shard is
//   gf_shard_eval         dFOM of the candidates anchored in its pixel rows (others -inf);
//   (caller)              elementwise max of the dFOM arrays over the shards;
//   gf_select_topk        the same choice on every shard;
//   gf_shard_gather_rows  its rows of the update set V into a p x n panel (others zero);
//   (caller)              sum of the panels over the shards: every shard has G[V, :];
//   gf_shard_apply_update capacitance solve from the panel, update of its own rows, of E (from
//                         the panel, G[i, V] = G[V, i]) and of its bands;
//   gf_shard_pack_halo / gf_shard_unpack_halo  the first pixel row's bands to the previous shard.
#include <math.h>

#include "gf_internal.cuh"

namespace gf {

struct ShardGeo {
  int nx, ny, y0, y1;
  int64_t N, n, r0, r1;          // global rows [r0, r1) held
};

static ShardGeo shard_geo(const gf_shard& s) {
  ShardGeo g;
  g.nx = s.geom.nx;
  g.ny = s.geom.ny;
  g.y0 = s.y0;
  g.y1 = s.y1;
  g.N = (int64_t)g.nx * g.ny;
  g.n = g.N + 1;
  g.r0 = (int64_t)g.y0 * g.nx;
  g.r1 = (int64_t)g.y1 * g.nx + (g.y1 == g.ny ? 1 : 0);
  return g;
}

template <typename T>
__device__ __forceinline__ void st_g(void* G, int64_t off, cplx v);
template <>
__device__ __forceinline__ void st_g<double2>(void* G, int64_t off, cplx v) {
  reinterpret_cast<double2*>(G)[off] = make_double2(v.re, v.im);
}
template <>
__device__ __forceinline__ void st_g<float2>(void* G, int64_t off, cplx v) {
  reinterpret_cast<float2*>(G)[off] = make_float2((float)v.re, (float)v.im);
}

// Background rows [r0, r1) of G0 (the fill's offset table; monitor values after the N offsets):
// one block per row, threads along its ldg columns.
template <typename T>
__global__ void k_shard_fill_rows(ShardGeo g, int64_t ldg, const cplx* __restrict__ table, void* __restrict__ G) {
  const cplx* mon = table + g.N;
  for (int64_t il = blockIdx.x; il < g.r1 - g.r0; il += gridDim.x) {
    const int64_t i = g.r0 + il;
    const int64_t row = il * ldg;
    if (i < g.N) {
      const int iy = (int)(i / g.nx), ix = (int)(i % g.nx);
      for (int64_t j = threadIdx.x; j < ldg; j += blockDim.x) {
        cplx v;
        if (j < g.N) {
          const int jy = (int)(j / g.nx), jx = (int)(j - (int64_t)jy * g.nx);
          const int ay = iy > jy ? iy - jy : jy - iy, ax = ix > jx ? ix - jx : jx - ix;
          v = table[(int64_t)ay * g.nx + ax];
        } else {
          v = j == g.N ? mon[i] : mk(0.0, 0.0);
        }
        st_g<T>(G, row + j, v);
      }
    } else {                       // the monitor row (G_NN = 0)
      for (int64_t j = threadIdx.x; j < ldg; j += blockDim.x) st_g<T>(G, row + j, j < g.N ? mon[j] : mk(0.0, 0.0));
    }
  }
}

// Bands and monitor entries of pixel rows [ya, yb) of the background (from the offset table).
__global__ void k_shard_bands_g0(ShardGeo g, int ya, int yb, const cplx* __restrict__ table, cplx* __restrict__ bands,
                                 cplx* __restrict__ mon) {
  const int64_t j0 = (int64_t)ya * g.nx, cnt = (int64_t)(yb - ya) * g.nx;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (GF_NBANDS + 1) * cnt;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / cnt);
    const int64_t j = j0 + (t - (int64_t)b * cnt);
    if (b == GF_NBANDS) {
      mon[j] = table[g.N + j];
      continue;
    }
    const int iy = (int)(j / g.nx), ix = (int)(j % g.nx);
    int ddx, ddy;
    band_offset(b, ddx, ddy);
    const int jx = ix + ddx, jy = iy + ddy;
    cplx v = mk(0.0, 0.0);
    if (jx >= 0 && jx < g.nx && jy >= 0 && jy < g.ny) v = table[(int64_t)(ddy < 0 ? -ddy : ddy) * g.nx + (ddx < 0 ? -ddx : ddx)];
    bands[(int64_t)b * g.N + j] = v;
  }
}

// Bands and monitor entries G[j, N] of the shard's own pixel rows, read from its rows of G.
__global__ void k_shard_bands(ShardGeo g, int dtype, const void* __restrict__ G, int64_t ldg, cplx* __restrict__ bands,
                              cplx* __restrict__ mon) {
  const int64_t j0 = (int64_t)g.y0 * g.nx, cnt = (int64_t)(g.y1 - g.y0) * g.nx;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (GF_NBANDS + 1) * cnt;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / cnt);
    const int64_t j = j0 + (t - (int64_t)b * cnt);
    const int64_t il = j - g.r0;
    if (b == GF_NBANDS) {
      mon[j] = ldG(G, dtype, ldg, il, g.N);
      continue;
    }
    const int iy = (int)(j / g.nx), ix = (int)(j % g.nx);
    int ddx, ddy;
    band_offset(b, ddx, ddy);
    const int jx = ix + ddx, jy = iy + ddy;
    cplx v = mk(0.0, 0.0);
    if (jx >= 0 && jx < g.nx && jy >= 0 && jy < g.ny) v = ldG(G, dtype, ldg, il, (int64_t)jy * g.nx + jx);
    bands[(int64_t)b * g.N + j] = v;
  }
}

// Halo record of one pixel row y: its nine bands and its monitor entries, (GF_NBANDS + 1) x nx.
__global__ void k_shard_pack(ShardGeo g, int y, const cplx* __restrict__ bands, const cplx* __restrict__ mon,
                             cplx* __restrict__ out) {
  const int64_t j0 = (int64_t)y * g.nx;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)(GF_NBANDS + 1) * g.nx;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / g.nx);
    const int64_t x = t - (int64_t)b * g.nx;
    out[t] = b == GF_NBANDS ? mon[j0 + x] : bands[(int64_t)b * g.N + j0 + x];
  }
}
__global__ void k_shard_unpack(ShardGeo g, int y, const cplx* __restrict__ in, cplx* __restrict__ bands,
                               cplx* __restrict__ mon) {
  const int64_t j0 = (int64_t)y * g.nx;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)(GF_NBANDS + 1) * g.nx;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / g.nx);
    const int64_t x = t - (int64_t)b * g.nx;
    if (b == GF_NBANDS) mon[j0 + x] = in[t];
    else bands[(int64_t)b * g.N + j0 + x] = in[t];
  }
}

__global__ void k_fill_neg_inf(double* __restrict__ d, int64_t cnt) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
    d[t] = -INFINITY;
}

// The update set V of the chosen candidates (the union of idx[0..k) in order, as the capacitance
// kernel forms it) and the shard's rows of it: panel row u = G[V[u], :] when the shard holds row
// V[u], zero otherwise (so that summing the panels of all shards gives every row once); rows
// u >= |V| and columns j >= n are zero.  A step whose status is not GF_OK gathers nothing.
constexpr int kGatherMaxV = 4 * 256;
template <typename T>
__global__ void k_shard_gather(ShardGeo g, int kind, int dir_mask, int k, double chi, const uint8_t* __restrict__ state,
                               const int32_t* __restrict__ idx, const int32_t* __restrict__ status,
                               const T* __restrict__ G, int64_t ldg, int pmax, T* __restrict__ panel, int64_t ldp) {
  __shared__ int32_t sV[kGatherMaxV];
  __shared__ double sD[kGatherMaxV];
  __shared__ int s_nv;
  if (threadIdx.x == 0) {
    int nv = 0;
    if (*status == GF_OK)
      for (int c = 0; c < k; ++c) {
        const int32_t id = idx[c];
        if (id < 0) break;
        nv += cand_pixels(id, kind, dir_mask, g.nx, g.ny, chi, state, sV + nv, sD + nv);
      }
    s_nv = nv;
  }
  __syncthreads();
  const int nv = s_nv;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)pmax * ldp;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int u = (int)(t / ldp);
    const int64_t j = t - (int64_t)u * ldp;
    T v;
    if (u < nv && j < g.n && sV[u] >= g.r0 && sV[u] < g.r1) v = G[(int64_t)(sV[u] - g.r0) * ldg + j];
    else memset(&v, 0, sizeof(T));
    panel[t] = v;
  }
}

static int grid_of(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace gf

// ----------------------------------------------------------------------------- C ABI
static gf_status check_shard(gf_handle* h, const gf_shard* s, int dtype) {
  if (!s) return gf::api_fail_msg(h, GF_EINVAL, "shard is NULL");
  gf_problem probe;
  probe.geom = s->geom;
  probe.G = s->G;
  probe.ldg = s->ldg;
  probe.E = s->E;
  probe.bands = s->bands;
  gf_status st = gf::api_check_problem(h, &probe, dtype);
  if (st) return st;
  if (s->geom.ny < 2 && s->y1 < s->geom.ny) return gf::api_fail_msg(h, GF_EINVAL, "bad shard rows");
  if (s->y0 < 0 || s->y1 <= s->y0 || s->y1 > s->geom.ny)
    return gf::api_fail_msg(h, GF_EINVAL, "shard pixel rows must satisfy 0 <= y0 < y1 <= ny");
  if (!s->mon || ((uintptr_t)s->mon & 15u)) return gf::api_fail_msg(h, GF_EINVAL, "mon must be non-NULL and 16-byte aligned");
  return gf::api_bind_device(h);
}

static gf::ShardGeo geo_of(const gf_shard* s) { return gf::shard_geo(*s); }

extern "C" {

int64_t gf_shard_rows(const gf_shard* s) {
  if (!s || s->geom.nx < 1 || s->geom.ny < 1 || s->y0 < 0 || s->y1 <= s->y0 || s->y1 > s->geom.ny) return 0;
  const gf::ShardGeo g = geo_of(s);
  return g.r1 - g.r0;
}

gf_status gf_shard_fill_g0(gf_handle* h, const gf_shard* shard, int32_t dtype, void* ws, size_t ws_bytes, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = check_shard(h, shard, dtype);
  if (s) return s;
  const gf::ShardGeo g = geo_of(shard);
  const size_t need = sizeof(gf::cplx) * (size_t)(2 * g.N);
  if (!ws || ((uintptr_t)ws & 255u)) return gf::api_fail_msg(h, GF_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need) return gf::api_fail_msg(h, GF_ENOMEM, "workspace too small for the fill table");
  cudaStream_t st = (cudaStream_t)stream;
  gf::cplx* table = reinterpret_cast<gf::cplx*>(ws);
  gf::launch_fill_table(shard->geom, table, st);
  const int64_t rows = g.r1 - g.r0;
  const int blocks = (int)(rows < 152 * 16 ? rows : 152 * 16);
  if (dtype == GF_C128)
    gf::k_shard_fill_rows<double2><<<blocks, 256, 0, st>>>(g, shard->ldg, table, shard->G);
  else
    gf::k_shard_fill_rows<float2><<<blocks, 256, 0, st>>>(g, shard->ldg, table, shard->G);
  gf::launch_fill_field(shard->geom, reinterpret_cast<gf::cplx*>(shard->E), st);
  const int yb = g.y1 < g.ny ? g.y1 + 1 : g.ny;
  gf::k_shard_bands_g0<<<gf::grid_of((int64_t)(GF_NBANDS + 1) * (yb - g.y0) * g.nx, 256), 256, 0, st>>>(
      g, g.y0, yb, table, reinterpret_cast<gf::cplx*>(shard->bands), reinterpret_cast<gf::cplx*>(shard->mon));
  return gf::api_cuda_check(h, "gf_shard_fill_g0 launch");
}

gf_status gf_shard_eval(gf_handle* h, const gf_shard* shard, int32_t dtype, const uint8_t* state,
                        const gf_cand_spec* spec, double* dfom, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = check_shard(h, shard, dtype);
  if (s) return s;
  if ((s = gf::api_check_spec(h, &shard->geom, spec))) return s;
  if (!state || !dfom || ((uintptr_t)dfom & 15u)) return gf::api_fail_msg(h, GF_EINVAL, "state and dfom must be non-NULL, dfom 16-byte aligned");
  const gf::ShardGeo g = geo_of(shard);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t ncand = gf_num_candidates(&shard->geom, spec);
  gf::k_fill_neg_inf<<<gf::grid_of(ncand, 256), 256, 0, st>>>(dfom, ncand);
  // the candidate kernels read bands, E and the monitor entries G[N, j]: a one-row "G" with
  // leading dimension 0 makes G[N * 0 + j] = mon[j]
  gf::EvalArgs a;
  a.nlam = 1;
  a.dtype = GF_C128;
  a.nx = g.nx;
  a.ny = g.ny;
  a.chi = shard->geom.eps_mat - shard->geom.eps_bg;
  if (spec->kind == GF_KIND_SINGLE) {
    a.c_begin = (int64_t)g.y0 * g.nx;
    a.c_end = (int64_t)g.y1 * g.nx;
  } else {
    const int ye = g.y1 < g.ny - 1 ? g.y1 : g.ny - 1;      // anchors of rows [y0, ye)
    a.c_begin = (int64_t)g.y0 * (g.nx - 1);
    a.c_end = ye > g.y0 ? (int64_t)ye * (g.nx - 1) : a.c_begin;
  }
  a.lam[0].G = shard->mon;
  a.lam[0].ldg = 0;
  a.lam[0].E = reinterpret_cast<const gf::cplx*>(shard->E);
  a.lam[0].bands = reinterpret_cast<const gf::cplx*>(shard->bands);
  if (a.c_end > a.c_begin) gf::launch_eval(a, state, *spec, dfom, st);
  return gf::api_cuda_check(h, "gf_shard_eval launch");
}

gf_status gf_shard_gather_rows(gf_handle* h, const gf_shard* shard, int32_t dtype, const uint8_t* state,
                               const gf_cand_spec* spec, const int32_t* idx, const int32_t* status, void* panel,
                               int64_t ldp, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = check_shard(h, shard, dtype);
  if (s) return s;
  if ((s = gf::api_check_spec(h, &shard->geom, spec))) return s;
  const gf::ShardGeo g = geo_of(shard);
  if (!state || !idx || !status || !panel || ((uintptr_t)panel & 15u))
    return gf::api_fail_msg(h, GF_EINVAL, "state, idx, status and panel must be non-NULL, panel 16-byte aligned");
  if (ldp < g.n || (ldp & 1)) return gf::api_fail_msg(h, GF_EINVAL, "ldp must be even and >= n");
  const int pmax = (spec->kind == GF_KIND_SINGLE ? 1 : gf::kMaxPixelsPerCand) * spec->k;
  if (pmax > gf::kGatherMaxV) return gf::api_fail_msg(h, GF_EINVAL, "k too large for the row gather");
  cudaStream_t st = (cudaStream_t)stream;
  const double chi = shard->geom.eps_mat - shard->geom.eps_bg;
  const int blocks = gf::grid_of((int64_t)pmax * ldp, 256);
  if (dtype == GF_C128)
    gf::k_shard_gather<double2><<<blocks, 256, 0, st>>>(g, spec->kind, spec->dir_mask, spec->k, chi, state, idx, status,
                                                         reinterpret_cast<const double2*>(shard->G), shard->ldg, pmax,
                                                         reinterpret_cast<double2*>(panel), ldp);
  else
    gf::k_shard_gather<float2><<<blocks, 256, 0, st>>>(g, spec->kind, spec->dir_mask, spec->k, chi, state, idx, status,
                                                        reinterpret_cast<const float2*>(shard->G), shard->ldg, pmax,
                                                        reinterpret_cast<float2*>(panel), ldp);
  return gf::api_cuda_check(h, "gf_shard_gather_rows launch");
}

gf_status gf_shard_apply_update(gf_handle* h, const gf_shard* shard, int32_t dtype, uint8_t* state,
                                const gf_cand_spec* spec, const int32_t* idx, const void* panel, int64_t ldp,
                                int32_t* status, double* fom_out, int32_t* applied, void* ws, size_t ws_bytes,
                                void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = check_shard(h, shard, dtype);
  if (s) return s;
  if ((s = gf::api_check_spec(h, &shard->geom, spec))) return s;
  const gf::ShardGeo g = geo_of(shard);
  if (!state || !idx || !status || !fom_out || !panel || ((uintptr_t)panel & 15u))
    return gf::api_fail_msg(h, GF_EINVAL, "state, idx, status, fom_out and panel must be non-NULL, panel 16-byte aligned");
  if (ldp < g.n || (ldp & 1)) return gf::api_fail_msg(h, GF_EINVAL, "ldp must be even and >= n");
  const gf::WsLayout L = gf::ws_layout(shard->geom, 1, dtype, *spec);
  if (!ws || ((uintptr_t)ws & 255u)) return gf::api_fail_msg(h, GF_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < L.total) return gf::api_fail_msg(h, GF_ENOMEM, "workspace too small");
  gf::UpdArgs a;
  a.nlam = 1;
  a.dtype = dtype;
  a.nx = g.nx;
  a.ny = g.ny;
  a.chi = shard->geom.eps_mat - shard->geom.eps_bg;
  a.pmax = L.pmax;
  a.algo = gf::api_update_algo(h);
  a.sm_count = gf::api_sm_count(h);
  a.nz = 0;
  a.ncomp = 1;
  a.mrow = g.N;
  a.mcount = 1;
  a.lam[0].G = shard->G;
  a.lam[0].ldg = shard->ldg;
  a.lam[0].E = reinterpret_cast<gf::cplx*>(shard->E);
  a.lam[0].bands = reinterpret_cast<gf::cplx*>(shard->bands);
  a.lam[0].vrows = panel;
  a.lam[0].ldv = ldp;
  a.lam[0].rows = g.r1 - g.r0;
  cudaStream_t st = (cudaStream_t)stream;
  gf::launch_update(a, L, reinterpret_cast<char*>(ws), state, *spec, idx, status, fom_out, applied, st,
                    gf::api_timer(h));
  gf::k_shard_bands<<<gf::grid_of((int64_t)(GF_NBANDS + 1) * (g.y1 - g.y0) * g.nx, 256), 256, 0, st>>>(
      g, dtype, shard->G, shard->ldg, reinterpret_cast<gf::cplx*>(shard->bands), reinterpret_cast<gf::cplx*>(shard->mon));
  return gf::api_cuda_check(h, "gf_shard_apply_update launch");
}

gf_status gf_shard_pack_halo(gf_handle* h, const gf_shard* shard, void* out, void* stream) {
  if (!h) return GF_EINVAL;
  if (!shard || !shard->bands || !shard->mon || !out || ((uintptr_t)out & 15u))
    return gf::api_fail_msg(h, GF_EINVAL, "shard, its bands and mon, and out must be non-NULL (out 16-byte aligned)");
  if (gf_shard_rows(shard) <= 0) return gf::api_fail_msg(h, GF_EINVAL, "bad shard rows");
  gf_status s = gf::api_bind_device(h);
  if (s) return s;
  const gf::ShardGeo g = geo_of(shard);
  gf::k_shard_pack<<<gf::grid_of((int64_t)(GF_NBANDS + 1) * g.nx, 256), 256, 0, (cudaStream_t)stream>>>(
      g, g.y0, reinterpret_cast<const gf::cplx*>(shard->bands), reinterpret_cast<const gf::cplx*>(shard->mon),
      reinterpret_cast<gf::cplx*>(out));
  return gf::api_cuda_check(h, "gf_shard_pack_halo launch");
}

gf_status gf_shard_unpack_halo(gf_handle* h, const gf_shard* shard, const void* in, void* stream) {
  if (!h) return GF_EINVAL;
  if (!shard || !shard->bands || !shard->mon || !in || ((uintptr_t)in & 15u))
    return gf::api_fail_msg(h, GF_EINVAL, "shard, its bands and mon, and in must be non-NULL (in 16-byte aligned)");
  if (gf_shard_rows(shard) <= 0) return gf::api_fail_msg(h, GF_EINVAL, "bad shard rows");
  gf_status s = gf::api_bind_device(h);
  if (s) return s;
  const gf::ShardGeo g = geo_of(shard);
  if (g.y1 >= g.ny) return GF_OK;
  gf::k_shard_unpack<<<gf::grid_of((int64_t)(GF_NBANDS + 1) * g.nx, 256), 256, 0, (cudaStream_t)stream>>>(
      g, g.y1, reinterpret_cast<const gf::cplx*>(in), reinterpret_cast<gf::cplx*>(shard->bands),
      reinterpret_cast<gf::cplx*>(shard->mon));
  return gf::api_cuda_check(h, "gf_shard_unpack_halo launch");
}

}  // extern "C"
