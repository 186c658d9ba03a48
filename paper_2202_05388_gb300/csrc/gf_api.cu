// Host side of the libgfopt C ABI: handles, argument validation, workspace layout and the
// launch sequence of each call.  Every entry point validates all arguments before it
// enqueues anything and reports failures through its return value and gf_last_error().
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "gf_internal.cuh"

struct gf_handle {
  int device;
  int sm_count;
  int update_algo;
  char err[512];
  gf::KernelTimer timer;
};

void gf::KernelTimer::release() {
  for (int i = 0; i < max; ++i) {
    if (ev0) cudaEventDestroy(ev0[i]);
    if (ev1) cudaEventDestroy(ev1[i]);
  }
  delete[] ev0;
  delete[] ev1;
  delete[] n2;
  delete[] bytes_per_entry;
  if (p_host) cudaFreeHost(p_host);
  ev0 = ev1 = nullptr;
  n2 = nullptr;
  bytes_per_entry = nullptr;
  p_host = p_dev = nullptr;
  max = used = 0;
  on = false;
}

static thread_local char g_create_err[512] = "";

static gf_status fail(gf_handle* h, gf_status s, const char* fmt, ...) {
  char* buf = h ? h->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return s;
}

static gf_status cuda_check(gf_handle* h, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, GF_ECUDA, "%s: %s", where, cudaGetErrorString(e));
  return GF_OK;
}

static gf_status bind_device(gf_handle* h) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return cuda_check(h, "cudaGetDevice");
  if (cur != h->device && cudaSetDevice(h->device) != cudaSuccess) return cuda_check(h, "cudaSetDevice");
  return GF_OK;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static gf_status check_geom(gf_handle* h, const gf_geom* g) {
  if (!g) return fail(h, GF_EINVAL, "geometry is NULL");
  if (g->nx < 1 || g->ny < 1) return fail(h, GF_EINVAL, "nx, ny must be >= 1 (got %d, %d)", g->nx, g->ny);
  const int64_t N = (int64_t)g->nx * g->ny;
  if (N + 1 > (int64_t)INT32_MAX) return fail(h, GF_EINVAL, "N + 1 = %lld exceeds int32", (long long)(N + 1));
  if (!(g->dx > 0.0) || !isfinite(g->dx)) return fail(h, GF_EINVAL, "dx must be positive and finite");
  if (!(g->wavelength > 0.0) || !isfinite(g->wavelength))
    return fail(h, GF_EINVAL, "wavelength must be positive and finite");
  if (g->eps_bg != 1.0) return fail(h, GF_EINVAL, "eps_bg must be 1 (vacuum background G0)");
  if (!isfinite(g->eps_mat) || g->eps_mat == g->eps_bg) return fail(h, GF_EINVAL, "eps_mat must differ from eps_bg");
  if (!isfinite(g->mon_x) || !isfinite(g->mon_y)) return fail(h, GF_EINVAL, "monitor position not finite");
  const double X = g->nx * g->dx, Y = g->ny * g->dx;
  if (g->mon_x >= 0.0 && g->mon_x <= X && g->mon_y >= 0.0 && g->mon_y <= Y)
    return fail(h, GF_EINVAL, "monitor (%g, %g) lies inside the design region", g->mon_x, g->mon_y);
  return GF_OK;
}

static gf_status check_spec(gf_handle* h, const gf_geom* g, const gf_cand_spec* s) {
  if (!s) return fail(h, GF_EINVAL, "candidate spec is NULL");
  if (s->kind != GF_KIND_SINGLE && s->kind != GF_KIND_BRUSH2) return fail(h, GF_EINVAL, "unknown candidate kind %d", s->kind);
  if (s->dir_mask < 1 || s->dir_mask > 3) return fail(h, GF_EINVAL, "dir_mask must be 1, 2 or 3");
  if (s->k < 1 || s->k > 256) return fail(h, GF_EINVAL, "k must be in [1, 256]");
  if (s->excl_radius < 0) return fail(h, GF_EINVAL, "excl_radius must be >= 0");
  if (!(s->tie_rel >= 0.0) || !isfinite(s->tie_rel)) return fail(h, GF_EINVAL, "tie_rel must be >= 0");
  if (s->kind == GF_KIND_BRUSH2 && (g->nx < 2 || g->ny < 2))
    return fail(h, GF_EINVAL, "2x2 brushes need nx, ny >= 2");
  return GF_OK;
}

static gf_status check_problem(gf_handle* h, const gf_problem* p, int dtype, bool need_bands) {
  if (!p) return fail(h, GF_EINVAL, "problem is NULL");
  gf_status s = check_geom(h, &p->geom);
  if (s) return s;
  if (dtype != GF_C128 && dtype != GF_C64) return fail(h, GF_EINVAL, "unknown dtype %d", dtype);
  const int64_t n = (int64_t)p->geom.nx * p->geom.ny + 1;
  if (!p->G || !p->E) return fail(h, GF_EINVAL, "G and E must be non-NULL");
  if (need_bands && !p->bands) return fail(h, GF_EINVAL, "bands must be non-NULL");
  if (!aligned16(p->G) || !aligned16(p->E) || (p->bands && !aligned16(p->bands)))
    return fail(h, GF_EINVAL, "G, E and bands must be 16-byte aligned");
  if (p->ldg < n || (p->ldg & 1)) return fail(h, GF_EINVAL, "ldg (%lld) must be even and >= n (%lld)",
                                              (long long)p->ldg, (long long)n);
  return GF_OK;
}

static gf_status check_lams(gf_handle* h, const gf_problem* probs, int32_t nlam, int dtype) {
  if (!probs) return fail(h, GF_EINVAL, "problems array is NULL");
  if (nlam < 1 || nlam > gf::kMaxLam) return fail(h, GF_EINVAL, "nlam must be in [1, %d]", gf::kMaxLam);
  for (int l = 0; l < nlam; ++l) {
    gf_status s = check_problem(h, &probs[l], dtype, true);
    if (s) return s;
    const gf_geom &a = probs[0].geom, &b = probs[l].geom;
    if (a.nx != b.nx || a.ny != b.ny || a.dx != b.dx || a.mon_x != b.mon_x || a.mon_y != b.mon_y ||
        a.eps_mat != b.eps_mat)
      return fail(h, GF_EINVAL, "all wavelengths must share the grid, the monitor and eps_mat");
  }
  return GF_OK;
}

namespace gf {

// Host helpers shared with other translation units that add entry points.
gf_status api_check_problem(gf_handle* h, const gf_problem* p, int dtype) { return check_problem(h, p, dtype, true); }
gf_status api_bind_device(gf_handle* h) { return bind_device(h); }
gf_status api_cuda_check(gf_handle* h, const char* where) { return cuda_check(h, where); }
gf_status api_fail_msg(gf_handle* h, gf_status s, const char* msg) { return fail(h, s, "%s", msg); }
int api_device(const gf_handle* h) { return h->device; }
int api_sm_count(const gf_handle* h) { return h->sm_count; }
int api_update_algo(const gf_handle* h) { return h->update_algo; }
KernelTimer* api_timer(gf_handle* h) { return &h->timer; }
gf_status api_check_spec(gf_handle* h, const gf_geom* g, const gf_cand_spec* s) { return check_spec(h, g, s); }

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

WsLayout ws_layout(const gf_geom& g, int nlam, int dtype, const gf_cand_spec& spec) {
  const int64_t N = (int64_t)g.nx * g.ny;
  const int per = spec.kind == GF_KIND_SINGLE ? 1 : kMaxPixelsPerCand;
  return ws_layout_n(N + 1, 2 * N, per * (spec.k < 1 ? 1 : spec.k), nlam, dtype);
}

// n unknowns, a fill table of `table_entries` complex values, pmax unknowns per step
WsLayout ws_layout_n(int64_t n, int64_t table_entries, int pmax, int nlam, int dtype) {
  WsLayout L;
  L.n = n;
  L.pmax = pmax;
  size_t o = 0;
  L.ctl = o; o = up256(o + sizeof(UpdCtl));
  L.V = o; o = up256(o + sizeof(int32_t) * L.pmax);
  L.dchi = o; o = up256(o + sizeof(double) * L.pmax);
  L.sel = o; o = up256(o + topk_scratch_bytes());   // selection scratch: offset independent of nlam, dtype
  L.lu_s = up256(sizeof(cplx) * (size_t)L.pmax * L.pmax);
  L.piv_s = up256(sizeof(int32_t) * L.pmax);
  L.yd_s = up256(sizeof(cplx) * L.pmax);
  L.lu = o; o += L.lu_s * nlam;
  L.piv = o; o += L.piv_s * nlam;
  L.yd = o; o += L.yd_s * nlam;
  L.panel_s = up256(sizeof(cplx) * (size_t)L.n * L.pmax);
  L.C0 = o; o += L.panel_s * nlam;
  L.S = o; o += L.panel_s * nlam;
  const OzLayout oz = oz_layout(L.n);
  L.ozA = o; o = up256(o + oz.bytesA);
  L.ozE = o; o = up256(o + oz.bytesE);
  L.ozB = o; o = up256(o + oz.bytesB);
  L.ozF = o; o = up256(o + oz.bytesF);
  const C64Layout c6 = c64_layout(L.n, L.pmax);
  L.c64M = o; o = up256(o + c6.bytesM);
  L.c64A = o; o = up256(o + (dtype == GF_C64 ? c6.bytesA : 0));
  L.c64B = o; o = up256(o + (dtype == GF_C64 ? c6.bytesB : 0));
  L.c64E = o; o = up256(o + (dtype == GF_C64 ? c6.bytesE : 0));
  L.c64F = o; o = up256(o + (dtype == GF_C64 ? c6.bytesF : 0));
  L.total = o;
  // the fill's Toeplitz table reuses the start of the workspace
  L.table = 0;
  size_t tab = up256(sizeof(cplx) * (size_t)table_entries);
  if (tab > L.total) L.total = tab;
  return L;
}

}  // namespace gf

extern "C" {

const char* gf_version(void) { return "libgfopt 0.1 (sm_103a)"; }

const char* gf_status_string(gf_status s) {
  switch (s) {
    case GF_OK: return "ok";
    case GF_EINVAL: return "invalid argument";
    case GF_ECUDA: return "CUDA error";
    case GF_ESINGULAR: return "singular capacitance matrix";
    case GF_ENOIMPROVE: return "no candidate improves the FOM";
    case GF_ETIMEOUT: return "bounded wait timed out";
    case GF_ENOMEM: return "workspace too small";
    default: return "unknown status";
  }
}

gf_status gf_create(gf_handle** out, int32_t device) {
  if (!out) return fail(nullptr, GF_EINVAL, "handle pointer is NULL");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, GF_ECUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
  }
  if (device < 0 || device >= count) return fail(nullptr, GF_ECUDA, "device %d does not exist (%d devices)", device, count);
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return fail(nullptr, GF_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
  gf_handle* h = new (std::nothrow) gf_handle;
  if (!h) return fail(nullptr, GF_ENOMEM, "out of host memory");
  h->device = device;
  h->sm_count = sms;
  h->update_algo = GF_UPDATE_TC;
  h->err[0] = 0;
  *out = h;
  return GF_OK;
}

void gf_destroy(gf_handle* h) {
  if (!h) return;
  h->timer.release();
  delete h;
}

const char* gf_last_error(const gf_handle* h) { return h ? h->err : g_create_err; }

int64_t gf_num_candidates(const gf_geom* g, const gf_cand_spec* s) {
  if (!g || !s || g->nx < 1 || g->ny < 1) return 0;
  if (s->kind == GF_KIND_SINGLE) return (int64_t)g->nx * g->ny;
  if (g->nx < 2 || g->ny < 2) return 0;
  return 2 * (int64_t)(g->nx - 1) * (g->ny - 1);
}

size_t gf_workspace_size(const gf_geom* g, int32_t nlam, int32_t dtype, const gf_cand_spec* s) {
  if (!g || !s || nlam < 1 || nlam > gf::kMaxLam || g->nx < 1 || g->ny < 1) return 0;
  if (dtype != GF_C128 && dtype != GF_C64) return 0;
  return gf::ws_layout(*g, nlam, dtype, *s).total;
}

gf_status gf_fill_g0(gf_handle* h, const gf_problem* prob, int32_t dtype, void* ws, size_t ws_bytes,
                     void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = check_problem(h, prob, dtype, true);
  if (s) return s;
  const int64_t N = (int64_t)prob->geom.nx * prob->geom.ny;
  const size_t need = sizeof(gf::cplx) * (size_t)(2 * N);
  if (!ws || ((uintptr_t)ws & 255u)) return fail(h, GF_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need) return fail(h, GF_ENOMEM, "workspace has %zu bytes, fill needs %zu", ws_bytes, need);
  if ((s = bind_device(h))) return s;
  cudaStream_t st = (cudaStream_t)stream;
  gf::cplx* table = reinterpret_cast<gf::cplx*>(ws);
  gf::launch_fill_table(prob->geom, table, st);
  gf::launch_fill_expand(prob->geom, dtype, prob->G, prob->ldg, table, reinterpret_cast<gf::cplx*>(prob->E), st);
  gf::launch_bands(prob->geom, dtype, prob->G, prob->ldg, reinterpret_cast<gf::cplx*>(prob->bands), st);
  return cuda_check(h, "gf_fill_g0 launch");
}

gf_status gf_fom(gf_handle* h, const gf_problem* probs, int32_t nlam, int32_t dtype, double* fom_out, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = check_lams(h, probs, nlam, dtype);
  if (s) return s;
  if (!fom_out) return fail(h, GF_EINVAL, "fom_out must be non-NULL");
  if ((s = bind_device(h))) return s;
  gf::FomArgs a;
  a.nlam = nlam;
  a.ncomp = 1;
  a.mrow = (int64_t)probs[0].geom.nx * probs[0].geom.ny;
  for (int l = 0; l < nlam; ++l) a.E[l] = reinterpret_cast<const gf::cplx*>(probs[l].E);
  gf::launch_fom(a, fom_out, (cudaStream_t)stream);
  return cuda_check(h, "gf_fom launch");
}

gf_status gf_extract_bands(gf_handle* h, const gf_problem* prob, int32_t dtype, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = check_problem(h, prob, dtype, true);
  if (s) return s;
  if ((s = bind_device(h))) return s;
  gf::launch_bands(prob->geom, dtype, prob->G, prob->ldg, reinterpret_cast<gf::cplx*>(prob->bands),
                   (cudaStream_t)stream);
  return cuda_check(h, "gf_extract_bands launch");
}

gf_status gf_eval_candidates(gf_handle* h, const gf_problem* probs, int32_t nlam, int32_t dtype,
                             const uint8_t* state, const gf_cand_spec* spec, double* dfom, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = check_lams(h, probs, nlam, dtype);
  if (s) return s;
  if ((s = check_spec(h, &probs[0].geom, spec))) return s;
  if (!state || !dfom || !aligned16(dfom)) return fail(h, GF_EINVAL, "state and dfom must be non-NULL, dfom 16-byte aligned");
  if ((s = bind_device(h))) return s;
  gf::EvalArgs a;
  a.nlam = nlam;
  a.dtype = dtype;
  a.nx = probs[0].geom.nx;
  a.ny = probs[0].geom.ny;
  a.chi = probs[0].geom.eps_mat - probs[0].geom.eps_bg;
  a.c_begin = 0;
  a.c_end = -1;
  for (int l = 0; l < nlam; ++l) {
    a.lam[l].G = probs[l].G;
    a.lam[l].ldg = probs[l].ldg;
    a.lam[l].E = reinterpret_cast<const gf::cplx*>(probs[l].E);
    a.lam[l].bands = reinterpret_cast<const gf::cplx*>(probs[l].bands);
  }
  gf::launch_eval(a, state, *spec, dfom, (cudaStream_t)stream);
  return cuda_check(h, "gf_eval_candidates launch");
}

gf_status gf_select_topk(gf_handle* h, const gf_geom* geom, const gf_cand_spec* spec, const double* dfom,
                         int64_t ncand, int32_t* idx, double* val, int32_t* status, void* ws, size_t ws_bytes,
                         void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = check_geom(h, geom);
  if (s) return s;
  if ((s = check_spec(h, geom, spec))) return s;
  if (ncand != gf_num_candidates(geom, spec))
    return fail(h, GF_EINVAL, "ncand %lld does not match the candidate family (%lld)", (long long)ncand,
                (long long)gf_num_candidates(geom, spec));
  if (!dfom || !idx || !val || !status) return fail(h, GF_EINVAL, "dfom, idx, val and status must be non-NULL");
  if ((s = bind_device(h))) return s;
  // the greedy choice over many CTAs and the pooled top-k use the workspace's selection area when
  // a workspace is given
  void* sel = nullptr;
  if (ws) {
    const gf::WsLayout L = gf::ws_layout(*geom, 1, GF_C128, *spec);
    if (((uintptr_t)ws & 255u) == 0 && ws_bytes >= L.sel + gf::topk_scratch_bytes()) sel = (char*)ws + L.sel;
  }
  gf::launch_select(*geom, *spec, dfom, ncand, idx, val, status, sel, (cudaStream_t)stream);
  return cuda_check(h, "gf_select_topk launch");
}

gf_status gf_select_egreedy(gf_handle* h, const gf_geom* geom, const gf_cand_spec* spec, const double* dfom,
                            int64_t ncand, double epsilon, const double* u, int32_t* idx, double* val,
                            int32_t* status, void* ws, size_t ws_bytes, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = check_geom(h, geom);
  if (s) return s;
  if ((s = check_spec(h, geom, spec))) return s;
  if (spec->k != 1) return fail(h, GF_EINVAL, "the epsilon-greedy policy chooses one candidate (k = 1, got %d)", spec->k);
  if (ncand != gf_num_candidates(geom, spec))
    return fail(h, GF_EINVAL, "ncand %lld does not match the candidate family (%lld)", (long long)ncand,
                (long long)gf_num_candidates(geom, spec));
  if (!(epsilon >= 0.0 && epsilon <= 1.0)) return fail(h, GF_EINVAL, "epsilon must lie in [0, 1]");
  if (!dfom || !u || !idx || !val || !status) return fail(h, GF_EINVAL, "dfom, u, idx, val and status must be non-NULL");
  const gf::WsLayout L = gf::ws_layout(*geom, 1, GF_C128, *spec);
  if (!ws || ((uintptr_t)ws & 255u)) return fail(h, GF_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < L.sel + gf::topk_scratch_bytes())
    return fail(h, GF_ENOMEM, "workspace has %zu bytes, selection needs %zu", ws_bytes, L.sel + gf::topk_scratch_bytes());
  if ((s = bind_device(h))) return s;
  gf::launch_select_egreedy(*geom, *spec, dfom, ncand, epsilon, u, idx, val, status, (char*)ws + L.sel,
                            (cudaStream_t)stream);
  return cuda_check(h, "gf_select_egreedy launch");
}

gf_status gf_apply_update(gf_handle* h, const gf_problem* probs, int32_t nlam, int32_t dtype, uint8_t* state,
                          const gf_cand_spec* spec, const int32_t* idx, int32_t* status, double* fom_out,
                          int32_t* applied, void* ws, size_t ws_bytes, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = check_lams(h, probs, nlam, dtype);
  if (s) return s;
  if ((s = check_spec(h, &probs[0].geom, spec))) return s;
  if (!state || !idx || !status || !fom_out) return fail(h, GF_EINVAL, "state, idx, status and fom_out must be non-NULL");
  gf::WsLayout L = gf::ws_layout(probs[0].geom, nlam, dtype, *spec);
  if (!ws || ((uintptr_t)ws & 255u)) return fail(h, GF_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < L.total) return fail(h, GF_ENOMEM, "workspace has %zu bytes, update needs %zu", ws_bytes, L.total);
  if ((s = bind_device(h))) return s;
  gf::UpdArgs a;
  a.nlam = nlam;
  a.dtype = dtype;
  a.nx = probs[0].geom.nx;
  a.ny = probs[0].geom.ny;
  a.chi = probs[0].geom.eps_mat - probs[0].geom.eps_bg;
  a.pmax = L.pmax;
  a.algo = h->update_algo;
  a.sm_count = h->sm_count;
  a.nz = 0;
  a.ncomp = 1;
  a.mrow = L.n - 1;
  a.mcount = 1;
  for (int l = 0; l < nlam; ++l) {
    a.lam[l].G = probs[l].G;
    a.lam[l].ldg = probs[l].ldg;
    a.lam[l].E = reinterpret_cast<gf::cplx*>(probs[l].E);
    a.lam[l].bands = reinterpret_cast<gf::cplx*>(probs[l].bands);
    a.lam[l].vrows = nullptr;
    a.lam[l].ldv = 0;
    a.lam[l].rows = L.n;
  }
  cudaStream_t st = (cudaStream_t)stream;
  gf::launch_update(a, L, reinterpret_cast<char*>(ws), state, *spec, idx, status, fom_out, applied, st, &h->timer);
  for (int l = 0; l < nlam; ++l)
    gf::launch_bands(probs[l].geom, dtype, probs[l].G, probs[l].ldg, reinterpret_cast<gf::cplx*>(probs[l].bands), st);
  return cuda_check(h, "gf_apply_update launch");
}

size_t gf_refresh_workspace_size(const gf_geom* g, int32_t restart) {
  if (!g || g->nx < 1 || g->ny < 1 || g->nx > 4096 || g->ny > 4096 || restart < 1 || restart > 200) return 0;
  return gf::refresh_workspace_size(*g, restart);
}

gf_status gf_refresh(gf_handle* h, const gf_problem* prob, int32_t dtype, const uint8_t* state, int32_t nsample,
                     const int32_t* cols, int32_t restart, int32_t max_iter, double tol, double* resid_out,
                     int32_t* iters_out, double* colres_out, void* ws, size_t ws_bytes, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = check_problem(h, prob, dtype, false);
  if (s) return s;
  if (prob->geom.nx > 4096 || prob->geom.ny > 4096) return fail(h, GF_EINVAL, "gf_refresh supports nx, ny <= 4096");
  if (!state || !resid_out) return fail(h, GF_EINVAL, "state and resid_out must be non-NULL");
  if (nsample < 0 || (nsample > 0 && !cols)) return fail(h, GF_EINVAL, "nsample must be >= 0 with a cols array");
  if (restart < 1 || restart > 200) return fail(h, GF_EINVAL, "restart must be in [1, 200]");
  if (max_iter < 1) return fail(h, GF_EINVAL, "max_iter must be >= 1");
  if (!(tol > 0.0) || !isfinite(tol)) return fail(h, GF_EINVAL, "tol must be positive");
  const int64_t n = (int64_t)prob->geom.nx * prob->geom.ny + 1;
  for (int q = 0; q < nsample; ++q)
    if (cols[q] < 0 || cols[q] >= n) return fail(h, GF_EINVAL, "column %d out of range", cols[q]);
  const size_t need = gf::refresh_workspace_size(prob->geom, restart);
  if (!ws || ((uintptr_t)ws & 255u)) return fail(h, GF_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need) return fail(h, GF_ENOMEM, "workspace has %zu bytes, refresh needs %zu", ws_bytes, need);
  if ((s = bind_device(h))) return s;
  s = gf::refresh(*prob, dtype, state, nsample, cols, restart, max_iter, tol, resid_out, iters_out, colres_out,
                  reinterpret_cast<char*>(ws), (cudaStream_t)stream);
  if (s) return cuda_check(h, "gf_refresh");
  return GF_OK;
}

gf_status gf_refresh_field(gf_handle* h, const gf_problem* prob, int32_t dtype, const uint8_t* state, double e_tol,
                           int32_t restart, int32_t max_iter, double tol, gf_refresh_report* report, void* ws,
                           size_t ws_bytes, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = check_problem(h, prob, dtype, false);
  if (s) return s;
  if (prob->geom.nx > 4096 || prob->geom.ny > 4096) return fail(h, GF_EINVAL, "gf_refresh_field supports nx, ny <= 4096");
  if (!state || !report) return fail(h, GF_EINVAL, "state and report must be non-NULL");
  if (restart < 1 || restart > 200) return fail(h, GF_EINVAL, "restart must be in [1, 200]");
  if (max_iter < 1) return fail(h, GF_EINVAL, "max_iter must be >= 1");
  if (!(tol > 0.0) || !isfinite(tol)) return fail(h, GF_EINVAL, "tol must be positive");
  if (!(e_tol >= 0.0) || !isfinite(e_tol)) return fail(h, GF_EINVAL, "e_tol must be >= 0");
  const size_t need = gf::refresh_workspace_size(prob->geom, restart);
  if (!ws || ((uintptr_t)ws & 255u)) return fail(h, GF_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need) return fail(h, GF_ENOMEM, "workspace has %zu bytes, refresh needs %zu", ws_bytes, need);
  if ((s = bind_device(h))) return s;
  s = gf::refresh_field(*prob, state, e_tol, restart, max_iter, tol, report, reinterpret_cast<char*>(ws),
                        (cudaStream_t)stream);
  if (s) return cuda_check(h, "gf_refresh_field");
  return GF_OK;
}

gf_status gf_set_update_algo(gf_handle* h, int32_t algo) {
  if (!h) return GF_EINVAL;
  if (algo != GF_UPDATE_TC && algo != GF_UPDATE_DFMA && algo != GF_UPDATE_TENSOR)
    return fail(h, GF_EINVAL, "unknown update algorithm %d", algo);
  h->update_algo = algo;
  return GF_OK;
}

gf_status gf_profile_begin(gf_handle* h, int32_t max_records) {
  if (!h) return GF_EINVAL;
  if (max_records < 1 || max_records > (1 << 20)) return fail(h, GF_EINVAL, "max_records must be in [1, 2^20]");
  gf_status s = bind_device(h);
  if (s) return s;
  h->timer.release();
  gf::KernelTimer& t = h->timer;
  t.ev0 = new (std::nothrow) cudaEvent_t[max_records];
  t.ev1 = new (std::nothrow) cudaEvent_t[max_records];
  t.n2 = new (std::nothrow) double[max_records];
  t.bytes_per_entry = new (std::nothrow) int[max_records];
  if (!t.ev0 || !t.ev1 || !t.n2 || !t.bytes_per_entry) { t.release(); return fail(h, GF_ENOMEM, "out of host memory"); }
  for (int i = 0; i < max_records; ++i) {
    if (cudaEventCreate(&t.ev0[i]) != cudaSuccess || cudaEventCreate(&t.ev1[i]) != cudaSuccess) {
      t.max = i;
      t.release();
      return cuda_check(h, "cudaEventCreate");
    }
    t.max = i + 1;
  }
  if (cudaHostAlloc((void**)&t.p_host, sizeof(int32_t) * max_records, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&t.p_dev, t.p_host, 0) != cudaSuccess) {
    t.p_host = nullptr;
    t.release();
    return cuda_check(h, "cudaHostAlloc(mapped)");
  }
  memset(t.p_host, 0, sizeof(int32_t) * max_records);
  t.used = 0;
  t.on = true;
  return GF_OK;
}

gf_status gf_profile_end(gf_handle* h, double* ms_total, int64_t* launches, double* bytes_total,
                         double* flops_total) {
  if (!h) return GF_EINVAL;
  gf::KernelTimer& t = h->timer;
  if (!t.on) return fail(h, GF_EINVAL, "profiling is not armed");
  gf_status s = bind_device(h);
  if (s) return s;
  double ms = 0.0, bytes = 0.0, flops = 0.0;
  int64_t count = 0;
  if (t.used > 0 && cudaEventSynchronize(t.ev1[t.used - 1]) != cudaSuccess) {
    t.release();
    return cuda_check(h, "cudaEventSynchronize");
  }
  for (int i = 0; i < t.used; ++i) {
    float e = 0.f;
    if (cudaEventElapsedTime(&e, t.ev0[i], t.ev1[i]) != cudaSuccess) {
      t.release();
      return cuda_check(h, "cudaEventElapsedTime");
    }
    const int p = ((volatile int32_t*)t.p_host)[i];
    if (p <= 0) continue;         // a skipped (no-op) launch is not a G update
    ms += e;
    ++count;
    bytes += t.n2[i] * t.bytes_per_entry[i];
    flops += 8.0 * p * t.n2[i];
  }
  if (ms_total) *ms_total = ms;
  if (launches) *launches = count;
  if (bytes_total) *bytes_total = bytes;
  if (flops_total) *flops_total = flops;
  t.release();
  return GF_OK;
}

}  // extern "C"
