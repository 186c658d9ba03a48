// Host side of the batch entry points: many independent single-wavelength problems advanced
// together through the greedy step (Fig. 1: evaluate every candidate, select, update), either
// by the persistent step kernel (default; gf_batch_step.cu) or by one launch per stage.  The item
// table and the persistent kernel's queue and phase counters live in caller-owned device memory;
// the complex128 update's TMA descriptors live in a host parameter block that every step passes
// to the persistent tensor-core launch.
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "gf_internal.cuh"

struct gf_batch {
  gf_handle* h;
  int nitems;
  int dtype;
  gf_cand_spec spec;
  gf::BatchItem* table;            // device
  std::vector<gf::BatchItem> host; // host copy
  void* oz_params;                 // complex128: parameter block of the persistent update
  int64_t widest_n, widest_N, widest_units;
  int update_ctas;
  int form;                        // GF_BATCH_PERSISTENT or GF_BATCH_STAGED
  bool c128_fma;                   // complex128 with the FP64 FMA update (every problem small, or
                                   // GF_UPDATE_DFMA), else the tensor-core update
  int step_ctas, scale, tile_rows; // launch shape of the persistent step (step_ctas 0: fill the GPU)
  gf::BatchPlan plan;
};

static size_t items_bytes(int32_t nitems) { return ((size_t)nitems * sizeof(gf::BatchItem) + 255) & ~(size_t)255; }
static size_t sync_bytes() { return (sizeof(gf::BatchSync) + 255) & ~(size_t)255; }

static gf_status bfail(gf_handle* h, gf_status s, const char* fmt, int a = 0, long long b = 0, long long c = 0) {
  char msg[256];
  snprintf(msg, sizeof msg, fmt, a, b, c);
  return gf::api_fail_msg(h, s, msg);
}

extern "C" {

size_t gf_batch_table_size(int32_t nitems) {
  if (nitems < 1 || nitems > gf::kBatchMax) return 0;
  return items_bytes(nitems) + sync_bytes();
}

gf_status gf_batch_create(gf_handle* h, int32_t nitems, const gf_batch_item* items, int32_t dtype,
                          const gf_cand_spec* spec, void* table, size_t table_bytes, void* stream,
                          gf_batch** out) {
  if (!h) return GF_EINVAL;
  if (!out) return bfail(h, GF_EINVAL, "output pointer is NULL");
  *out = nullptr;
  if (nitems < 1 || nitems > gf::kBatchMax) return bfail(h, GF_EINVAL, "nitems must be in [1, %d]", gf::kBatchMax);
  if (!items) return bfail(h, GF_EINVAL, "items array is NULL");
  if (dtype != GF_C128 && dtype != GF_C64) return bfail(h, GF_EINVAL, "unknown dtype %d", dtype);
  if (!spec) return bfail(h, GF_EINVAL, "candidate spec is NULL");
  if (spec->k != 1) return bfail(h, GF_EINVAL, "batches take k = 1 (got %d)", spec->k);
  if (!table || ((uintptr_t)table & 255u)) return bfail(h, GF_EINVAL, "table must be non-NULL and 256-byte aligned");
  if (table_bytes < gf_batch_table_size(nitems))
    return bfail(h, GF_ENOMEM, "table has %d bytes too few", (int)(gf_batch_table_size(nitems) - table_bytes));
  gf_batch* b = new (std::nothrow) gf_batch;
  if (!b) return bfail(h, GF_ENOMEM, "out of host memory");
  b->h = h;
  b->nitems = nitems;
  b->dtype = dtype;
  b->spec = *spec;
  b->table = reinterpret_cast<gf::BatchItem*>(table);
  b->oz_params = nullptr;
  b->widest_n = b->widest_N = b->widest_units = 0;
  b->update_ctas = 0;
  b->form = GF_BATCH_PERSISTENT;
  b->step_ctas = 0;
  b->scale = 1;
  b->tile_rows = 32;
  b->host.resize(nitems);
  for (int i = 0; i < nitems; ++i) {
    const gf_batch_item& it = items[i];
    gf_status s = gf::api_check_problem(h, &it.prob, dtype);
    if (!s) s = gf::api_check_spec(h, &it.prob.geom, spec);
    if (s) { delete b; return s; }
    if (!it.state || !it.dfom || !it.idx || !it.val || !it.status || !it.fom_out) {
      delete b;
      return bfail(h, GF_EINVAL, "item %d: state, dfom, idx, val, status and fom_out must be non-NULL", i);
    }
    const gf::WsLayout L = gf::ws_layout(it.prob.geom, 1, dtype, *spec);
    if (!it.ws || ((uintptr_t)it.ws & 255u)) {
      delete b;
      return bfail(h, GF_EINVAL, "item %d: workspace must be non-NULL and 256-byte aligned", i);
    }
    if (it.ws_bytes < L.total) {
      delete b;
      return bfail(h, GF_ENOMEM, "item %d: workspace has %lld bytes, needs %lld", i, (long long)it.ws_bytes,
                   (long long)L.total);
    }
    if (!(it.epsilon >= 0.0 && it.epsilon <= 1.0)) {
      delete b;
      return bfail(h, GF_EINVAL, "item %d: epsilon must lie in [0, 1]", i);
    }
    if (it.epsilon > 0.0 && (!it.uniforms || !it.step || it.horizon < 1)) {
      delete b;
      return bfail(h, GF_EINVAL, "item %d: the epsilon-greedy policy needs uniforms, a step counter and horizon >= 1", i);
    }
    gf::BatchItem& d = b->host[i];
    d.G = it.prob.G;
    d.ldg = it.prob.ldg;
    d.E = reinterpret_cast<gf::cplx*>(it.prob.E);
    d.bands = reinterpret_cast<gf::cplx*>(it.prob.bands);
    d.nx = it.prob.geom.nx;
    d.ny = it.prob.geom.ny;
    d.chi = it.prob.geom.eps_mat - it.prob.geom.eps_bg;
    d.ws = reinterpret_cast<char*>(it.ws);
    d.L = L;
    d.state = it.state;
    d.dfom = it.dfom;
    d.ncand = gf_num_candidates(&it.prob.geom, spec);
    d.idx = it.idx;
    d.val = it.val;
    d.status = it.status;
    d.fom = it.fom_out;
    d.applied = it.applied;
    d.epsilon = it.epsilon;
    d.uniforms = it.uniforms;
    d.step = it.step;
    d.horizon = it.horizon;
    const int64_t N = (int64_t)d.nx * d.ny;
    const int64_t units = spec->kind == GF_KIND_SINGLE ? N : (int64_t)(d.nx - 1) * (d.ny - 1);
    if (N + 1 > b->widest_n) b->widest_n = N + 1;
    if (N > b->widest_N) b->widest_N = N;
    if (units > b->widest_units) b->widest_units = units;
  }
  gf_status s = gf::api_bind_device(h);
  if (s) { delete b; return s; }
  // the update arithmetic follows the handle's setting: GF_UPDATE_DFMA the FP64 FMA form;
  // GF_UPDATE_TC that form when the whole batch is small (the sum of n^2 p_max within
  // kC128SmallWork, so every problem is small too and a single problem would take it as well),
  // else the tensor cores; GF_UPDATE_TENSOR the tensor cores
  b->c128_fma = false;
  if (dtype == GF_C128) {
    const int algo = gf::api_update_algo(h);
    double work = 0.0;
    for (int i = 0; i < nitems; ++i) {
      const double n = (double)b->host[i].L.n;
      work += n * n * b->host[i].L.pmax;
    }
    b->c128_fma = algo == GF_UPDATE_DFMA || (algo == GF_UPDATE_TC && work <= gf::kC128SmallWork);
  }
  if (dtype == GF_C128 && !b->c128_fma) {
    b->oz_params = ::operator new(gf::ozaki_batch_params_bytes(), std::align_val_t(64), std::nothrow);
    if (!b->oz_params) { delete b; return bfail(h, GF_ENOMEM, "out of host memory"); }
    if (!gf::ozaki_batch_params(b->oz_params, b->host.data(), nitems)) {
      ::operator delete(b->oz_params, std::align_val_t(64));
      delete b;
      return bfail(h, GF_ECUDA, "cannot encode the TMA descriptors of the batch (driver entry point missing)");
    }
  }
  gf::build_batch_plan(b->plan, b->host.data(), nitems, dtype, *spec, b->scale, b->tile_rows, b->c128_fma);
  b->plan.items = b->table;
  b->plan.sync = reinterpret_cast<gf::BatchSync*>(reinterpret_cast<char*>(table) + items_bytes(nitems));
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemcpyAsync(table, b->host.data(), sizeof(gf::BatchItem) * (size_t)nitems, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(b->plan.sync, 0, sizeof(gf::BatchSync), st);
  cudaStreamSynchronize(st);
  s = gf::api_cuda_check(h, "gf_batch_create upload");
  if (s) {
    gf_batch_destroy(b);
    return s;
  }
  *out = b;
  return GF_OK;
}

gf_status gf_batch_set_schedule(gf_batch* b, int32_t update_ctas) {
  if (!b) return GF_EINVAL;
  if (update_ctas < 0 || update_ctas > 65535) return bfail(b->h, GF_EINVAL, "update_ctas must be in [0, 65535]");
  b->update_ctas = update_ctas;
  return GF_OK;
}

gf_status gf_batch_set_form(gf_batch* b, int32_t form, int32_t step_ctas, int32_t scale, int32_t tile_rows) {
  if (!b) return GF_EINVAL;
  if (form != GF_BATCH_PERSISTENT && form != GF_BATCH_STAGED) return bfail(b->h, GF_EINVAL, "unknown form %d", form);
  if (step_ctas < 0 || step_ctas > 65535) return bfail(b->h, GF_EINVAL, "step_ctas must be in [0, 65535]");
  if (scale < 1 || scale > 16) return bfail(b->h, GF_EINVAL, "scale must be in [1, 16] (got %d)", scale);
  if (tile_rows != 0 && tile_rows != 16 && tile_rows != 32 && tile_rows != 64)
    return bfail(b->h, GF_EINVAL, "tile_rows must be 0, 16, 32 or 64 (got %d)", tile_rows);
  b->form = form;
  b->step_ctas = step_ctas;
  b->scale = scale;
  b->tile_rows = tile_rows;
  gf::BatchPlan P;
  gf::build_batch_plan(P, b->host.data(), b->nitems, b->dtype, b->spec, scale, tile_rows, b->c128_fma);
  P.items = b->plan.items;
  P.sync = b->plan.sync;
  b->plan = P;
  return GF_OK;
}

static void persistent_step(gf_batch* b, const gf::BatchPlan& plan, cudaStream_t st) {
  const int sms = gf::api_sm_count(b->h);
  const int ctas = b->step_ctas > 0 ? b->step_ctas : sms * gf::batch_step_ctas_per_sm(b->tile_rows, b->spec.kind);
  gf::launch_batch_step(plan, ctas, b->tile_rows, st);
  if (b->dtype == GF_C128 && !b->c128_fma) {
    gf::launch_rank_update_ozaki_batch(b->oz_params, b->update_ctas > 0 ? b->update_ctas : sms, st);
    gf::launch_bands_batch(b->table, b->nitems, b->dtype, b->widest_N, st);
  } else if (b->tile_rows == 0) {
    gf::launch_rank_update_c64_fp32_batch(b->table, b->nitems, b->update_ctas > 0 ? b->update_ctas : 3 * sms, st);
    gf::launch_bands_batch(b->table, b->nitems, b->dtype, b->widest_N, st);
  }
}

gf_status gf_batch_selftest_timeout(gf_batch* b, int64_t timeout_ns, void* stream) {
  if (!b) return GF_EINVAL;
  if (timeout_ns < 1000 || timeout_ns > 2000000000ll)
    return bfail(b->h, GF_EINVAL, "timeout_ns must be in [1 us, 2 s]");
  gf_status s = gf::api_bind_device(b->h);
  if (s) return s;
  gf::BatchPlan P = b->plan;
  P.timeout_ns = timeout_ns;
  P.stall_q = 0;
  persistent_step(b, P, (cudaStream_t)stream);
  return gf::api_cuda_check(b->h, "gf_batch_selftest_timeout launch");
}

gf_status gf_batch_step(gf_batch* b, void* stream) {
  if (!b) return GF_EINVAL;
  gf_status s = gf::api_bind_device(b->h);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = b->nitems;
  const int sms = gf::api_sm_count(b->h);
  if (b->form == GF_BATCH_PERSISTENT) {
    persistent_step(b, b->plan, st);
    return gf::api_cuda_check(b->h, "gf_batch_step launch");
  }
  gf::launch_eval_batch(b->table, n, b->dtype, b->spec, b->widest_units, st);
  gf::launch_select_batch(b->table, n, b->spec.tie_rel, st);
  gf::launch_capacitance_batch(b->table, n, b->dtype, b->spec, st);
  gf::launch_panels_batch(b->table, n, b->dtype, b->widest_n, st);
  if (b->dtype == GF_C128 && b->c128_fma) {
    gf::launch_rank_update_f64_batch(b->table, n, b->widest_n, st);
  } else if (b->dtype == GF_C128) {
    gf::launch_oz_prep_batch(b->table, n, b->widest_n, st);
    gf::launch_rank_update_ozaki_batch(b->oz_params, b->update_ctas > 0 ? b->update_ctas : sms, st);
  } else {
    gf::launch_rank_update_c64_fp32_batch(b->table, n, b->update_ctas > 0 ? b->update_ctas : 3 * sms, st);
  }
  gf::launch_finish_batch(b->table, n, b->dtype, b->widest_n, st);
  gf::launch_bands_batch(b->table, n, b->dtype, b->widest_N, st);
  return gf::api_cuda_check(b->h, "gf_batch_step launch");
}

void gf_batch_destroy(gf_batch* b) {
  if (!b) return;
  if (b->oz_params) ::operator delete(b->oz_params, std::align_val_t(64));
  delete b;
}

}  // extern "C"
