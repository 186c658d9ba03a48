// Persistent batched step: one launch runs the stages of a greedy step (Fig. 1) for every problem
// of a batch as work items.  Each CTA takes the next item from a device queue (stage-major order,
// the largest problems first within a stage), waits -- bounded -- until the stage the item depends
// on has finished for its problem, runs the stage's body on a virtual block index, and counts the
// item done.  Problems proceed independently: a small problem's selection runs while a large one
// still evaluates, and no stage boundary drains the GPU.
//
// complex64 runs the whole step in this launch (evaluation, selection + capacitance, panels, the
// FP32 G update in R x 512 tiles, field/FOM, bands), or everything up to the field/FOM with the
// update and the bands as their own launches.  complex128 with small problems runs the whole step
// too, its G update the FP64 FMA form in 16 x 256 tiles; otherwise evaluation .. digit-operand
// preparation and the field/FOM, the warp-specialised tensor-core update and the bands following
// as their own launches.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "gf_internal.cuh"
#include "gf_stage_bodies.cuh"
#include "gf_tc.cuh"

namespace gf {

namespace {

__device__ __forceinline__ int ld_acquire_gpu(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu_add(int32_t* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Wait until *cnt >= need; gives up when another CTA has set *abort or after timeout_ns (then sets
// *abort so that every other waiter gives up too).  Called by one thread.
__device__ bool wait_done(const int32_t* cnt, int need, int32_t* abort, uint64_t timeout_ns) {
  if (ld_acquire_gpu(cnt) >= need) return true;
  const uint64_t t0 = tc::globaltimer_ns();
  for (;;) {
    __nanosleep(64);
    if (ld_acquire_gpu(cnt) >= need) return true;
    if (*reinterpret_cast<volatile int32_t*>(abort)) return false;
    if (tc::globaltimer_ns() - t0 > timeout_ns) {
      atomicExch(abort, 1);
      return false;
    }
  }
}

__device__ __forceinline__ void fill_eval_args(const BatchItem& it, int dtype, EvalArgs& a) {
  a.nlam = 1;
  a.dtype = dtype;
  a.nx = it.nx;
  a.ny = it.ny;
  a.chi = it.chi;
  a.c_begin = 0;
  a.c_end = -1;
  a.lam[0].G = it.G;
  a.lam[0].ldg = it.ldg;
  a.lam[0].E = it.E;
  a.lam[0].bands = it.bands;
}

}  // namespace

// R: rows of a complex64 update tile.  kBrush: 2x2-brush candidates (their evaluation needs about
// twice the registers of the single-pixel one, so the single-pixel form is held to two CTAs per SM).
template <int R, bool kBrush>
__global__ void __launch_bounds__(kBatchThreads, kBrush ? 1 : 2) k_batch_step(const __grid_constant__ BatchPlan P) {
  __shared__ EvalArgs s_ev;
  __shared__ CapArgs s_cap;
  __shared__ WsLayout s_L;
  __shared__ float2 sC[R][kC64Fp32MaxP];
  __shared__ int s_item, s_s, s_q, s_go;
  BatchSync* sy = P.sync;
  const int tid = threadIdx.x;
  // thread 0 keeps the CTA's next item in reserve, taken from the queue while the current one
  // runs (it is the next item this CTA runs, so every wait still goes to items that a running CTA
  // is processing or will process next: the one unfinished item with the smallest index never
  // waits, and the queue drains)
  int reserved = tid == 0 ? atomicAdd(&sy->next, 1) : 0;
  for (;;) {
    if (tid == 0) {
      const int t = reserved;
      if (t < P.total) reserved = atomicAdd(&sy->next, 1);
      int s = 0, q = 0, go = 0;
      if (t < P.total) {
        while (s + 1 < P.nstage && t >= P.first[s + 1][0]) ++s;
        int lo = 0, hi = P.nprob - 1;             // last queue position whose range starts at or before t
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (P.first[s][mid] <= t) lo = mid; else hi = mid - 1;
        }
        q = lo;
        const BatchItem& it = P.items[P.order[q]];
        const int d = P.dep[s];
        const int st = P.stage[s];
        const int need = d < 0 ? 0 : P.first[d][q + 1] - P.first[d][q] + (st == kStSelCap && q == P.stall_q);
        go = d < 0 || wait_done(&sy->done[q][d], need, &sy->abort, (uint64_t)P.timeout_ns);
        if (!go) {
          // the problem's step is abandoned: the update launches that follow skip it
          atomicExch(it.status, GF_ETIMEOUT);
          reinterpret_cast<UpdCtl*>(it.ws + it.L.ctl)->skip = 1;
        } else if (st == kStEval) {
          fill_eval_args(it, P.dtype, s_ev);
        } else if (st == kStSelCap || st == kStPanels || st == kStFinish) {
          batch_upd_args(it, P.dtype, s_cap.u);
          s_cap.kind = P.kind;
          s_cap.dir_mask = P.dir_mask;
          s_cap.k = 1;
          s_cap.pmax = it.L.pmax;
          s_L = it.L;
        }
      }
      s_item = t;
      s_s = s;
      s_q = q;
      s_go = go;
    }
    __syncthreads();
    const int t = s_item;
    if (t >= P.total) break;
    const int s = s_s, q = s_q;
    if (s_go) {
      const BatchItem& it = P.items[P.order[q]];
      const int64_t vb = t - P.first[s][q], vg = P.first[s][q + 1] - P.first[s][q];
      switch (P.stage[s]) {
        case kStEval:
          if constexpr (kBrush)
            eval_brush_body(s_ev, it.state, P.eval_mask, it.dfom, vb, vg);
          else
            eval_single_body(s_ev, it.state, P.eval_mask, it.dfom, vb, vg);
          break;
        case kStSelCap:
          batch_select_body(it, P.tie_rel);
          __syncthreads();
          capacitance_body(s_cap, s_L, it.ws, it.state, it.idx, it.status);
          break;
        case kStPanels:
          panels_body(s_cap.u, s_L, it.ws, 1, vb, vg);
          break;
        case kStPrep: {          // the table's fields are read directly (no argument block)
          char* ws = it.ws;
          const int64_t n = it.L.n;
          const UpdCtl* ctl = reinterpret_cast<const UpdCtl*>(ws + it.L.ctl);
          oz_prep_rows_body(reinterpret_cast<const cplx*>(ws + it.L.C0), it.L.pmax, n, ((n + kOzM - 1) / kOzM) * kOzM,
                            ctl, reinterpret_cast<uint8_t*>(ws + it.L.ozA), reinterpret_cast<int32_t*>(ws + it.L.ozE),
                            vb, vg);
          oz_prep_cols_body(reinterpret_cast<const cplx*>(ws + it.L.S), n, ((2 * n + kOzN - 1) / kOzN) * (kOzN / 2), ctl,
                            reinterpret_cast<uint8_t*>(ws + it.L.ozB), vb, vg);
          break;
        }
        case kStUpdate: {        // tiles [vb P.upd_tiles, (vb + 1) P.upd_tiles) of the problem
          char* ws = it.ws;
          const UpdCtl* ctl = reinterpret_cast<const UpdCtl*>(ws + it.L.ctl);
          const int p = ctl->skip ? 0 : ctl->nv;
          if (P.dtype == GF_C128) {
            if (p >= 1) {
              const int64_t n = it.L.n, nct = (n + 255) / 256, nt = ((n + kF64BatchRows - 1) / kF64BatchRows) * nct;
              double2* G = reinterpret_cast<double2*>(it.G);
              const cplx* C0 = reinterpret_cast<const cplx*>(ws + it.L.C0);
              const cplx* S = reinterpret_cast<const cplx*>(ws + it.L.S);
              for (int64_t tile = vb * P.upd_tiles; tile < (vb + 1) * P.upd_tiles && tile < nt; ++tile)
                f64_update_tile(G, it.ldg, n, it.L.pmax, p, C0, S, tile / nct, tile % nct);
            }
          } else if (p >= 1 && p <= kC64Fp32MaxP) {
            const int64_t n = it.L.n, nct = (n + kF32Cols - 1) / kF32Cols, nt = ((n + R - 1) / R) * nct;
            const int pmax = it.L.pmax;
            float2* G = reinterpret_cast<float2*>(it.G);
            const int64_t ldg = it.ldg;
            const cplx* C0 = reinterpret_cast<const cplx*>(ws + it.L.C0);
            const cplx* S = reinterpret_cast<const cplx*>(ws + it.L.S);
            for (int64_t tile = vb * P.upd_tiles; tile < (vb + 1) * P.upd_tiles && tile < nt; ++tile)
              c64_fp32_tile<R>(G, ldg, n, n, pmax, p, C0, S, tile / nct, tile % nct, sC);
          }
          break;
        }
        case kStFinish:
          finish_body(s_cap.u, s_L, it.ws, it.state, it.fom, it.applied, vb, vg);
          break;
        case kStBands:
          bands_body(it.nx, it.ny, P.dtype, it.G, it.ldg, it.bands, vb, vg);
          break;
        default:
          break;
      }
    }
    __syncthreads();
    if (tid == 0 && s_go) red_release_gpu_add(&sy->done[q][s], 1);
  }
  // leave; the last CTA out clears the block for the next launch (no other CTA touches it now)
  if (tid == 0) {
    __threadfence();
    s_go = atomicAdd(&sy->exited, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (s_go) {
    for (int i = tid; i < kBatchMax * kPlanStages; i += blockDim.x) (&sy->done[0][0])[i] = 0;
    if (tid == 0) {
      sy->next = 0;
      sy->abort = 0;
      sy->exited = 0;
    }
  }
}

// ----------------------------------------------------------------------------- host
static int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

void build_batch_plan(BatchPlan& P, const BatchItem* host_items, int nprob, int dtype, const gf_cand_spec& spec,
                      int scale, int rows, bool c128_fma) {
  P = BatchPlan{};
  P.nprob = nprob;
  P.dtype = dtype;
  P.kind = spec.kind;
  P.dir_mask = spec.dir_mask;
  P.eval_mask = spec.dir_mask | (spec.aligned ? kEvalAligned : 0);
  P.tie_rel = spec.tie_rel;
  P.timeout_ns = 2000000000ll;
  P.stall_q = -1;
  P.upd_tiles = scale;
  if (dtype == GF_C128 && c128_fma) {      // the whole step, the FP64 FMA update in the launch
    const int32_t st[] = {kStEval, kStSelCap, kStPanels, kStUpdate, kStFinish, kStBands};
    const int32_t dp[] = {-1, 0, 1, 2, 2, 3};
    P.nstage = 6;
    for (int s = 0; s < P.nstage; ++s) { P.stage[s] = st[s]; P.dep[s] = dp[s]; }
  } else if (dtype == GF_C128) {
    const int32_t st[] = {kStEval, kStSelCap, kStPanels, kStPrep, kStFinish};
    const int32_t dp[] = {-1, 0, 1, 2, 2};
    P.nstage = 5;
    for (int s = 0; s < P.nstage; ++s) { P.stage[s] = st[s]; P.dep[s] = dp[s]; }
  } else if (rows == 0) {      // complex64, the update and the bands as their own launches
    const int32_t st[] = {kStEval, kStSelCap, kStPanels, kStFinish};
    const int32_t dp[] = {-1, 0, 1, 2};
    P.nstage = 4;
    for (int s = 0; s < P.nstage; ++s) { P.stage[s] = st[s]; P.dep[s] = dp[s]; }
  } else {
    const int32_t st[] = {kStEval, kStSelCap, kStPanels, kStUpdate, kStFinish, kStBands};
    const int32_t dp[] = {-1, 0, 1, 2, 2, 3};
    P.nstage = 6;
    for (int s = 0; s < P.nstage; ++s) { P.stage[s] = st[s]; P.dep[s] = dp[s]; }
  }
  // queue order: the largest problems first (their chains of stages are the longest)
  std::vector<int> ord(nprob);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return host_items[a].L.n > host_items[b].L.n; });
  for (int q = 0; q < nprob; ++q) P.order[q] = ord[q];
  const int64_t per = (int64_t)kBatchThreads * scale;
  int64_t acc = 0;
  for (int s = 0; s < P.nstage; ++s) {
    for (int q = 0; q < nprob; ++q) {
      const BatchItem& it = host_items[P.order[q]];
      const int64_t n = it.L.n, N = (int64_t)it.nx * it.ny;
      int64_t c = 1;
      switch (P.stage[s]) {
        case kStEval:
          c = cdiv64(spec.kind == GF_KIND_SINGLE ? N : (int64_t)(it.nx - 1) * (it.ny - 1), per);
          break;
        case kStSelCap: c = 1; break;
        case kStPanels: c = cdiv64(n, per); break;
        case kStPrep: c = cdiv64(std::max(cdiv64(n, kOzM) * kOzM, cdiv64(2 * n, kOzN) * (kOzN / 2)), per); break;
        case kStUpdate:
          c = dtype == GF_C128 ? cdiv64(cdiv64(n, kF64BatchRows) * cdiv64(n, 256), P.upd_tiles)
                               : cdiv64(cdiv64(n, rows) * cdiv64(n, kF32Cols), P.upd_tiles);
          break;
        case kStFinish: c = cdiv64(n, per); break;
        case kStBands: c = cdiv64(N, per); break;
        default: break;
      }
      P.first[s][q] = (int32_t)acc;
      acc += c < 1 ? 1 : c;
    }
    P.first[s][nprob] = (int32_t)acc;
  }
  P.total = (int32_t)acc;
}

template <int R, bool kBrush>
static int ctas_per_sm_t() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_step<R, kBrush>, kBatchThreads, 0) != cudaSuccess) nb = 1;
  return nb < 1 ? 1 : nb;
}

int batch_step_ctas_per_sm(int rows, int kind) {
  const bool br = kind != GF_KIND_SINGLE;
  if (rows == 16) return br ? ctas_per_sm_t<16, true>() : ctas_per_sm_t<16, false>();
  if (rows == 64) return br ? ctas_per_sm_t<64, true>() : ctas_per_sm_t<64, false>();
  return br ? ctas_per_sm_t<32, true>() : ctas_per_sm_t<32, false>();
}

template <bool kBrush>
static void launch_t(const BatchPlan& P, int ctas, int rows, cudaStream_t st) {
  if (rows == 16)
    k_batch_step<16, kBrush><<<ctas, kBatchThreads, 0, st>>>(P);
  else if (rows == 64)
    k_batch_step<64, kBrush><<<ctas, kBatchThreads, 0, st>>>(P);
  else
    k_batch_step<32, kBrush><<<ctas, kBatchThreads, 0, st>>>(P);
}

void launch_batch_step(const BatchPlan& P, int ctas, int rows, cudaStream_t st) {
  if (P.kind == GF_KIND_SINGLE)
    launch_t<false>(P, ctas, rows, st);
  else
    launch_t<true>(P, ctas, rows, st);
}

}  // namespace gf
