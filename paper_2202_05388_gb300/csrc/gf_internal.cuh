// Internal declarations shared by the libgfopt translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/gfopt.h"

namespace gf {

// ----------------------------------------------------------------------------- complex
struct cplx {
  double re, im;
};

__host__ __device__ __forceinline__ cplx mk(double r, double i) { return cplx{r, i}; }
__host__ __device__ __forceinline__ cplx operator+(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ cplx operator-(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cplx operator*(cplx a, cplx b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cplx operator*(double s, cplx a) { return {s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ double abs2(cplx a) { return a.re * a.re + a.im * a.im; }
__host__ __device__ __forceinline__ double cabs1(cplx a) { return sqrt(abs2(a)); }
// a / b by scaling with 1/|b|^2 (b is a pivot bounded away from 0 by the singularity test)
__host__ __device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  double d = 1.0 / abs2(b);
  return {(a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d};
}
// cdiv with the reciprocal d = 1 / |b|^2 formed beforehand (the same bits as cdiv(a, b))
__host__ __device__ __forceinline__ cplx cdiv_r(cplx a, cplx b, double d) {
  return {(a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d};
}
// acc + a*b with fused multiply-adds
__device__ __forceinline__ cplx cfma(cplx a, cplx b, cplx acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}

// 1 / v for a positive normal v whose reciprocal is normal: Newton's iteration y <- y + y (1 - m y)
// on the mantissa m in [1, 2), seeded with the correctly rounded FP32 reciprocal of m (relative
// error <= 2^-24, squared by each step: two steps reach the FP64 rounding), then scaled by the
// exact power of two.  Six FP64 operations instead of the division routine, which sits on the
// per-column critical path of the pivoting and costs microseconds on GB300's narrow FP64 pipe.
// Error <= 1 ulp; correctly rounded for random mantissas in the CPU model of these operations (not
// at every value: just above a power of two the result may round to that power).  The pivot
// reciprocal of the capacitance factorisations, one CTA or a cluster (so they agree bit for bit).
__device__ __forceinline__ double rcp_nr(double v) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  const double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
  double y = (double)__frcp_rn((float)m);
  double r = fma(-m, y, 1.0);
  y = fma(y, r, y);
  r = fma(-m, y, 1.0);
  y = fma(y, r, y);
  return y * __longlong_as_double((long long)(1023 - e) << 52);
}

// The same iteration seeded without FP64 conversions (which run on GB300's narrow FP64 pipe): the
// FP32 reciprocal of m truncated to 24 bits (relative error <= 2^-23 before the FP32 rounding,
// so the seed is within 2^-22 and two steps still reach the FP64 rounding), its bits moved into
// an FP64 pattern by integer operations.  Four FP64 operations on the chain instead of six.
// Error <= 1 ulp; correctly rounded for random mantissas in the CPU model of these operations.
// The pivot reciprocal of the cluster factorisation.
__device__ __forceinline__ double rcp_nr_i(double v) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  const double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
  const float yf = __frcp_rn(__int_as_float(0x3F800000 | (int)((b >> 29) & 0x7FFFFF)));   // in (0.5, 1]
  const int fb = __float_as_int(yf);
  double y = __longlong_as_double(((long long)(((fb >> 23) & 0xFF) + (1023 - 127)) << 52) |
                                  ((long long)(fb & 0x7FFFFF) << 29));
  double r = fma(-m, y, 1.0);
  y = fma(y, r, y);
  r = fma(-m, y, 1.0);
  y = fma(y, r, y);
  return y * __longlong_as_double((long long)(1023 - e) << 52);
}

// a - l u with fused multiply-adds: the elimination step (and forward solve) of the capacitance
// factorisations, in one CTA or over a cluster, which therefore agree bit for bit
__device__ __forceinline__ cplx cfms(cplx l, cplx u, cplx a) { return cfma(mk(-l.re, -l.im), u, a); }

__device__ __forceinline__ cplx ldc(const void* base, int64_t idx) {
  double2 v = reinterpret_cast<const double2*>(base)[idx];
  return {v.x, v.y};
}
__device__ __forceinline__ void stc(void* base, int64_t idx, cplx v) {
  reinterpret_cast<double2*>(base)[idx] = make_double2(v.re, v.im);
}
// G entry (i, j) of either storage type, widened to FP64
__device__ __forceinline__ cplx ldG(const void* G, int32_t dtype, int64_t ldg, int64_t i, int64_t j) {
  if (dtype == GF_C128) return ldc(G, i * ldg + j);
  float2 v = reinterpret_cast<const float2*>(G)[i * ldg + j];
  return {(double)v.x, (double)v.y};
}

// ----------------------------------------------------------------------------- constants
constexpr double kSingularRel = 1e-13;     // |pivot| < kSingularRel * ||A||_inf => singular
constexpr int kMaxPixelsPerCand = 4;       // 2x2 brush

// Band offsets in pixel units (dx, dy), matching the ABI's off_b list.
__host__ __device__ __forceinline__ void band_offset(int b, int& ddx, int& ddy) {
  const int tx[GF_NBANDS] = {0, 1, -1, -1, 1, 0, 0, 1, -1};
  const int ty[GF_NBANDS] = {0, 0, 0, 1, -1, 1, -1, 1, -1};
  ddx = tx[b];
  ddy = ty[b];
}

// Unknowns and contrast changes of candidate c given the current state (same rule as the
// candidate kernels).  Appends to V/dchi; returns the number appended.  2-D (nz = 0): single
// pixels and 2x2 brushes, one unknown per pixel.  3-D (nz >= 1, kind GF_KIND_PILLAR): the 2x2
// lateral block through all nz layers, three unknowns (x, y, z) per flipped voxel, voxel-major.
__device__ __forceinline__ int cand_pixels(int64_t c, int kind, int dir_mask, int nx, int ny, double chi,
                                           const uint8_t* state, int32_t* V, double* dchi, int nz = 0) {
  const int64_t N = (int64_t)nx * ny;
  if (kind == GF_KIND_SINGLE) {
    if (c < 0 || c >= N) return 0;
    uint8_t s = state[c];
    if (s == 0 && (dir_mask & GF_DIR_FILL)) { V[0] = (int32_t)c; dchi[0] = chi; return 1; }
    if (s != 0 && (dir_mask & GF_DIR_CLEAR)) { V[0] = (int32_t)c; dchi[0] = -chi; return 1; }
    return 0;
  }
  const int64_t P = (int64_t)(nx - 1) * (ny - 1);
  if (c < 0 || c >= 2 * P) return 0;
  const int dir = (int)(c / P);
  const int64_t a = c - dir * P;
  if (!(dir_mask & (dir == 0 ? GF_DIR_FILL : GF_DIR_CLEAR))) return 0;
  const int ay = (int)(a / (nx - 1)), ax = (int)(a - (int64_t)ay * (nx - 1));
  const uint8_t target = dir == 0 ? 0 : 1;
  const double d = dir == 0 ? chi : -chi;
  int m = 0;
  if (kind == GF_KIND_PILLAR) {
    for (int iz = 0; iz < nz; ++iz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int64_t j = ((int64_t)iz * ny + ay + dy) * nx + ax + dx;
          if (state[j] != target) continue;
          for (int comp = 0; comp < 3; ++comp) {
            V[m] = (int32_t)(3 * j + comp);
            dchi[m] = d;
            ++m;
          }
        }
    return m;
  }
  const int64_t j0 = (int64_t)ay * nx + ax;
  const int64_t q[4] = {j0, j0 + 1, j0 + nx, j0 + nx + 1};
  for (int u = 0; u < 4; ++u) {
    if (state[q[u]] == target) {
      V[m] = (int32_t)q[u];
      dchi[m] = d;
      ++m;
    }
  }
  return m;
}

// ----------------------------------------------------------------------------- workspace
// Per-step control block written by the capacitance kernel, read by the panel/update kernels.
constexpr int kMaxLamCtl = 8;  // wavelengths per problem (kMaxLam)
struct UpdCtl {
  int32_t skip;       // 1: nothing is applied this step
  int32_t nv;         // number of flipped pixels (0 < nv <= pmax)
  int32_t ncand;      // number of candidates applied
  int32_t pad;
  double joint_dfom;  // dFOM of the applied set (FP64)
  double lam_df[kMaxLamCtl];     // per-wavelength dFOM of the joint set (parallel capacitance solve)
  int32_t lam_bad[kMaxLamCtl];   // per-wavelength singular flag (parallel capacitance solve)
};

struct WsLayout {
  int pmax;           // pixel slots
  int64_t n;
  size_t ctl, V, dchi;        // shared
  size_t lu, piv, yd;         // per wavelength, strides lu_s, piv_s, yd_s
  size_t lu_s, piv_s, yd_s;
  size_t C0, S, panel_s;      // per wavelength, C0 (n x pmax), S (pmax x n), stride panel_s
  size_t sel;                 // selection scratch
  size_t ozA, ozE, ozB, ozF;  // tensor-core update: digit slices and scale exponents (wavelength-shared)
  size_t c64M, c64A, c64B;    // complex64 tensor-core update: D A^{-1}, split-FP16 operand blocks
  size_t c64E, c64F;          //   and their row / column scale exponents
  size_t table;               // fill: Toeplitz table + monitor vector
  size_t total;
};

// Digit-slice buffers of the tensor-core complex128 update for an n x n G.
struct OzLayout {
  int64_t nrow_tiles, ncol_tiles;
  size_t bytesA, bytesE, bytesB, bytesF;
};
OzLayout oz_layout(int64_t n);

// Operand blocks of the complex64 tensor-core update (K = 2P real, P = p rounded up to 16).
struct C64Layout {
  int64_t P, K, nkc, nrt, nct, ncp;
  size_t bytesA, bytesB, bytesM, bytesE, bytesF;
};
C64Layout c64_layout(int64_t n, int pmax);
constexpr int kC64MaxP = 128;        // the complex64 tensor-core path takes p <= 128

WsLayout ws_layout(const gf_geom& g, int nlam, int dtype, const gf_cand_spec& spec);
WsLayout ws_layout_n(int64_t n, int64_t table_entries, int pmax, int nlam, int dtype);

// host helpers of gf_api.cu for entry points defined in other translation units
gf_status api_check_problem(gf_handle* h, const gf_problem* p, int dtype);
gf_status api_bind_device(gf_handle* h);
gf_status api_cuda_check(gf_handle* h, const char* where);
gf_status api_fail_msg(gf_handle* h, gf_status s, const char* msg);
int api_device(const gf_handle* h);
int api_sm_count(const gf_handle* h);
int api_update_algo(const gf_handle* h);
gf_status api_check_spec(gf_handle* h, const gf_geom* g, const gf_cand_spec* s);

// ----------------------------------------------------------------------------- kernels
void launch_fill_table(const gf_geom& g, cplx* table, cudaStream_t st);
void launch_fill_expand(const gf_geom& g, int dtype, void* G, int64_t ldg, const cplx* table,
                        cplx* E, cudaStream_t st);
void launch_bands(const gf_geom& g, int dtype, const void* G, int64_t ldg, cplx* bands,
                  cudaStream_t st);
void launch_fill_field(const gf_geom& g, cplx* E, cudaStream_t st);

struct EvalLam {     // one wavelength as seen by the candidate kernels
  const void* G;
  int64_t ldg;
  const cplx* E;
  const cplx* bands;
};
constexpr int kMaxLam = 8;
static_assert(kMaxLam == kMaxLamCtl, "control block sized for every wavelength");
struct EvalArgs {
  int nlam;
  int dtype;
  int nx, ny;
  double chi;           // eps_mat - eps_bg
  int64_t c_begin, c_end;   // anchors (brushes) or pixels (single) evaluated: [c_begin, c_end); c_end < 0: all
  EvalLam lam[kMaxLam];
};
void launch_eval(const EvalArgs& a, const uint8_t* state, const gf_cand_spec& spec, double* dfom,
                 cudaStream_t st);

size_t topk_scratch_bytes();
size_t topk_selftest_bytes();
bool launch_topk_selftest(void* ws, uint64_t wait_ns, int32_t* status, cudaStream_t st);
void launch_select(const gf_geom& g, const gf_cand_spec& spec, const double* dfom, int64_t ncand,
                   int32_t* idx, double* val, int32_t* status, void* ws, cudaStream_t st);
void launch_select_egreedy(const gf_geom& g, const gf_cand_spec& spec, const double* dfom, int64_t ncand,
                           double epsilon, const double* u, int32_t* idx, double* val, int32_t* status, void* ws,
                           cudaStream_t st);

struct UpdLam {
  void* G;
  int64_t ldg;
  cplx* E;
  cplx* bands;
  // Row-block form (a shard of G): G holds `rows` rows (== n for the whole matrix); when vrows is
  // set, the rows G[V[u], :] of the update set come from it (row u, ldv entries apart, storage
  // dtype) instead of from G, and G[i, V[u]] for the field update is read there as G[V[u], i]
  // (reciprocity).
  const void* vrows;
  int64_t ldv;
  int64_t rows;
};
struct UpdArgs {
  int nlam;
  int dtype;
  int nx, ny;
  double chi;
  int pmax;
  int algo;            // GF_UPDATE_TC or GF_UPDATE_DFMA
  int sm_count;
  int nz;              // 0: 2-D scalar problem; >= 1: 3-D dyadic problem with nz layers
  int ncomp;           // unknowns per point (1 or 3)
  int64_t mrow;        // first monitor unknown
  int mcount;          // monitor unknowns (1 or 3); FOM = sum of their |E|^2
  UpdLam lam[kMaxLam];
};
// CUDA-event timer of the G-update kernel launches (armed by gf_profile_begin).  Each record
// holds an event pair and the rank p that the launch applied (written by the kernel into
// mapped host memory, since p is only known on the device).
// Eq. 1 at the monitor: FOM = sum over components q < ncomp and wavelengths l < nlam of
// |E_l[mrow + q]|^2, written to *out (device).
struct FomArgs {
  const cplx* E[kMaxLam];
  int nlam;
  int ncomp;
  int64_t mrow;
};
void launch_fom(const FomArgs& a, double* out, cudaStream_t st);

struct KernelTimer {
  bool on = false;
  int max = 0, used = 0;
  cudaEvent_t* ev0 = nullptr;
  cudaEvent_t* ev1 = nullptr;
  int32_t* p_host = nullptr;     // mapped pinned host memory, one int per record
  int32_t* p_dev = nullptr;      // its device alias
  double* n2 = nullptr;          // n*n entries updated by each record (host)
  int* bytes_per_entry = nullptr;
  void release();
};

KernelTimer* api_timer(gf_handle* h);

bool launch_rank_update_ozaki(double2* G, int64_t ldg, int64_t n, int64_t rows, int pmax, const cplx* C0,
                              const cplx* S, const UpdCtl* ctl, uint8_t* ozA, int32_t* ozE,
                              uint8_t* ozB, int32_t* ozF, int32_t* status, int32_t* prof_p,
                              int sm_count, cudaStream_t st);

bool c64_tc_make_map(float2* G, int64_t ldg, int64_t n, int64_t rows, void* map128);
void launch_rank_update_c64_tc(const void* map128, float2* G, int64_t ldg, int64_t n, int64_t rows,
                               const void* vrows, int64_t ldv, const WsLayout& L, char* ws, int lam,
                               int32_t* status, int32_t* prof_p, int sm_count, cudaStream_t st);

size_t refresh_workspace_size(const gf_geom& g, int restart);
gf_status refresh(const gf_problem& prob, int dtype, const uint8_t* state, int nsample, const int32_t* cols,
                  int restart, int max_iter, double tol, double* resid, int32_t* iters, double* colres, char* ws,
                  cudaStream_t st);
gf_status refresh_field(const gf_problem& prob, const uint8_t* state, double e_tol, int restart, int max_iter,
                        double tol, gf_refresh_report* rep, char* ws, cudaStream_t st);

void launch_update(const UpdArgs& a, const WsLayout& L, char* ws, uint8_t* state,
                   const gf_cand_spec& spec, const int32_t* idx, int32_t* status, double* fom_out,
                   int32_t* applied, cudaStream_t st, KernelTimer* timer);

// ----------------------------------------------------------------------------- batches
// One problem of a batch (single wavelength, rank <= 4 steps), as the batched kernels read it
// from the device table: blockIdx.y of a batched launch selects the problem.
constexpr int kBatchMax = 64;        // problems per batched launch
struct BatchItem {
  void* G;
  int64_t ldg;
  cplx* E;
  cplx* bands;
  int32_t nx, ny;
  double chi;
  char* ws;
  WsLayout L;
  uint8_t* state;
  double* dfom;
  int64_t ncand;
  int32_t* idx;
  double* val;
  int32_t* status;
  double* fom;
  int32_t* applied;
  double epsilon;              // 0: greedy; else epsilon-greedy with the uniforms below
  const double* uniforms;      // 2 per step
  int32_t* step;               // device step counter
  int32_t horizon;
};
__device__ __forceinline__ void batch_upd_args(const BatchItem& it, int dtype, UpdArgs& a) {
  a.nlam = 1;
  a.dtype = dtype;
  a.nx = it.nx;
  a.ny = it.ny;
  a.chi = it.chi;
  a.pmax = it.L.pmax;
  a.algo = GF_UPDATE_TC;
  a.sm_count = 0;
  a.nz = 0;
  a.ncomp = 1;
  a.mrow = it.L.n - 1;
  a.mcount = 1;
  a.lam[0].G = it.G;
  a.lam[0].ldg = it.ldg;
  a.lam[0].E = it.E;
  a.lam[0].bands = it.bands;
  a.lam[0].vrows = nullptr;
  a.lam[0].ldv = 0;
  a.lam[0].rows = it.L.n;
}
// each launcher covers problems [0, nprob) of the device table; `widest` is the largest
// per-problem extent of the launch's x dimension (pixels, candidates or rows)
void launch_eval_batch(const BatchItem* items, int nprob, int dtype, const gf_cand_spec& spec, int64_t widest,
                       cudaStream_t st);
void launch_select_batch(const BatchItem* items, int nprob, double tie_rel, cudaStream_t st);
void launch_capacitance_batch(const BatchItem* items, int nprob, int dtype, const gf_cand_spec& spec,
                              cudaStream_t st);
void launch_panels_batch(const BatchItem* items, int nprob, int dtype, int64_t widest, cudaStream_t st);
void launch_finish_batch(const BatchItem* items, int nprob, int dtype, int64_t widest, cudaStream_t st);
void launch_bands_batch(const BatchItem* items, int nprob, int dtype, int64_t widest, cudaStream_t st);
// complex64 rank <= 4 update in FP32 on the CUDA cores (HBM-bound streaming)
void launch_rank_update_c64_fp32_batch(const BatchItem* items, int nprob, int ctas, cudaStream_t st);
void launch_rank_update_c64_fp32(float2* G, int64_t ldg, int64_t n, int64_t rows, int pmax, const cplx* C0, const cplx* S,
                                 const UpdCtl* ctl, int32_t* prof_p, int ctas, cudaStream_t st);
constexpr int kC64Fp32MaxP = 4;
// complex128: n^2 p_max below which the FP64 FMA update beats the tensor-core pipeline's fixed cost
// (G resident in L2; 32x32 single pixel: 19 vs 44 us)
constexpr double kC128SmallWork = 2.5e6;
void launch_rank_update_f64_batch(const BatchItem* items, int nprob, int64_t widest_n, cudaStream_t st);
// complex128 rank <= 4 update on the tensor cores for a whole batch: the operand preparation
// of every problem, then one persistent launch over all problems' tiles.  The parameter block
// (tensor maps and descriptors) is built once per batch by ozaki_batch_params.
size_t ozaki_batch_params_bytes();
bool ozaki_batch_params(void* out, const BatchItem* host_items, int nprob);
void launch_oz_prep_batch(const BatchItem* items, int nprob, int64_t widest, cudaStream_t st);
void launch_rank_update_ozaki_batch(const void* params, int ctas, cudaStream_t st);

// ----------------------------------------------------------------------------- persistent batched step
// One launch runs the stages of a step for every problem as work items, taken from a device queue
// in stage-major order; an item of stage s of a problem first waits (bounded) until every item of
// the stage that s depends on has finished for that problem.  Waits only go to items taken earlier
// from the queue, held by running CTAs, so every wait ends without a cooperative launch.
enum BatchStage : int32_t {
  kStEval = 0,     // dFOM of every candidate (Eq. 9)
  kStSelCap,       // selection, then the capacitance solve (one CTA)
  kStPanels,       // C0 = G[:, V], S = D A^-1 G[V, :]
  kStPrep,         // complex128: digit operands of the tensor-core update
  kStUpdate,       // G += C0 S: complex64 in FP32 (tiles of R x 512), complex128 in FP64 FMA (16 x 256)
  kStFinish,       // E, state, FOM
  kStBands,        // bands of the new G (when the update runs in the launch)
};
constexpr int kPlanStages = 6;
constexpr int kBatchThreads = 256;
struct BatchSync {                          // device; zero between launches (the last CTA clears it)
  int32_t next;                             // next work item
  int32_t exited;                           // CTAs that have left
  int32_t abort;                            // a bounded wait gave up
  int32_t pad;
  int32_t done[kBatchMax][kPlanStages];     // finished items per queue position and plan stage
};
struct BatchPlan {                          // built on the host, passed by value
  const BatchItem* items;
  BatchSync* sync;
  int32_t nprob, nstage, total, dtype;
  int32_t kind, dir_mask, eval_mask;        // eval_mask: dir_mask plus the aligned-brush bit
  double tie_rel;
  int64_t timeout_ns;
  int32_t stall_q;                          // diagnostic: this queue position's selection waits for
                                            // one evaluation item more than exist (-1: none)
  int32_t upd_tiles;                        // complex64 update tiles per work item
  int32_t stage[kPlanStages];               // BatchStage of each plan stage
  int32_t dep[kPlanStages];                 // plan stage waited for (-1: none)
  int32_t order[kBatchMax];                 // queue position -> problem (largest first)
  int32_t first[kPlanStages][kBatchMax + 1];  // item ranges: [first[s][q], first[s][q + 1])
};
// plan of the persistent launch: complex128 runs evaluation .. operand preparation and finish (the
// tensor-core update and the bands follow as their own launches); complex64 runs the whole step.
// scale: candidates / rows per thread and item; rows: row tile of the complex64 update (16, 32, 64;
// 0: the complex64 update and bands run as their own launches)
// c128_fma: complex128 with the FP64 FMA update stage in the persistent launch (small problems)
void build_batch_plan(BatchPlan& P, const BatchItem* host_items, int nprob, int dtype, const gf_cand_spec& spec,
                      int scale, int rows, bool c128_fma);
int batch_step_ctas_per_sm(int rows, int kind);
void launch_batch_step(const BatchPlan& P, int ctas, int rows, cudaStream_t st);

}  // namespace gf
