/*
 * libgfopt -- C ABI of the GB300 (sm_103a) hot path of the Green's-function
 * pixel-by-pixel optimizer (Wang et al., arXiv:2202.05388).
 *
 * One greedy step (Sec. II, Fig. 1; partitioned form of Sec. III) is
 *   gf_eval_candidates  -> exact dFOM of every candidate flip     (Eqs. 4-9, Eq. 1)
 *   gf_select_topk      -> the reduction to the chosen flip(s)     (Sec. III reduction)
 *   gf_apply_update     -> rank-p update of G and update of E      (Eqs. 10-14, Eq. 4)
 * and gf_fill_g0 builds the analytic background G0 and E_inc      (Sec. II-B, Sec. IV).
 *
 * Problem statement in this library's variables (2-D scalar E_z restatement):
 *   Points: N = nx*ny pixels, row-major j = iy*nx + ix with centre ((ix+1/2)dx, (iy+1/2)dx),
 *   then the monitor point at index N; n = N + 1.
 *   G is a dense n x n complex matrix, row-major with leading dimension ldg (entries).  The
 *   paper's b = k0^2 d_eps dV is folded into G, so a flip changes the contrast chi_j of pixel
 *   j by d_chi = +-(eps_mat - eps_bg).  E is the field at the n points (complex128).
 *   Background (vacuum) values written by gf_fill_g0, with k = 2 pi / wavelength:
 *     G_ij = (i/4) k^2 dx^2 H0(k |r_i - r_j|)  (i != j),
 *     G_jj = (i pi/2) k a H1(k a) - 1, a = dx / sqrt(pi),  G_NN = 0,  E_j = exp(i k y_j).
 *
 * Conventions for every call:
 *   - Return value is a host-side status (GF_OK or an error); the message of the last error
 *     on a handle is returned by gf_last_error().  Arguments are validated on the host
 *     before anything is launched; an invalid argument launches nothing.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream).  No call synchronises the device.
 *   - All array arguments are device pointers owned by the caller unless stated; the library
 *     allocates no device memory in any call.  Scratch space is the caller's `ws` buffer of
 *     at least gf_workspace_size() bytes (256-byte aligned).
 *   - Data-dependent outcomes (no improving candidate, singular capacitance matrix) are
 *     written to the caller's device status word (int32), so no host round trip is needed;
 *     later calls in the same step read it and turn into no-ops when it is not GF_OK.
 *   - Pointers must be 16-byte aligned; ldg >= n and ldg even.
 *   - A handle is not thread safe; use one handle per host thread / stream.
 */
#ifndef GFOPT_H
#define GFOPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gf_status;
#define GF_OK          0
#define GF_EINVAL      1   /* invalid argument (host check) */
#define GF_ECUDA       2   /* a CUDA runtime call failed */
#define GF_ESINGULAR   3   /* device status: capacitance matrix I - G_VV D singular (Sec. II-A) */
#define GF_ENOIMPROVE  4   /* device status: no candidate increases the FOM (Sec. IV stop rule) */
#define GF_ETIMEOUT    5   /* device status: a bounded wait gave up */
#define GF_ENOMEM      6   /* workspace too small */

#define GF_C128 0          /* G stored as complex128 (interleaved re, im doubles) */
#define GF_C64  1          /* G stored as complex64 (interleaved re, im floats) */

#define GF_KIND_SINGLE 0   /* candidate id = pixel j */
#define GF_KIND_BRUSH2 1   /* candidate id = dir*P + iy*(nx-1) + ix, P = (nx-1)(ny-1) */
#define GF_KIND_PILLAR 2   /* 3-D: 2x2 lateral block through all layers; ids as GF_KIND_BRUSH2 */
#define GF_DIR_FILL  1     /* eps_bg -> eps_mat allowed */
#define GF_DIR_CLEAR 2     /* eps_mat -> eps_bg allowed */

#define GF_NBANDS 9        /* G entries of each pixel row with its 3x3 neighbourhood */

/* Design-region geometry for one wavelength (Sec. III notation: nx, ny; monitor r_m).
 * eps_bg must be 1 (vacuum background with the analytic G0 of Sec. IV). The monitor must
 * lie outside the closed design rectangle [0, nx dx] x [0, ny dx] (Sec. III). */
typedef struct gf_geom {
  int32_t nx, ny;
  double dx;
  double wavelength;
  double eps_bg, eps_mat;
  double mon_x, mon_y;
} gf_geom;

/* One wavelength's state.  G: n x ldg entries of the storage dtype.  E: n complex128.
 * bands: GF_NBANDS * N complex128, band b at bands + b*N, entry i = G[i, i + off_b] with
 * off = {0, +1, -1, nx-1, -(nx-1), nx, -nx, nx+1, -(nx+1)} (0 where the neighbour pixel is
 * outside the grid); they are the G_VV entries that brush candidates need (Eq. 8). */
typedef struct gf_problem {
  gf_geom geom;
  void* G;
  int64_t ldg;
  void* E;
  void* bands;
} gf_problem;

/* Candidate family (Sec. II-A "shapes and sizes for region V"; Sec. IV 2x2 brushes).
 * k > 1 accepts up to k non-conflicting candidates per step (conflict: Chebyshev distance of
 * anchors <= excl_radius).  Ties: lowest id among dFOM >= max - tie_rel*|max|.
 * aligned != 0 (brushes and pillars): only anchors with even ix and iy are candidates -- the
 * aligned, non-overlapping 2x2 partitions of Sec. IV; the others evaluate to -inf. */
typedef struct gf_cand_spec {
  int32_t kind;
  int32_t dir_mask;
  int32_t k;
  int32_t excl_radius;
  double tie_rel;
  int32_t aligned;
  int32_t pad;
} gf_cand_spec;

typedef struct gf_handle gf_handle;

/* Create a handle bound to CUDA device `device`.  Returns GF_ECUDA if it does not exist. */
gf_status gf_create(gf_handle** h, int32_t device);
void gf_destroy(gf_handle* h);
/* Message of the last error on h (never NULL; "" when none).  h may be NULL for the last
 * gf_create failure of this thread. */
const char* gf_last_error(const gf_handle* h);
const char* gf_status_string(gf_status s);
/* Library version string. */
const char* gf_version(void);

/* Number of candidate ids for a geometry and candidate family (N, or 2(nx-1)(ny-1)). */
int64_t gf_num_candidates(const gf_geom* geom, const gf_cand_spec* spec);
/* Workspace bytes needed by gf_fill_g0 / gf_select_topk / gf_apply_update for nlam
 * wavelengths of this geometry, storage dtype and candidate family (0 on bad arguments). */
size_t gf_workspace_size(const gf_geom* geom, int32_t nlam, int32_t dtype,
                         const gf_cand_spec* spec);

/* Background Green's matrix, incident field and bands of one wavelength (Sec. II-B: the
 * initial G of a vacuum background is known analytically; Sec. IV).  Writes all n x ldg
 * entries of G (padding columns zero), E[0..n) and the bands.  Hankel functions are
 * evaluated once per distinct pixel offset (a Toeplitz table in ws) and expanded. */
gf_status gf_fill_g0(gf_handle* h, const gf_problem* prob, int32_t dtype,
                     void* ws, size_t ws_bytes, void* stream);

/* gf_fill_g0 without a workspace, for callers that cannot allocate device memory (a host
 * application that owns all device allocations, or a loop that must not call cudaMalloc).
 * The paper has no counterpart.  The Hankel table lives in a fixed 4 MiB array inside the
 * library (held on every GPU that loads it until exit), so N = nx*ny <= 131072 (GF_EINVAL
 * otherwise).  All calls share that array: calls overlapping on the GPU race and must be
 * ordered by the caller.  Every call looks up the array's address on the handle's device;
 * the first call on a device also loads the library's device code there, so make that first
 * call before any stream capture.  Writes the same G, E and bands as gf_fill_g0. */
gf_status gf_fill_g0_static(gf_handle* h, const gf_problem* prob, int32_t dtype, void* stream);

/* Figure of merit of the current fields (Eq. 1): *fom_out (device double) = sum over the nlam
 * wavelengths of |E(r_m)|^2 = |E[N]|^2.  gf_apply_update writes the FOM after every step;
 * this call gives it for a state no step has produced yet, e.g. right after gf_fill_g0.
 * probs as for gf_eval_candidates (only E is read). */
gf_status gf_fom(gf_handle* h, const gf_problem* probs, int32_t nlam, int32_t dtype, double* fom_out,
                 void* stream);

/* Re-extract the bands of one wavelength from its G (used after external edits of G). */
gf_status gf_extract_bands(gf_handle* h, const gf_problem* prob, int32_t dtype, void* stream);

/* Exact dFOM of every candidate (Eqs. 4-9 at the monitor, then Eq. 1 with
 * FOM = sum over wavelengths of |E(r_m)|^2), written to dfom[0..ncand) in FP64; -inf for a
 * candidate that changes no pixel, whose direction is not enabled, or whose capacitance
 * matrix is singular (|pivot| < 1e-13 ||A||_inf).  state: N bytes, 0 = eps_bg, 1 = eps_mat.
 * probs: host array of nlam problems sharing nx, ny, dx and the monitor. */
gf_status gf_eval_candidates(gf_handle* h, const gf_problem* probs, int32_t nlam,
                             int32_t dtype, const uint8_t* state, const gf_cand_spec* spec,
                             double* dfom, void* stream);

/* Reduction of dFOM to the accepted candidate ids (Sec. III, CombineGlobally).  k == 1:
 * idx[0] = the lowest id with dfom >= m - tie_rel*|m| where m = max dfom.  k > 1: up to k
 * ids in (-dfom, id) order skipping conflicts; unused slots are -1.  val[] gets their dFOM.
 * *status (device) = GF_OK, or GF_ENOIMPROVE when m <= 0 (idx[0] = -1).
 * ws (optional; gf_workspace_size bytes, 256-byte aligned, else NULL): its selection area lets
 * the k == 1 reduction run over many CTAs (from 32768 candidates: two launches) and holds the
 * top-k passes' state; without it one CTA sweeps dfom (the same result). */
gf_status gf_select_topk(gf_handle* h, const gf_geom* geom, const gf_cand_spec* spec,
                         const double* dfom, int64_t ncand, int32_t* idx, double* val,
                         int32_t* status, void* ws, size_t ws_bytes, void* stream);

/* epsilon-greedy policy (Sec. V): with probability 1 - epsilon the greedy choice of
 * gf_select_topk (k = 1), with probability epsilon a uniformly random one of the (up to) four
 * best improving candidates ranked by (-dFOM, id).  The randomness is an input: u (device, 2
 * doubles in [0, 1)) -- explore when u[0] < epsilon, then take rank floor(u[1] m) of the m <= 4
 * ranked candidates (rank 0 is the best).  Outputs and statuses as gf_select_topk with k = 1.
 * spec->k must be 1; ws is required (gf_workspace_size bytes, 256-byte aligned). */
gf_status gf_select_egreedy(gf_handle* h, const gf_geom* geom, const gf_cand_spec* spec,
                            const double* dfom, int64_t ncand, double epsilon, const double* u,
                            int32_t* idx, double* val, int32_t* status, void* ws, size_t ws_bytes,
                            void* stream);

/* Apply the candidates idx[0..k) (device; -1 ends the list) to every wavelength:
 * snapshot rows G[V,:] and columns G[:,V], solve A R = G[V,:] with A = I - G_VV D (Eq. 14,
 * FP64, partial pivoting), then G <- G + G[:,V] D R (Eq. 10) and E <- E + G[:,V] D y with
 * y = A^{-1} E_V (Eqs. 4, 9); flip state at V, re-extract bands and write the new
 * FOM (sum over wavelengths of |E_N|^2) to *fom_out (device double).  With more than one
 * candidate, the union is applied only if its joint dFOM is positive; otherwise idx[0]
 * alone (the best one) is applied.  *applied (device int32, may be NULL) receives the number
 * of candidates applied (0 when nothing changed).  No-op when *status != GF_OK on entry; sets
 * *status = GF_ESINGULAR (and changes nothing) when A is singular. */
gf_status gf_apply_update(gf_handle* h, const gf_problem* probs, int32_t nlam, int32_t dtype,
                          uint8_t* state, const gf_cand_spec* spec, const int32_t* idx,
                          int32_t* status, double* fom_out, int32_t* applied, void* ws,
                          size_t ws_bytes, void* stream);

/* Drift refresh of one wavelength (checks against the discrete Eqs. 3 and 2; run every few
 * hundred steps).  resid_out (host, 1 + nsample doubles):
 *   resid_out[0]   = ||E - E_inc - G0 X E||_2 / ||E||_2 (Lippmann-Schwinger residual, with G0 X E
 *                    computed by FFT convolution of the Toeplitz pixel block, FP64);
 *   resid_out[1+s] = ||G[:, cols[s]] - g||_2 / ||g||_2 where (I - G0 X) g = G0[:, cols[s]] is
 *                    solved by restarted GMRES(restart) from the stored column to relative
 *                    residual tol (at most max_iter iterations; iters_out[s] = iterations, may
 *                    be NULL).  A stored column that already meets tol takes no iteration and
 *                    reads 0 here; its backward error is in colres_out.
 *   colres_out[s]  (host, nsample doubles, may be NULL) = ||G0[:, c] - (I - G0 X) G[:, c]||_2 /
 *                    ||G0[:, c]||_2 for c = cols[s], the stored column's own Eq. 2 residual
 *                    (its forward error is at most the condition number of I - G0 X times it).
 * cols: host array of nsample indices in [0, n).  Blocking: returns after synchronising
 * `stream`.  ws: at least gf_refresh_workspace_size() bytes.  nx, ny <= 4096. */
size_t gf_refresh_workspace_size(const gf_geom* geom, int32_t restart);
gf_status gf_refresh(gf_handle* h, const gf_problem* prob, int32_t dtype, const uint8_t* state,
                     int32_t nsample, const int32_t* cols, int32_t restart, int32_t max_iter,
                     double tol, double* resid_out, int32_t* iters_out, double* colres_out, void* ws,
                     size_t ws_bytes, void* stream);

/* Field repair of one wavelength (the discrete Eq. 3, (I - G0 X) E = E_inc).  Computes
 * rho = ||E_inc - (I - G0 X) E||_2 / ||E_inc||_2 with the FFT matvec of gf_refresh; when
 * rho > e_tol, re-solves the system by restarted GMRES(restart) from the stored E to relative
 * residual tol (at most max_iter iterations) and replaces E by the solution if its residual is
 * smaller.  G is not read or changed.  The FOM of the new field is not written: call gf_fom.
 * report (host): e_residual = rho on entry, e_residual_after = the residual of E on return,
 * e_iters = GMRES iterations (0 when E was kept), e_replaced = 1 when E was replaced.
 * Blocking (synchronises `stream`); ws as for gf_refresh; nx, ny <= 4096. */
typedef struct gf_refresh_report {
  double e_residual;
  double e_residual_after;
  int32_t e_iters;
  int32_t e_replaced;
} gf_refresh_report;
gf_status gf_refresh_field(gf_handle* h, const gf_problem* prob, int32_t dtype, const uint8_t* state,
                           double e_tol, int32_t restart, int32_t max_iter, double tol,
                           gf_refresh_report* report, void* ws, size_t ws_bytes, void* stream);

/* Arithmetic of the G update (Eq. 10).  GF_UPDATE_TC (default), the fast form per case:
 *   complex128, p <= 4: exact digit products on the tensor cores with an integer
 *     recombination (FP64-accurate to ~2^-50 of |C0||S|), except on problems with
 *     n^2 p_max <= 2.5e6 (L2-resident; the persistent tensor-core pipeline's fixed cost
 *     dominates there), which take native FP64 FMA; larger p: native FP64 FMA;
 *   complex64, p <= 4: FP32 FMA on the CUDA cores (a pure HBM stream);
 *   complex64, 4 < p <= 128: the Woodbury form S = D A^-1 G[V,:] and a scaled split-FP16
 *     tensor-core GEMM with FP32 accumulation.
 * GF_UPDATE_DFMA: native FP64 FMA for every case (complex64 storage rounded once per entry).
 * GF_UPDATE_TENSOR: as GF_UPDATE_TC, but the tensor-core forms at every problem size.
 * The complex128 forms match the FP64 oracle within 1e-10; they differ only in speed on GB300
 * (whose FP64 pipe is 1/64 of its FP32 rate).  Applies to later gf_apply_update calls on h.
 * For complex64 G the setting also selects the arithmetic of gf3_eval_candidates: GF_UPDATE_TC
 * and GF_UPDATE_TENSOR factorise each pillar's system in FP32 and refines the solution once with an FP64 residual
 * (the accuracy of an FP64 solve of the stored system); GF_UPDATE_DFMA factorises in FP64. */
#define GF_UPDATE_TC     0
#define GF_UPDATE_DFMA   1
#define GF_UPDATE_TENSOR 2
gf_status gf_set_update_algo(gf_handle* h, int32_t algo);

/* Deferred (low-rank) form, single wavelength, one candidate per step (k = 1), FP64.
 * Eq. 10 applied step after step gives G_t = G0 + sum_s C_s D_s R_s (C_s = G_s[:, V_s],
 * R_s = A_s^-1 G_s[V_s, :], Eq. 14); with G = G^T (reciprocity) every term is C_s M_s C_s^T with
 * M_s = D_s A_s^-1.  This form keeps G0 implicit (its offset table, in ws) and stores only the
 * columns C_s (n x K, K = pixels flipped so far) and the blocks M_s, plus the entries candidate
 * evaluation reads: the bands, the monitor row G[N, :] and E.  Memory O(n K) instead of
 * O(n^2); a step costs O(n K p).  Steps: gf_lowrank_eval, gf_select_topk (or
 * gf_select_egreedy), gf_lowrank_update.  Fields (device, 16-byte aligned, caller-owned):
 *   E (n complex128), bands (9 N complex128, layout of gf_problem.bands), monrow (n
 *   complex128), U (n x max_cols complex128, column-major: column k at U + k n).
 * ws (gf_lowrank_workspace_size bytes, 256-byte aligned) must be the same buffer for
 * gf_lowrank_init and every later call on the problem: it holds the G0 table, the blocks and
 * the term bookkeeping.  When K would exceed max_cols, the update sets *status = GF_ENOMEM and
 * changes nothing. */
typedef struct gf_lowrank {
  gf_geom geom;
  void* E;
  void* bands;
  void* monrow;
  void* U;
  int32_t max_cols;
} gf_lowrank;
size_t gf_lowrank_workspace_size(const gf_geom* geom, int32_t max_cols);
/* Vacuum start: G0 table, bands, monitor row, E = E_inc, no terms. */
gf_status gf_lowrank_init(gf_handle* h, const gf_lowrank* lr, void* ws, size_t ws_bytes, void* stream);
/* Eq. 1 for the low-rank state: *fom_out (device double) = |E[N]|^2 (only lr->E is read). */
gf_status gf_lowrank_fom(gf_handle* h, const gf_lowrank* lr, double* fom_out, void* stream);
/* dFOM of every candidate (as gf_eval_candidates). */
gf_status gf_lowrank_eval(gf_handle* h, const gf_lowrank* lr, const uint8_t* state, const gf_cand_spec* spec,
                          double* dfom, void* stream);
/* Apply idx[0 .. spec->k) as gf_apply_update does (top-k candidates applied jointly when their
 * joint dFOM is positive, else idx[0] alone; *applied = candidates applied): new columns
 * G[:, V], capacitance solve, append the term, update bands, monitor row, E, state and
 * *fom_out.  At most 32 pixels per step: k <= 32 single pixels or k <= 8 brushes. */
gf_status gf_lowrank_update(gf_handle* h, const gf_lowrank* lr, uint8_t* state, const gf_cand_spec* spec,
                            const int32_t* idx, int32_t* status, double* fom_out, int32_t* applied,
                            void* ws, size_t ws_bytes, void* stream);
/* Terms and columns stored so far (blocking: synchronises stream). */
gf_status gf_lowrank_count(gf_handle* h, const gf_lowrank* lr, void* ws, size_t ws_bytes, int32_t* nterms,
                           int32_t* ncols, void* stream);
/* Dense complex128 G (n x ldg) = G0 + sum_s C_s M_s C_s^T, for checks or a switch to the dense
 * form; O(n^2 K) work. */
gf_status gf_lowrank_materialize(gf_handle* h, const gf_lowrank* lr, void* G, int64_t ldg, void* ws,
                                 size_t ws_bytes, void* stream);

/* 3-D form (the paper's own setting, Sec. II with 3x3 dyadic blocks; Sec. IV's metalens).
 * A slab of nx*ny*nz cubic voxels of side dx, voxel j = (iz*ny + iy)*nx + ix with centre
 * ((ix+1/2)dx, (iy+1/2)dx, (iz+1/2)dx); one monitor point (mon_x, mon_y, mon_z) outside the
 * slab.  Unknowns u = 3*point + component (x, y, z), the monitor last: n = 3 (N + 1).
 *   G_ij (3x3 block) = k^2 dV G0(r_i - r_j), G0(R) = (I + grad grad / k^2) e^{ikR} / (4 pi R);
 *   G_jj = [(2/3)((1 - i k a) e^{ika} - 1) - 1/3] I, a = (3 dV / (4 pi))^(1/3) (principal volume
 *   over the equal-volume sphere with the depolarisation I/3); the monitor's own block is 0;
 *   E_inc = x^ e^{ikz} (x-polarised, travelling +z); FOM = |E(r_m)|^2 over the three components.
 * Candidates: GF_KIND_PILLAR (2x2 lateral blocks through all layers, p = 12 nz unknowns, ids as
 * for 2-D brushes, both directions per dir_mask).  Restrictions: 1 <= nz <= 8, one wavelength,
 * complex128 or complex64 G (n x ldg, ldg even >= n); a flip changes all three components.
 * The steps mirror the 2-D calls: gf3_fill_g0, gf3_eval_candidates, gf3_select_topk,
 * gf3_apply_update (the update kernels are the 2-D ones on the 3n unknowns). */
typedef struct gf_geom3d {
  int32_t nx, ny, nz, pad;
  double dx;
  double wavelength;
  double eps_bg, eps_mat;
  double mon_x, mon_y, mon_z;
} gf_geom3d;
typedef struct gf_problem3d {
  gf_geom3d geom;
  void* G;
  int64_t ldg;
  void* E;       /* n complex128 */
} gf_problem3d;
int64_t gf3_num_unknowns(const gf_geom3d* geom);
int64_t gf3_num_candidates(const gf_geom3d* geom);
size_t gf3_workspace_size(const gf_geom3d* geom, int32_t dtype, const gf_cand_spec* spec);
gf_status gf3_fill_g0(gf_handle* h, const gf_problem3d* prob, int32_t dtype, void* ws, size_t ws_bytes, void* stream);
/* Eq. 1 in 3-D: *fom_out (device double) = sum over the three components of |E(r_m)|^2. */
gf_status gf3_fom(gf_handle* h, const gf_problem3d* prob, int32_t dtype, double* fom_out, void* stream);
gf_status gf3_eval_candidates(gf_handle* h, const gf_problem3d* prob, int32_t dtype, const uint8_t* state,
                              const gf_cand_spec* spec, double* dfom, void* stream);
gf_status gf3_select_topk(gf_handle* h, const gf_geom3d* geom, const gf_cand_spec* spec, const double* dfom,
                          int64_t ncand, int32_t* idx, double* val, int32_t* status, void* ws, size_t ws_bytes,
                          void* stream);
gf_status gf3_apply_update(gf_handle* h, const gf_problem3d* prob, int32_t dtype, uint8_t* state,
                           const gf_cand_spec* spec, const int32_t* idx, int32_t* status, double* fom_out,
                           int32_t* applied, void* ws, size_t ws_bytes, void* stream);

/* Row-block shards of one problem (Sec. III: the rows of G split over partitions, a
 * partition-local dFOM, a global combine, a broadcast of the chosen pixels' rows and each
 * partition's update of its own rows), for G larger than one GPU's memory.  A shard holds the
 * rows of G of pixel rows [y0, y1), 0 <= y0 < y1 <= ny; the shard with y1 = ny also holds the
 * monitor row.  Global rows [r0, r1), r0 = y0 nx, r1 = y1 nx (+1 when y1 = ny), are stored as
 * (r1 - r0) x ldg entries of the storage dtype at G (ldg even, >= n).
 *   E (n complex128) and the design state (N bytes) are whole on every shard; the calls below
 *   keep them identical on all shards when every shard makes the same calls with the same idx.
 *   bands (GF_NBANDS N complex128, layout of gf_problem.bands) and mon (n complex128, mon[j] =
 *   G[N, j] = G[j, N] by reciprocity) are valid for the pixels of rows [y0, min(y1 + 1, ny)): the
 *   shard's own rows and the halo row y1, which the next shard supplies.
 * A step on every shard: gf_shard_eval; elementwise maximum of the dfom arrays over the shards;
 * gf_select_topk (the same choice everywhere); gf_shard_gather_rows; sum of the panels over the
 * shards; gf_shard_apply_update; gf_shard_pack_halo, exchange, gf_shard_unpack_halo.  One
 * wavelength; ws = gf_workspace_size(&geom, 1, dtype, spec) bytes, 256-byte aligned. */
typedef struct gf_shard {
  gf_geom geom;
  int32_t y0, y1;
  void* G;
  int64_t ldg;
  void* E;
  void* bands;
  void* mon;
} gf_shard;
/* Rows of G the shard holds (r1 - r0; 0 on bad arguments). */
int64_t gf_shard_rows(const gf_shard* shard);
/* Vacuum start: the shard's rows of G0, E = E_inc, and bands and mon of rows [y0, min(y1+1, ny)). */
gf_status gf_shard_fill_g0(gf_handle* h, const gf_shard* shard, int32_t dtype, void* ws, size_t ws_bytes,
                           void* stream);
/* dFOM (as gf_eval_candidates) of the candidates anchored in the shard's pixel rows: brushes with
 * anchor row iy in [y0, min(y1, ny - 1)), single pixels of rows [y0, y1).  Every other entry of
 * dfom (gf_num_candidates doubles) is -inf, so the elementwise maximum over the shards is the
 * dFOM array of the whole problem. */
gf_status gf_shard_eval(gf_handle* h, const gf_shard* shard, int32_t dtype, const uint8_t* state,
                        const gf_cand_spec* spec, double* dfom, void* stream);
/* The shard's part of the broadcast of the update set's rows.  V = the union of the candidates
 * idx[0..k) (-1 ends the list) in the order gf_apply_update forms it; panel (pmax x ldp entries of
 * the storage dtype, pmax = 4k for brushes and k for single pixels, ldp even and >= n): row u =
 * G[V[u], :] where the shard holds row V[u], zero elsewhere, so the sum of all shards' panels holds
 * every row of V exactly once.  All zero when *status != GF_OK. */
gf_status gf_shard_gather_rows(gf_handle* h, const gf_shard* shard, int32_t dtype, const uint8_t* state,
                               const gf_cand_spec* spec, const int32_t* idx, const int32_t* status, void* panel,
                               int64_t ldp, void* stream);
/* gf_apply_update for one shard, with the rows G[V, :] from the summed panel: the capacitance solve
 * (Eqs. 9, 14; G_VV and G[N, V] = G[V, N] from the panel), the update of the shard's rows (Eq. 10),
 * of the whole E (Eq. 4, G[i, V] = G[V, i] from the panel) and of the state, *fom_out, *applied,
 * and the bands and mon of the shard's own rows read back from its updated rows. */
gf_status gf_shard_apply_update(gf_handle* h, const gf_shard* shard, int32_t dtype, uint8_t* state,
                                const gf_cand_spec* spec, const int32_t* idx, const void* panel, int64_t ldp,
                                int32_t* status, double* fom_out, int32_t* applied, void* ws, size_t ws_bytes,
                                void* stream);
/* Halo exchange: pack writes the bands and mon of pixel row y0 to out ((GF_NBANDS + 1) nx complex128:
 * band 0 .. band 8, then mon); unpack writes the next shard's record as pixel row y1 (nothing when
 * y1 = ny). */
gf_status gf_shard_pack_halo(gf_handle* h, const gf_shard* shard, void* out, void* stream);
gf_status gf_shard_unpack_halo(gf_handle* h, const gf_shard* shard, const void* in, void* stream);

/* Batches: many independent problems advanced together (the problems of a design study, e.g.
 * sweeps over sizes, wavelengths and focal distances; the paper parallelises one problem's
 * partitions instead, Sec. III).  Each item is one single-wavelength problem with its own
 * design state, step buffers and workspace -- the arguments of the single-problem calls.  One
 * gf_batch_step runs a whole greedy step (dFOM of every candidate, greedy selection, capacitance
 * solve, panels, G and E update, band extraction) for every item with one launch per stage: the
 * G update is one persistent launch over the tiles of all items that accepted a flip.  The
 * step only enqueues kernels (no host synchronisation, no copies), so it can be captured in a
 * CUDA graph.  Limits: k = 1 (rank <= 4), 1 to 64 items, shared dtype and candidate spec.
 * The items' buffers must stay valid until gf_batch_destroy. */
typedef struct gf_batch_item {
  gf_problem prob;      /* one wavelength: geometry, G (n x ldg), E (n), bands (9 N) */
  uint8_t* state;       /* N bytes, 0 = eps_bg, 1 = eps_mat */
  double* dfom;         /* gf_num_candidates(&prob.geom, spec) doubles */
  int32_t* idx;         /* 1: chosen candidate id (-1: none) */
  double* val;          /* 1: its dFOM */
  int32_t* status;      /* 1: device status word of this item */
  double* fom_out;      /* 1: FOM after the step */
  int32_t* applied;     /* 1: candidates applied by the step; may be NULL */
  void* ws;             /* gf_workspace_size(&prob.geom, 1, dtype, spec) bytes, 256-byte aligned */
  size_t ws_bytes;
  /* policy: epsilon = 0 greedy; epsilon in (0, 1] the epsilon-greedy policy of
   * gf_select_egreedy, reading the pair uniforms[2 t], uniforms[2 t + 1] at step t = *step (device
   * counter, incremented by every batch step, so graph replays draw new numbers); a step with
   * t >= horizon sets the item's status to GF_ENOMEM.  uniforms and step may be NULL when
   * epsilon = 0. */
  double epsilon;
  const double* uniforms;
  int32_t* step;
  int32_t horizon;
} gf_batch_item;
typedef struct gf_batch gf_batch;
/* Device bytes of the item table of a batch of nitems (the problem descriptors, then the work
 * queue and per-problem phase counters of the persistent step kernel). */
size_t gf_batch_table_size(int32_t nitems);
/* Validate every item like the single-problem calls, write the item table to `table` (device,
 * 256-byte aligned, gf_batch_table_size bytes, owned by the caller) and build the launch
 * parameters (one TMA descriptor per complex128 G).  Blocking (synchronises `stream`). */
gf_status gf_batch_create(gf_handle* h, int32_t nitems, const gf_batch_item* items, int32_t dtype,
                          const gf_cand_spec* spec, void* table, size_t table_bytes, void* stream,
                          gf_batch** out);
/* Enqueue one greedy step of every item on `stream` (capturable). */
gf_status gf_batch_step(gf_batch* b, void* stream);
/* Launch shape of the persistent G update: update_ctas CTAs (0: one per SM for complex128,
 * three per SM for complex64).  Used by the autotuner; results do not depend on it. */
gf_status gf_batch_set_schedule(gf_batch* b, int32_t update_ctas);
/* Form of the batched step.
 *   GF_BATCH_PERSISTENT (default): one persistent launch takes the step's stages as work items
 *     from a device queue; an item waits (bounded, 2 s) until the stage it depends on has
 *     finished for its own problem.  A wait that gives up writes GF_ETIMEOUT to the problem's
 *     status word and abandons that problem's step (its G, E and state are then unspecified:
 *     fill it again); once one wait has given up, every later wait gives up at once.
 *     complex64: the whole step is that launch; complex128: the tensor-core G update and the
 *     bands follow as two more launches.
 *   GF_BATCH_STAGED: one launch per stage (evaluation, selection, capacitance, panels, [operand
 *     preparation], update, field/FOM, bands).
 * step_ctas: CTAs of the persistent launch (0: as many as are resident on the device at once).
 * scale (1..16): candidates, rows or band entries per thread in one work item.
 * tile_rows (16, 32 or 64): rows of one complex64 update tile (x 512 columns) inside the
 *   persistent launch; 0: the complex64 update and the bands run as two more launches.
 * The knobs of the autotuner: results are bit-identical for every form and shape. */
#define GF_BATCH_STAGED     0
#define GF_BATCH_PERSISTENT 1
gf_status gf_batch_set_form(gf_batch* b, int32_t form, int32_t step_ctas, int32_t scale, int32_t tile_rows);
void gf_batch_destroy(gf_batch* b);
/* Diagnostic of the persistent step's bounded waits (no counterpart in the paper): one step of
 * the batch in the persistent form in which the selection of the largest problem waits for one
 * evaluation item more than exist, with a limit of timeout_ns (1 us .. 2 s).  That problem's
 * status word receives GF_ETIMEOUT (so does any problem with an item still waiting when the wait
 * gave up); the launch ends and the context stays usable. */
gf_status gf_batch_selftest_timeout(gf_batch* b, int64_t timeout_ns, void* stream);

/* Diagnostic of the bounded waits (no counterpart in the paper): one CTA waits on a barrier that
 * nothing signals, with the abortable bounded wait of the tensor-core kernels, for timeout_ns
 * (1 us .. 2 s), then writes GF_ETIMEOUT to *status (device int32) -- the status a stalled
 * update reports -- without faulting the GPU; later calls on the context work as usual. */
gf_status gf_selftest_timeout(gf_handle* h, int64_t timeout_ns, int32_t* status, void* stream);

/* Diagnostic of the one-launch top-k selection's grid barrier (no counterpart in the paper): the
 * cooperative top-k kernel runs on 4096 zero dFOM values in ws with a barrier that waits for one
 * CTA more than the grid holds, each CTA's wait giving up after timeout_ns (1 us .. 2 s); its
 * end writes GF_ETIMEOUT to *status (device int32), without faulting the GPU.  ws: 256-byte
 * aligned, at least gf_select_selftest_bytes() bytes (scratch, values, outputs).  GF_ECUDA when
 * the device cannot launch a cooperative kernel. */
size_t gf_select_selftest_bytes(void);
gf_status gf_select_selftest_timeout(gf_handle* h, int64_t timeout_ns, void* ws, size_t ws_bytes, int32_t* status,
                                     void* stream);

/* Kernel timing (no counterpart in the paper; it backs the per-step timers of the bench).
 * gf_profile_begin arms up to max_records CUDA-event pairs that the library records on the
 * launching stream around every launch of the G-update kernel (in the deferred form: of the
 * column product, whose flops are counted as 8 K p n).  gf_profile_end waits for the
 * last recorded event, returns the summed kernel time in ms, the number of timed launches and
 * the algorithmic bytes (read + write of every G entry) and flops of those launches, and
 * disarms.  Launches beyond max_records are not timed.  Not for use inside graph capture. */
gf_status gf_profile_begin(gf_handle* h, int32_t max_records);
gf_status gf_profile_end(gf_handle* h, double* ms_total, int64_t* launches, double* bytes_total,
                         double* flops_total);

#ifdef __cplusplus
}
#endif

#endif /* GFOPT_H */
