/*
 * tp.h - C ABI of libtp, a GB300 (sm_103a) solver for the tent-pitched
 * space-time Trefftz-DG method for the acoustic wave equation
 * (Perugia, Schoberl, Stocker, Wintersteiger, "Tent pitching and Trefftz-DG
 * method for the acoustic wave equation").
 *
 * Conventions
 *   - Every call returns an int status (TP_OK = 0).  On failure a message is
 *     available from tp_last_error() (thread-local, valid until the next call
 *     on the same thread).
 *   - Host pointers are read during the call only; the library keeps copies.
 *   - Device pointers ("d_" prefix) are caller-owned CUDA global memory on the
 *     current device; the library never frees them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy stream).
 *     Device work is enqueued on it and is asynchronous; device-side errors
 *     (singular local system) are recorded in a status word read by
 *     tp_sync_status().
 *   - Handles are opaque and owned by the library (tp_destroy_*).
 *   - Field layout: a "front" array holds, for every right-hand side r,
 *     element K and front point q, the n+2 values (U, v, sigma_1..sigma_n)
 *     with v = dU/dt and sigma = -grad U (Section 2.1, eq. 2.2):
 *       front[((r * n_elem + K) * Q + q) * (n + 2) + comp],  Q = (p+1)^n.
 */
#ifndef TP_H
#define TP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  TP_OK = 0,
  TP_ERR_ARG = 1,          /* invalid argument (sizes, pointers, unsupported p/dim) */
  TP_ERR_CAUSALITY = 2,    /* a front or tent violates c|grad tau| < 1 (Section 2.2) */
  TP_ERR_SINGULAR = 3,     /* zero or non-finite pivot in a local system */
  TP_ERR_NOCONV = 4,       /* iterative refinement did not converge (reserved: stalled refinements fall back to a direct LU) */
  TP_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
  TP_ERR_CUDA = 6,         /* a CUDA runtime call failed */
  TP_ERR_OOM = 7,          /* allocation failed */
  TP_ERR_UNSUPPORTED = 8   /* valid input outside what this build implements */
};

enum { TP_FP64 = 0, TP_MIXED = 1 };
enum { TP_SCHED_DATAFLOW = 0, TP_SCHED_LEVELS = 1 };

/* Spatial mesh (Section 2.1): simplices aligned with the jumps of the
 * piecewise-constant wave speed c.  dim in {1,2,3}; coords n_vert x dim;
 * elems n_elem x (dim+1) vertex ids; c n_elem values > 0.
 * bnd_type (optional, NULL = every boundary facet Dirichlet): n_elem x
 * (dim+1) host bytes, entry (k, o) for the facet of element k opposite its
 * local vertex o: 0 = Dirichlet (v = g_D on Gamma_D), 1 = Neumann
 * (sigma.n = g_N on Gamma_N), eq. 2.1; entries of interior facets are
 * ignored, other values are TP_ERR_ARG. */
typedef struct tp_mesh_desc {
  int32_t dim;
  int64_t n_vert;
  const double* coords;
  int64_t n_elem;
  const int32_t* elems;
  const double* c;
  const int8_t* bnd_type;
} tp_mesh_desc;

/* p: degree of the second-order Trefftz space U^p (Section 3; unknowns per
 * single-material tent dim U^p = C(p+n,n) + C(p-1+n,n)); alpha: Dirichlet
 * penalty of eq. (2.5) (the paper uses 0.5); beta: penalty of the [[sigma]]_N
 * term on time-like interface facets (eq. 2.5, Section 4.2; the paper uses
 * 0.5); kappa: pitching slope factor (edge-slope limit delta_e = kappa l_e /
 * c_e); T: final time; precision: TP_FP64 (every step in binary64) or
 * TP_MIXED (assembly, residual and outflow in float-float on the binary32
 * pipes, binary32 inverse of the equilibrated local matrix, iterative
 * refinement to float-float accuracy; a tent whose refinement does not
 * settle is solved by a direct binary64 LU instead);
 * nrhs: right-hand sides advanced together (same tents, same matrices;
 * when one CTA's shared memory cannot hold all of them, tp_create picks the
 * largest divisor of nrhs that fits and every sweep runs the groups of that
 * size one after the other, each assembling its own tent matrices);
 * schedule: how tp_advance runs the levels -- TP_SCHED_DATAFLOW (default):
 * one resident kernel whose clusters take the tents in level order and each
 * start as soon as the earlier tents of its vertex and neighbours are done
 * (bounded waits; TP_ERR_TIMEOUT if one gives up), or TP_SCHED_LEVELS: one
 * launch per level. */
typedef struct tp_params {
  int32_t p;
  double alpha;
  double beta;
  double kappa;
  double T;
  int32_t precision;
  int32_t nrhs;
  int32_t schedule;
  /* rhs_split: how a tent's right-hand sides are shared out over the CTAs of
   * its cluster.  0 = automatic (split when each CTA keeps 16 or more,
   * i.e. nrhs >= 32 and divisible by 2, 4 or 8), 1 = never split
   * (every CTA takes a slice of the points for all right-hand sides), 2, 4
   * or 8 = that many CTAs, each owning nrhs / rhs_split of the right-hand
   * sides at every point of the tent (data moments, solve and outflow),
   * while the tent matrix is assembled once, its points split over the
   * same CTAs.  A value that does not divide nrhs is TP_ERR_ARG. */
  int32_t rhs_split;
  /* dissipation: 1 = every forward tent adds the energy it loses,
   *   D = 1/2 int_bot Q(u - u_b) + int_bot (U - U_b) U + the Dirichlet, Neumann
   *   and interface terms of eq. (2.5)/(4.1) tested with its own solution,
   * to a per-right-hand-side sum reported by tp_energy (an extra pass over
   * the tent's bottom and vertical-face points); 0 = not tracked. */
  int32_t dissipation;
  /* ckpt_stride: levels between the forward checkpoints tp_adjoint keeps
   * for the wave-speed gradient; 0 = the context does not compute it (> 0
   * also keeps a copy of the initial front at every tp_set_state). */
  int32_t ckpt_stride;
  /* tensor_cores: 0 = automatic: the mixed forward sweep with split
   *   right-hand sides (rhs_split > 1) runs the data moments and the outflow
   *   of single-material tents as exact digit products on the tensor cores
   *   (tcgen05): each float-float operand split into five signed 9-bit
   *   digits with a power-of-two scale per row (per column), the digit
   *   products summed exactly in binary32 tensor memory, i.e. contractions
   *   exact to ~2^-42 of the scales, as close as the compensated float-float
   *   sums they replace; used when the context's shared-memory plan allows
   *   it (nrhs / rhs_split * (dim + 2) <= 96, dim U^p <= 32, point chunks a
   *   multiple of 16 and at most 48; the CTA then takes one SM and all 512
   *   tensor-memory columns; multi-material tents keep the float-float sums;
   *   tp_ctx_tensor_cores reports the choice).  -1 = never (float-float sums
   *   on the CUDA cores). */
  int32_t tensor_cores;
} tp_params;

typedef struct tp_tents tp_tents;
typedef struct tp_basis tp_basis;
typedef struct tp_ctx tp_ctx;

const char* tp_last_error(void);

/* Tent pitching (Section 2.2; the edge-slope limited variant named in the
 * Section 6 setup).  Host only, deterministic, IEEE binary64 without fused
 * multiply-add:
 *   delta_e = (kappa * l_e) / c_e, l_e = sqrt(((dx0*dx0) + dx1*dx1) + dx2*dx2),
 *   c_e = max c over the elements of edge e;
 *   each round takes the local minima of tau (tau_v < T and tau_v <= tau_w for
 *   all neighbours w), keeps a greedy independent subset scanning v upward,
 *   and pitches v to t_top = min(T, min_w tau_w + delta_vw) at
 *   level = 1 + max(level of the last tents at v and at its neighbours).
 * Tents are stored sorted by (level, round, v); tents of one level are
 * independent.  Errors: TP_ERR_ARG for bad sizes/ids or non-positive
 * kappa, T or c. */
int tp_pitch_mesh(const tp_mesh_desc* mesh, const tp_params* prm, tp_tents** out);
int tp_tents_info(const tp_tents* tents, int64_t* n_tents, int32_t* n_levels);
/* Copies the sorted tent list into caller arrays of n_tents entries. */
int tp_tents_export(const tp_tents* tents, int32_t* vert, double* t_bot, double* t_top,
                    int32_t* level);
void tp_destroy_tents(tp_tents* tents);

/* Trefftz basis of U^p for c = 1 (Section 3, eq. 3.1, monomial initial data,
 * Remark 3.1 for the mapping to a tent).  Host tables, exact rationals
 * rounded once to binary64.  exps: nmono x (dim+1) exponents (t, x_1..x_n);
 * coef: nb x nmono coefficients of U.  dim in {1,2,3}, 1 <= p <= 8. */
int tp_build_basis(int32_t dim, int32_t p, tp_basis** out);
int tp_basis_info(const tp_basis* basis, int32_t* nb, int32_t* nmono);
int tp_basis_export(const tp_basis* basis, int32_t* exps, double* coef);
void tp_destroy_basis(tp_basis* basis);

/* Uploads mesh, tents, basis and quadrature tables to the current device and
 * allocates the front state (n_elem * Q * (dim+2) * nrhs doubles).  A tent
 * whose patch holds elements of several wave speeds gets one polynomial of
 * U^p per speed (Section 4.2), coupled through the time-like interface
 * facets.  The wave speeds are read from mesh, the tent times from tents:
 * tents pitched with other speeds on the same mesh are accepted (e.g. the
 * speeds perturbed with the space-time mesh held fixed); a top face that is
 * not space-like for the mesh's speeds is reported by the sweep
 * (TP_ERR_CAUSALITY through tp_sync_status).
 * Errors: TP_ERR_ARG on mismatched dim/p; TP_ERR_UNSUPPORTED when a
 * patch has more than 4 wave speeds, more than 64 elements or more than 16
 * boundary plus interface facets, or the shared-memory plan (dim U^p,
 * materials) does not fit one CTA even for one right-hand side; TP_ERR_OOM. */
int tp_create(const tp_mesh_desc* mesh, const tp_tents* tents, const tp_basis* basis,
              const tp_params* prm, tp_ctx** out);
/* n_front = n_elem * Q points, n_comp = dim + 2, n_bnd = number of Dirichlet
 * quadrature points over all tents, n_levels. */
int tp_ctx_info(const tp_ctx* ctx, int64_t* n_front, int32_t* n_comp, int64_t* n_bnd,
                int32_t* n_levels);
/* How tp_advance runs this context (chosen by tp_create or tp_autotune):
 * *dataflow = 1 for the persistent dataflow sweep, 0 for one launch per
 * level; *cluster = CTAs per tent (the largest, per level, with one launch
 * per level); *rhs_split = CTAs a tent's right-hand sides are split over
 * (1: not split); *rhs_groups = groups of right-hand sides swept one after
 * the other.  Any pointer may be NULL. */
int tp_ctx_schedule(const tp_ctx* ctx, int32_t* dataflow, int32_t* cluster, int32_t* rhs_split,
                    int32_t* rhs_groups);
/* *used = 1 when the context's forward sweep runs the data moments and the
 * outflow of single-material tents on the tensor cores (tp_params.tensor_cores),
 * 0 when it sums them on the CUDA cores.  Errors: TP_ERR_ARG for a null
 * context or pointer. */
int tp_ctx_tensor_cores(const tp_ctx* ctx, int32_t* used);
/* Front points (Section 4.1: one spatial rule mapped onto the faces):
 * host arrays xq (n_front x dim) and wq (n_front) physical weights. */
int tp_front_points(const tp_ctx* ctx, double* xq, double* wq);
/* Quadrature points (x, t) on the vertical boundary faces of every tent, in
 * sweep order: host array xt (n_bnd x (dim+1)).  The caller evaluates the
 * boundary data there: g_D on Dirichlet facets (eq. 2.1: v = g_D on
 * Gamma_D), g_N on Neumann facets (sigma.n = g_N on Gamma_N). */
int tp_boundary_points(const tp_ctx* ctx, double* xt);
/* For the same points: host arrays nrm (n_bnd x dim, the facet's outward unit
 * normal) and kind (n_bnd bytes, 0 = Dirichlet, 1 = Neumann); either may be NULL. */
int tp_boundary_kinds(const tp_ctx* ctx, double* nrm, int8_t* kind);
/* Sets the state at t = 0: d_front (device, front layout above, nrhs sets),
 * d_gD (device, nrhs x n_bnd boundary data at the points of
 * tp_boundary_points: g_D or g_N by the facet's kind; NULL for zero data).  Both are
 * copied; the front times are reset to 0.  Asynchronous on `stream`. */
int tp_set_state(tp_ctx* ctx, const double* d_front, const double* d_gD, void* stream);
/* Point outputs (Section 6.7 measures U_C(t) = ||U(., t)||_L1 over a small
 * box at every time): U_h at the samples (x_j, t_k) of n_pts points xq
 * (host, n_pts x dim, each inside some element) and n_t increasing times
 * (host).  Every sample lies in exactly one tent -- the one at a vertex of
 * x_j's element with t_bot(x_j) <= t_k < t_top(x_j) on that element (at the
 * final time: the tent whose top reaches it) -- and the forward sweep writes
 * U_h of that tent's solution there (Remark 3.1 map).  The assignment is
 * made here, on the host, for the context's tents; replaces earlier probes
 * (n_pts = 0 or n_t = 0: none); drops the captured forward graphs.
 * TP_ERR_ARG for a point outside the mesh or times that do not increase. */
int tp_set_probes(tp_ctx* ctx, int32_t n_pts, const double* xq, int32_t n_t, const double* times);
/* Copies the point outputs into d_out (device, nrhs x n_t x n_pts doubles,
 * [r][k][j]); samples no tent has reached since tp_set_state hold 0. */
int tp_get_probes(const tp_ctx* ctx, double* d_out, void* stream);
/* Resumes a sweep: copies a front (device, front layout) and the vertex
 * front times (device, n_vert doubles) into the context, e.g. the state
 * tp_get_state returned after some levels, so that tp_advance can continue
 * from the next level.  Boundary data, status and counters are kept. */
int tp_set_front(tp_ctx* ctx, const double* d_front, const double* d_tau, void* stream);
/* Bounds of the device-side loops (defaults for values <= 0, resp. < 0):
 * max_polls, the polls of a dependency wait of the dataflow sweep before it
 * reports TP_ERR_TIMEOUT (default 2^20, well under a second); max_refine,
 * the refinement steps after which a tent's solve falls back to the direct
 * binary64 LU (default 40; 0 sends every tent to the LU).  Drops the
 * context's captured graphs. */
int tp_set_limits(tp_ctx* ctx, int64_t max_polls, int32_t max_refine);
/* Failure injection for testing the bounded waits (the paper has no
 * counterpart): from now on tent `tent` of the sorted list waits for `extra`
 * more completions of each vertex it depends on than will ever come, so the
 * next dataflow sweep's wait runs out (TP_ERR_TIMEOUT through
 * tp_sync_status, first failing tent = `tent`; the other waits stop once the
 * error is flagged).  extra = 0 restores the true counts.  TP_ERR_ARG if the
 * tent waits for no earlier tent. */
int tp_inject_wait(tp_ctx* ctx, int64_t tent, int32_t extra);
/* Solve statistics since tp_set_state (synchronises the context's last
 * stream): *direct_lu = tents solved by the direct binary64 LU because their
 * refinement did not settle (or max_refine is 0); hist[k] = tents whose
 * refinement settled after k steps, k < nhist (steps beyond 40 are 0). */
int tp_solve_stats(tp_ctx* ctx, int64_t* direct_lu, int64_t* hist, int32_t nhist);
/* Solves every tent of one level (1-based) of the sorted tent list:
 * assembly of eq. (4.1) with the Section 5 recovery terms (and the
 * interface terms of eq. 2.5 on multi-material tents), LU solve in the
 * context's precision, outflow written at the top points (Section 4.1).
 * One launch; levels must be solved in increasing order. */
int tp_solve_layer(tp_ctx* ctx, int32_t level, void* stream);
/* Levels [level_begin, level_end) (1-based, end exclusive) as one CUDA graph
 * (captured on first use for that range, then replayed).  With the dataflow
 * schedule the graph holds one small setup kernel and one persistent sweep
 * kernel; with TP_SCHED_LEVELS, one launch per level. */
int tp_advance(tp_ctx* ctx, int32_t level_begin, int32_t level_end, void* stream);
/* Autotuner of the sweep schedule (the paper has no counterpart): times a
 * full forward sweep of this context with one launch per level and with the
 * dataflow schedule at cluster sizes 1, 2, 4 and 8 (state saved and
 * restored), keeps the fastest for later tp_advance calls and caches it for
 * this process under (dim, p, nrhs, precision, rounded mean vertex-star size),
 * so contexts created later with the same key start from it.  *chosen = 0 for
 * one launch per level, else the cluster size; *best_ms = its sweep time.
 * Allocates a scratch copy of the state; synchronises `stream`. */
int tp_autotune(tp_ctx* ctx, void* stream, int32_t* chosen, double* best_ms);
/* Energy flux through the current front (Section 6.5 energy generalised to
 * a front t = tau(x)):  E_r = 1/2 sum_K sum_q w_q (c_K^-2 v^2 + |sigma|^2
 * - 2 v sigma.grad tau_K) for every rhs r; equals the paper's E on a flat
 * front.  And the energy the tents swept since tp_set_state have lost,
 * D_r = sum over tents of 1/2 int_bot Q(u - u_b) + int_bot (U - U_b) U
 * + int_D [alpha v^2 - g_D (alpha v - sigma.n)] + int_N [beta (sigma.n)^2
 * - g_N (beta sigma.n - v)] + int_time [alpha [[v]]^2 + beta [[sigma]]_N^2]
 * (eq. 2.5 and eq. 4.1 tested with each tent's own solution, Section 6.5),
 * accumulated in binary64 when the context was created with
 * tp_params.dissipation = 1, else 0.  The method conserves energy inside
 * each Trefftz tent, so E_r(now) = E_r(t = 0) - D_r.
 * d_out: device array of 2 nrhs doubles, (E_r, D_r) for r = 0 .. nrhs-1. */
int tp_energy(tp_ctx* ctx, double* d_out, void* stream);
/* Adjoint sweep (the paper has none; it differentiates the method of
 * Section 4).  With the tents fixed, the sweep maps the initial front to
 * the final one through the tent maps b = B f_bot (+ boundary data),
 * A x = b, f_top = E x of eq. (4.1) with the Section 5 recovery terms, so a
 * functional J of the final front with gradient d_lambda_T (device, front
 * layout, nrhs sets) has
 *   d_lambda_0 (device, same layout): dJ/d(initial front), F^* applied tent
 *     by tent in reverse level order (mu = A^-T E^T lambda_top,
 *     lambda_bot = B^T mu), binary64;
 *   d_dJ_dc (device, n_elem doubles, or NULL): dJ/dc, c the wave speed, with
 *     the tents held fixed: every tent adds
 *       lambda_top . (dE/dc) x + mu^T ((dB/dc) f_bot - (dA/dc) x),
 *     evaluated at its points through dF/dc = ((t - t_c)/c) F(x') + (0, v/c, 0),
 *     x' = (c/h) D_t^T x (Remark 3.1: the basis of a material moves with its
 *     speed through t^ = c (t - t_c)/h); summed over the right-hand sides.
 *     Entry K holds the terms of element K's points (and of its facets): for
 *     a material of several elements (bitwise-equal c) their sum is dJ/dc of
 *     that material; with one speed per element it is dJ/dc_K.  The forward
 *     solutions come from sweeping again from the initial state of the last
 *     tp_set_state (the boundary data set there count as fixed), keeping a
 *     checkpoint every tp_params.ckpt_stride levels and recomputing one
 *     segment at a time.  Needs a context created with ckpt_stride > 0
 *     (TP_ERR_ARG otherwise) and every right-hand side in one group
 *     (TP_ERR_UNSUPPORTED otherwise); allocates its checkpoints on first use
 *     (TP_ERR_OOM).
 * The forward state is not touched.  Without d_dJ_dc the reverse sweep is
 * one CUDA graph. */
int tp_adjoint(tp_ctx* ctx, const double* d_lambda_T, double* d_dJ_dc, double* d_lambda_0, void* stream);
/* Copies the front (device, front layout) and/or the vertex front times
 * (device, n_vert doubles); either may be NULL. */
int tp_get_state(const tp_ctx* ctx, double* d_front, double* d_tau, void* stream);
/* Synchronises the context's last stream and reports the device status:
 * *status = TP_OK, TP_ERR_CAUSALITY (a top face not space-like),
 * TP_ERR_SINGULAR (zero or non-finite pivot of the direct LU) or
 * TP_ERR_TIMEOUT (a bounded dependency wait of the
 * dataflow sweep gave up); *info = index of the first failing tent in the
 * sorted list.  The first error wins; tp_set_state clears it. */
int tp_sync_status(tp_ctx* ctx, int32_t* status, int64_t* info);
void tp_destroy_ctx(tp_ctx* ctx);

/* Measured arithmetic peaks of the current GPU's plain ALUs (the paper has
 * no counterpart; the rooflines of the tent sweep use them): independent
 * chains of binary64 and binary32 fused multiply-adds on every SM, timed
 * with events (best of three after a warm-up launch), 2 flops per fused
 * multiply-add.  *fp64_tflops, *fp32_tflops in TFLOP/s.  Allocates a small
 * scratch array; synchronises `stream`. */
int tp_measure_alu_peaks(double* fp64_tflops, double* fp32_tflops, void* stream);

/* Allocation-free variant of tp_energy for callers that may not allocate
 * device memory at that point (a framework that has reserved the free device
 * memory in its own pool, or a service that fixes its device-memory budget at
 * start-up).  The paper has no counterpart; this is a library convenience.
 * Computes the same E_r as tp_energy from caller-owned device arrays, with no
 * context and no cudaMalloc/cudaFree:
 *   d_coords n_vert x dim, d_elems n_elem x (dim+1), d_c n_elem, d_tau n_vert
 *   (front times), d_wref Q reference weights of the front rule (summing to
 *   1/dim!, e.g. wq / |det J| of tp_front_points), d_front in the front layout,
 *   d_out nrhs doubles.
 * Scratch: a fixed 256 KiB module array (32768 partial sums) held by every
 * GPU that loads libtp until exit; nrhs > 32768 is rejected with TP_ERR_ARG.
 * The first call on a device looks up that array's address and should come
 * before any stream capture.  All calls share the array: calls that overlap
 * on the GPU race. */
int tp_front_energy_noalloc(int32_t dim, int64_t n_elem, int32_t Q, int32_t nrhs,
                            const double* d_coords, const int32_t* d_elems, const double* d_c,
                            const double* d_tau, const double* d_wref, const double* d_front,
                            double* d_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TP_H */
