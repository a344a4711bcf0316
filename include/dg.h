/*
 * dg.h -- C ABI of the GB300 (sm_103a) BP RI-OEDG solver for the 2D Euler
 * equations with P1/P2 modal DG on triangles.
 *
 * Method: Ding, Cui & Wu, "Robust DG Schemes on Unstructured Triangular
 * Meshes: Oscillation Elimination and Bound Preservation via Optimal Convex
 * Decomposition" (arXiv 2409.09620).  Section / equation labels below refer
 * to that paper.
 *
 * Conventions shared by every call:
 *  - All functions return int32_t status: DG_OK (0) or a negative DG_E* code;
 *    dg_last_error() returns a thread-local message for the last failure.
 *  - Pointers named host_* or documented as "host" are host memory; the
 *    library copies what it needs and never keeps a caller pointer.
 *  - The library owns every handle and every device allocation behind it.
 *  - A modal state is double coeffs[(c * nb + l) * nt + K]: component c in
 *    (rho, m1, m2, E), mode l in 0..nb-1 (nb = 3 for P1, 6 for P2, basis of
 *    eq. basisfunc, vertex v1 of each triangle is the origin of the
 *    reference map), cell K in 0..nt-1.
 *  - Triangles are counter-clockwise; local edge i is the edge opposite local
 *    vertex i (Fig. 1: e3 joins v1 and v2).
 */
#ifndef DG_GB300_H
#define DG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DG_OK 0
#define DG_EINVAL (-1)    /* bad argument */
#define DG_EMESH (-2)     /* invalid mesh: area <= 0, non-manifold, unmatched edge */
#define DG_ENOMEM (-3)    /* host or device allocation failed */
#define DG_ENONPHYS (-4)  /* a cell average left the admissible set G (eq. G:Euler) */
#define DG_ECUDA (-5)     /* CUDA runtime error */
#define DG_ETIMEOUT (-6)  /* a bounded device wait ran out */
#define DG_EBUSY (-7)     /* resource busy */

/* boundary tags for edges without a neighbour (bc[3 * K + i]) */
#define DG_BC_NONE 0          /* must have a neighbour (interior, or periodic via canon) */
#define DG_BC_REFLECT 1       /* mirror state (solid wall) */
#define DG_BC_TRANSMISSIVE 2  /* exterior state = interior trace */
#define DG_BC_DIRICHLET0 3    /* 3..6: constant state cfg.bc_state[tag - 3] */
#define DG_BC_SHOCK 7         /* moving oblique shock: post state behind, pre state ahead */

/* configuration values */
#define DG_PREC_FP64 0        /* every operation in FP64 */
#define DG_PREC_MIXED 1       /* FP32 modes and flux arithmetic; FP64 cell averages and limiter */
#define DG_OE_OFF 0
#define DG_OE_RI 1            /* rotation-invariant OE (Sec. 3.3) */
#define DG_OE_CW 2            /* component-wise OE (Sec. 3.2) */
#define DG_BP_OFF 0
#define DG_BP_ON 1            /* simplified BP limiter at the decomposition points (Sec. 4.4) */
#define DG_DECOMP_OPTIMAL 0   /* optimal convex decomposition (Sec. 4.2) and its CFL */
#define DG_DECOMP_ZXS 1       /* classical Zhang-Xia-Shu decomposition and its CFL */

typedef struct dg_mesh dg_mesh;
typedef struct dg_solver dg_solver;
typedef struct dg_batch dg_batch;
typedef struct dg_server dg_server;

typedef struct dg_config {
  int32_t k;              /* polynomial degree: 1 or 2 */
  int32_t precision;      /* DG_PREC_* */
  int32_t oe;             /* DG_OE_* */
  int32_t bp;             /* DG_BP_* */
  int32_t decomp;         /* DG_DECOMP_* */
  int32_t reserved;       /* set to 0 */
  double gamma;           /* adiabatic index (1.4 in Sec. 5.3) */
  double cfl;             /* multiplies the BP time step of Sec. 5 (1.0 = the paper's step) */
  double bc_state[4][4];  /* conservative Dirichlet states for tags 3..6 */
  double shock_x0;        /* moving shock: its line meets y = 0 at x = shock_x0 at t = 0 */
  double shock_angle;     /* angle of the shock line to the x-axis (radians) */
  double shock_speed;     /* speed of the shock along its normal */
  int32_t shock_pre;      /* index into bc_state of the state ahead of the shock */
  int32_t shock_post;     /* index into bc_state of the state behind the shock */
} dg_config;

typedef struct dg_stats {
  int64_t steps;          /* time steps taken by the call */
  int64_t limited_cells;  /* cell-stages with a limiter scaling theta < 1 */
  int64_t nonphysical;    /* cell-stages whose average left G before limiting */
  int64_t cfl_breaches;   /* stages whose alpha * dt exceeded min C_K |K| (reading of eq. 1009) */
  double t;               /* time reached */
  double dt_last;         /* last step size */
  double alpha;           /* viscosity coefficient (eq. 1250) of the current state */
} dg_stats;

/* ---------------------------------------------------------------------- */
/* Mesh (Sec. 2 notation; Sec. 4.2 decomposition)                          */
/* ---------------------------------------------------------------------- */

/* Build a mesh from host arrays: xy[2 * nv] vertex coordinates, tri[3 * nt]
 * counter-clockwise vertex ids, canon[nv] periodic vertex identity (NULL =
 * identity: vertices with equal canon are the same point of a periodic
 * domain), bc[3 * nt] boundary tags of edges without a neighbour (NULL = all
 * DG_BC_NONE).  Computes the neighbour of every edge on the host and the
 * per-cell geometry and optimal convex decomposition (eqs. 1040, 1139) on the
 * GPU.  Errors: DG_EINVAL (nt <= 0, nv <= 0, NULL arrays), DG_EMESH (vertex id
 * or canon id out of range, area <= 0, an edge whose canonical ends coincide,
 * an edge shared by more than two cells or traversed twice in the same
 * direction, two copies of a periodic edge that are not translates of each
 * other (to 1e-9 relative), a boundary edge tagged DG_BC_NONE or out of
 * range), DG_ENOMEM, DG_ECUDA.  These input checks run on the host before any
 * device call.  *out receives a handle owned by the caller
 * (dg_mesh_destroy). */
int32_t dg_mesh_create(int64_t nv, const double *xy, int64_t nt, const int32_t *tri,
                       const int32_t *canon, const int8_t *bc, dg_mesh **out);
void dg_mesh_destroy(dg_mesh *mesh);
/* number of cells; min over cells of C_{K,k} |K| (eqs. 1692, 1713, or the ZXS
 * numbers when decomp = DG_DECOMP_ZXS) for k = 1 and 2 */
int32_t dg_mesh_info(const dg_mesh *mesh, int32_t decomp, int64_t *nt, double *min_cfl_area_p1,
                     double *min_cfl_area_p2);
/* host copies of the adjacency: nbr[3 * nt] (-1 on a boundary) and the
 * neighbour's local edge nbr_edge[3 * nt] (-1 on a boundary) */
int32_t dg_mesh_neighbors(const dg_mesh *mesh, int32_t *nbr, int32_t *nbr_edge);
/* host copies of the device geometry for degree k: area[nt], len[3 * nt],
 * normal[6 * nt] (per cell and edge: nx, ny), c_area[nt] = C_{K,k} |K| of the
 * chosen decomposition, nodes[4 * nt] = reference coordinates (xi, eta) of the
 * two P2 internal nodes (eq. 1139), limv[2 * nt] = local ids of the P1
 * limiter vertices v1, v2 (opposite the longest and second-longest edges) */
int32_t dg_mesh_geometry(const dg_mesh *mesh, int32_t k, int32_t decomp, double *area, double *len,
                         double *normal, double *c_area, double *nodes, int8_t *limv);

/* physical points of the 12-point rule (Appendix A, Table tab:6th):
 * xy[(K * 12 + mu) * 2 + d] (host) */
int32_t dg_quad_points(const dg_mesh *mesh, double *xy);
/* L2 projection onto P^k with the 12-point rule: vals[(K * 12 + mu) * 4 + c]
 * are conservative point values at dg_quad_points (host); coeffs is a host
 * modal state (layout above) */
int32_t dg_project(const dg_mesh *mesh, int32_t k, const double *vals, double *coeffs);

/* ---------------------------------------------------------------------- */
/* Solver: the SSP-RK3 BP RI-OEDG scheme of Sec. 4.5                        */
/* ---------------------------------------------------------------------- */

/* Create a solver on `mesh` (the mesh must outlive it) with host initial
 * coefficients; applies the BP limiter once (the theorems assume the
 * solution at t^n satisfies eq. 1526), computes alpha and captures one SSP-RK3
 * step as a CUDA graph on `cuda_stream` (a cudaStream_t, or NULL for a
 * stream the solver creates).  Time starts at 0.  Errors: DG_EINVAL,
 * DG_ENONPHYS (an initial cell average is not in G), DG_ENOMEM, DG_ECUDA. */
int32_t dg_init(const dg_mesh *mesh, const dg_config *cfg, const double *coeffs, void *cuda_stream,
                dg_solver **out);
/* Advance until t >= t_end or max_steps steps, with dt from the BP CFL
 * condition (Sec. 5: dt = cfl * min_K C_K |K| / alpha, clamped to t_end).
 * Blocks until done.  stats may be NULL.  Returns DG_ENONPHYS if any cell
 * average left G during the call (the state is still advanced). */
int32_t dg_advance(dg_solver *solver, double t_end, int64_t max_steps, dg_stats *stats);
/* Enqueue exactly n steps (t_end = +inf) on the solver's stream and return
 * without synchronising; pair with dg_sync.  For device-side timing. */
int32_t dg_advance_async(dg_solver *solver, int64_t n);
int32_t dg_sync(dg_solver *solver, dg_stats *stats);
/* host copy of the current state (len = number of doubles available in
 * coeffs, at least 4 * nb * nt) and time (t may be NULL) */
int32_t dg_get_state(const dg_solver *solver, double *coeffs, size_t len, double *t);
/* replace the state (host coefficients, used as given, not limited) and time */
int32_t dg_set_state(dg_solver *solver, const double *coeffs, double t);
/* Run n steps with the kernels of the captured step launched one by one and a
 * CUDA event pair around each launch on the solver's stream (t_end is left as
 * set by the last dg_advance call; use dg_advance_async-style open-ended runs
 * for timing).  ms[q] and launches[q] receive the summed duration and launch
 * count of kernel kind q: 0 step_begin (dt), 1 rk (volume + edge flux + RK
 * combine), 2 fin_mean (domain means), 3 stats (deviation maxima and edge OE
 * records), 4 fin_dev (normalisers), 5 oe_bp (RIOE + limiter + traces), 6
 * fin_alpha (alpha, counters, time).  A step is 19 launches (13 with OE off). */
#define DG_NUM_KERNEL_KINDS 7
int32_t dg_profile_steps(dg_solver *solver, int64_t n, double *ms, int64_t *launches);
/* Measured FMA throughput of the current device: a kernel of independent
 * fused multiply-add chains (2 flops each) on every SM, timed with CUDA
 * events on cuda_stream (a cudaStream_t, NULL = the legacy default stream);
 * two launch shapes (8 or 16 chains per thread, 2048 or 1024 threads per
 * SM), each the best of three launches after a warm-up, about 10-20 ms each;
 * the faster shape's rate is reported.  precision
 * DG_PREC_FP64 measures DFMA, DG_PREC_MIXED measures FFMA.  *tflops receives
 * TFLOP/s and *ms (nullable) the launch time.  Not part of the paper: the
 * FP64 stage kernels are bound by the FP64 pipe on GB300, and this is the
 * peak their roofline fraction is taken against.  Errors: DG_EINVAL,
 * DG_ECUDA. */
int32_t dg_probe_fma_peak(int32_t precision, double *tflops, double *ms, void *cuda_stream);
/* the solver's CUDA stream (cudaStream_t) */
void *dg_stream(const dg_solver *solver);
void dg_solver_destroy(dg_solver *solver);

/* ---------------------------------------------------------------------- */
/* Single operators of one stage, on host buffers (for verification).      */
/* Each runs the same kernels as dg_advance on the solver's mesh/config.    */
/* ---------------------------------------------------------------------- */

/* u_h = a * un + b * (v + dt * L(v)) with the LF viscosity alpha and
 * boundary time t (eqs. DGSystem:Dis, RKTime) */
int32_t dg_op_rk_stage(dg_solver *solver, const double *un, const double *v, double a, double b,
                       double dt, double alpha, double t, double *uh);
/* global OE statistics of u (eqs. normOmg, RIOESys:Coef1): stats[0..3]
 * domain means, [4] sup |rho - mean|, [5] sup |m - mean m|, [6] sup |E - mean|,
 * [7] |Omega|, [8] sup |m1 - mean|, [9] sup |m2 - mean| */
int32_t dg_op_stats(dg_solver *solver, const double *u, double *stats);
/* OE procedure (eq. oe:sys with the RIOE coefficients) with the given stats;
 * the limiter is not applied; t is the time of boundary ghost states */
int32_t dg_op_oe(dg_solver *solver, const double *u, double dt, const double *stats, double t,
                 double *out);
/* BP limiter (Sec. 4.4); counters[0] += limited cells, counters[1] +=
 * cells with an average outside G */
int32_t dg_op_limit(dg_solver *solver, const double *u, double *out, int64_t *counters);
/* viscosity coefficient alpha of u at time t (eq. 1250) */
int32_t dg_op_alpha(dg_solver *solver, const double *u, double t, double *alpha);

/* ---------------------------------------------------------------------- */
/* Batches: many independent solves advanced together                      */
/* ---------------------------------------------------------------------- */

/* Create a batch of n independent solves (meshes[i], cfgs[i], host initial
 * coefficients coeffs[i]; k may differ between solves, the precision may not).
 * Each solve is set up as by dg_init on the batch's stream (NULL = a stream
 * the batch creates).  Launch forms: 3 = a stage of all solves walks a work
 * list of (solve, cell range) chunks in three phases (flux; OE statistics;
 * OE + limiter), one ordinary launch per phase (default); 1 = the same work
 * list in one persistent cooperative launch per stage with grid barriers
 * between the phases; 0 = every solve's own step kernels (those of its
 * single-solve step graph), the solves as independent branches of one graph
 * per step, so that small solves run side by side (needs graph support).  A
 * step is captured as a CUDA graph when the runtime supports it.  Every
 * solve keeps its own alpha, dt, t and OE normalisers, and its results are
 * bitwise those of the same solve run alone, in every form.
 * Errors as dg_init; DG_EINVAL if the precisions differ. */
int32_t dg_batch_create(int32_t n, const dg_mesh *const *meshes, const dg_config *cfgs,
                        const double *const *coeffs, void *cuda_stream, dg_batch **out);
void dg_batch_destroy(dg_batch *batch);
/* Advance every solve i until t_i >= t_end[i] (t_end NULL: +inf) or max_steps
 * steps; solves that reached their end time idle.  stats (nullable) receives n
 * entries.  In form 1, a grid barrier that waits longer than its limit (2 s
 * unless set by dg_batch_set_barrier) ends the launch early and the call
 * returns DG_ETIMEOUT. */
int32_t dg_batch_advance(dg_batch *batch, const double *t_end, int64_t max_steps, dg_stats *stats);
/* Wait limit of the grid barriers of the cooperative form (default 2 s per
 * wait; a block whose wait runs out ends the launch, and the next
 * dg_batch_advance / dg_batch_sync returns DG_ETIMEOUT after clearing the
 * barrier and the solves' finalisation tickets; the solves' states are then
 * those of an interrupted step, to be restored with dg_set_state).
 * extra_arrivals is a fault-injection hook for tests: it raises the number of
 * arrivals the barrier waits for above the grid size, so that every wait runs
 * out; 0 in normal use.  DG_EINVAL for timeout_ns <= 0 or extra_arrivals < 0.
 * The paper has no counterpart (the batch is an interface addition). */
int32_t dg_batch_set_barrier(dg_batch *batch, int64_t timeout_ns, int32_t extra_arrivals);
/* enqueue exactly n steps of every solve; pair with dg_batch_sync */
int32_t dg_batch_advance_async(dg_batch *batch, int64_t nsteps);
int32_t dg_batch_sync(dg_batch *batch);
/* the solver handle of solve i (owned by the batch): dg_get_state /
 * dg_set_state work on it; do not destroy it or advance it on its own */
int32_t dg_batch_solver(dg_batch *batch, int32_t i, dg_solver **out);
/* launch shape: cells per work chunk (a positive multiple of 128), resident
 * blocks per SM of each launch's grid (clamped per kernel to its occupancy
 * limit) and the launch form (3, 1 or 0, as for dg_batch_create; the chunk
 * and blocks-per-SM values do not apply to form 0).  DG_EINVAL for another
 * form, or form 1 on a device without cooperative launch; DG_ECUDA when form
 * 0's graph cannot be built.  *grid receives the largest grid of the form's
 * launches. */
int32_t dg_batch_set_shape(dg_batch *batch, int32_t cells_per_block, int32_t blocks_per_sm,
                           int32_t launches_per_stage);
int32_t dg_batch_shape(const dg_batch *batch, int32_t *cells_per_block, int32_t *blocks_per_sm,
                       int32_t *launches_per_stage, int32_t *grid, int32_t *graph);
/* Time `steps` steps for form 0 and, for forms 3 and 1, every
 * cells-per-chunk in {128, 256, 512, 1024} and every blocks-per-SM up to the
 * occupancy limit; keep the fastest and restore every solve's state, time and
 * counters.  The shape changes no result (partials are per 128 cells of each
 * solve). */
int32_t dg_batch_autotune(dg_batch *batch, int32_t steps, int32_t *best_cells_per_block,
                          int32_t *best_blocks_per_sm, int32_t *best_launches_per_stage,
                          double *best_ms_per_step);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of independent solve requests               */
/* ---------------------------------------------------------------------- */

#define DG_REQ_QUEUED 0
#define DG_REQ_RUNNING 1
#define DG_REQ_DONE 2
#define DG_REQ_FAILED 3

typedef struct dg_request_info {
  int32_t state;          /* DG_REQ_* */
  int32_t error;          /* status of a failed request (DG_ENOMEM: larger than the budget) */
  int64_t cells;
  int64_t steps;          /* time steps taken so far */
  double t, t_end;
  double submit_s;        /* server clock (s) at submission, admission and completion */
  double start_s;
  double done_s;
  int64_t device_bytes;   /* device memory charged against the budget while running */
} dg_request_info;

/* Create a server of solves in one precision with an HBM budget (bytes of
 * device memory its running solves may hold) and a number of time steps per
 * tick; work goes to cuda_stream (NULL = a stream the server creates). */
int32_t dg_server_create(int32_t precision, size_t hbm_budget_bytes, int32_t steps_per_tick,
                         void *cuda_stream, dg_server **out);
void dg_server_destroy(dg_server *server);
/* Queue a solve: host mesh arrays (as dg_mesh_create), configuration, host
 * initial coefficients and end time are copied; *id identifies the request. */
int32_t dg_server_submit(dg_server *server, int64_t nv, const double *xy, int64_t nt, const int32_t *tri,
                         const int32_t *canon, const int8_t *bc, const dg_config *cfg, const double *coeffs,
                         double t_end, int64_t *id);
/* One scheduling round: wait for the steps of the previous round; retire
 * solves that reached their end time (result copied to the host, device memory
 * released); admit queued requests in order while they fit in the budget
 * (mesh built, initial limiter applied); enqueue steps_per_tick steps of every
 * running solve in one persistent launch per stage and return without waiting
 * for them.  A request larger than the whole budget fails with DG_ENOMEM. */
int32_t dg_server_tick(dg_server *server, int32_t *n_running, int32_t *n_queued);
int32_t dg_server_request(const dg_server *server, int64_t id, dg_request_info *info);
/* host copy of a finished request's coefficients (layout as dg_get_state) */
int32_t dg_server_result(dg_server *server, int64_t id, double *coeffs, size_t len);
/* device bytes held by running solves; cell-stage updates of retired solves */
int32_t dg_server_stats(const dg_server *server, int64_t *bytes_in_use, int64_t *cell_stages_done);

/* ---------------------------------------------------------------------- */
/* Statistics without device allocation                                    */
/* ---------------------------------------------------------------------- */

/* The OE global statistics of dg_op_stats (domain means and sup deviations at
 * the volume points, stats[10] with the same layout) for callers that cannot
 * allocate device memory when they call: hosts whose device memory is
 * reserved by their own pool allocator, and loops that must not pay for an
 * allocation or its implicit synchronisation.  The paper has no counterpart:
 * this is an interface addition.
 *
 * coeffs is a DEVICE modal state [4][nb][nt] (layout above, nb from k) and
 * stats a DEVICE array of 10 doubles, both owned by the caller and on the
 * device that holds the mesh, which must be the current device; the work is
 * enqueued on cuda_stream (a cudaStream_t, NULL = the legacy default stream)
 * and the call returns without synchronising.  The call allocates nothing: its
 * scratch is a fixed 2.36 MB device array inside the library, which every GPU
 * that loads the library holds until exit.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress) with the device current,
 * so make the first call on each device before any stream capture.  All calls
 * on a device share the array and it keeps the last call's contents: calls
 * whose kernels overlap on the same GPU race.  Errors: DG_EINVAL (NULL
 * argument, k not 1 or 2, more than 4,194,304 cells, the current device is
 * not the mesh's), DG_ECUDA. */
int32_t dg_stats_noalloc(const dg_mesh *mesh, int32_t k, const double *coeffs, double *stats,
                         void *cuda_stream);

/* ---------------------------------------------------------------------- */
/* Scalar conservation laws u_t + div F(u) = 0: the OEDG scheme of Sec. 2   */
/* (DG operator eq. DGScalar:Dis with the LF flux eq. fluxLF; OE procedure  */
/* eqs. oe:scalar, OEScalar:Coef1, OEScalar:beta, OEScalar:Coef2; SSP-RK    */
/* eq. RKTime; the time step of Sec. 5), P1-P3, FP64, on any dg_mesh whose  */
/* boundary edges are transmissive or constant-state (tags 2..6).            */
/* State layout: coeffs[l * nt + K], l = 0..nb-1, nb = (k+1)(k+2)/2 modes of */
/* the basis eq. basisfunc (Psi^(0..9)).                                    */
/* ---------------------------------------------------------------------- */
#define DG_FLUX_LINEAR 0   /* F(u) = (ax u, ay u) */
#define DG_FLUX_BURGERS 1  /* F(u) = (u^2 / 2, u^2 / 2) */

typedef struct dg_scalar_config {
  int32_t k;          /* 1, 2 or 3 */
  int32_t flux;       /* DG_FLUX_LINEAR or DG_FLUX_BURGERS */
  int32_t oe;         /* 1: OE procedure after every stage; 0: plain RKDG */
  int32_t rk;         /* 2: SSP-RK(2,2), 3: SSP-RK(3,3) (both C_SSP = 1) */
  double ax, ay;      /* velocity of the linear flux */
  double cfl;         /* dt = cfl / alpha * min_K |K| / ((2k+1) sum_i l_K^(i)) (Sec. 5; 1 = paper) */
  double bc_state[4]; /* values of the constant-state boundary tags 3..6 */
} dg_scalar_config;

typedef struct dg_scalar dg_scalar;

/* L2 projection of point values vals[K * 12 + mu] at the 12-point rule's
 * points (dg_quad_points) onto P^k, k = 1..3 (host). */
int32_t dg_scalar_project(const dg_mesh *mesh, int32_t k, const double *vals, double *coeffs);
/* New solver on the device; coeffs are used as given (host, nb * nt doubles).
 * alpha^LF is the maximum of |F'(u) . n| over the edge Gauss points and both
 * traces of each stage input.  DG_EINVAL for a bad configuration or a
 * boundary tag other than 2..6. */
int32_t dg_scalar_init(const dg_mesh *mesh, const dg_scalar_config *cfg, const double *coeffs, void *cuda_stream,
                       dg_scalar **out);
/* Steps until t_end (the last step clamped) or max_steps; stats may be NULL
 * (steps, t, dt_last, alpha are filled).  DG_ENONPHYS if the state stops
 * being finite. */
int32_t dg_scalar_advance(dg_scalar *solver, double t_end, int64_t max_steps, dg_stats *stats);
/* Enqueue n steps (t_end = +inf) without synchronising. */
int32_t dg_scalar_advance_async(dg_scalar *solver, int64_t n);
void *dg_scalar_stream(const dg_scalar *solver);
int32_t dg_scalar_get_state(const dg_scalar *solver, double *coeffs, size_t len, double *t);
/* L1, L2 and L-infinity errors of the current state against exact values
 * exact[K * 12 + mu] at the 12-point rule's points (dg_quad_points), the
 * norms integrated with that rule: out3 = (L1, L2, Linf). */
int32_t dg_scalar_errors(const dg_scalar *solver, const double *exact, double *out3);
void dg_scalar_destroy(dg_scalar *solver);

/* thread-local message of the last failure in the calling thread */
const char *dg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
