/*
 * cgl.h — C ABI of the GB300 (sm_103a) implementation of the explicit SSP-RK
 * stage of the element-based convex-limited CG-WENO scheme of Kuzmin, Hajduk
 * and Vedral (arXiv 2509.04673).
 *
 * Problem statement (Sec. 2 of the paper): a hyperbolic conservation law
 * u_t + div f(u) = 0 on a rectangle, weakly imposed boundary data u_hat with
 * boundary flux F(u, u_hat; n), discretised by continuous Bernstein Q_p
 * finite elements on a uniform mesh of squares (Sec. 2.1), stabilised by
 * the WENO dissipation of eq. (stab:WENO), written as the element-based
 * monolithic convex limiting scheme of eq. (mcl) and advanced by SSP-RK3
 * stages of the form eq. (eq:SSPupdate).
 *
 * Conventions for every entry point:
 *   - return value: CGL_OK (0) or a negative error code; on error
 *     cgl_last_error() returns a thread-local message;
 *   - no C++ exception crosses this boundary;
 *   - host arrays of nodal coefficients are float64, layout
 *     [component][gy][gx] with gx fastest; a periodic direction of n
 *     elements has n*p nodes (the duplicate at the far side is not stored),
 *     a non-periodic one n*p + 1;
 *   - per-element host arrays are float64, layout [component][ey][ex];
 *   - the library owns every object it creates; destroy functions accept
 *     NULL;
 *   - a state is used from one host thread at a time; all its device work
 *     runs on the stream given at creation, and every function that returns
 *     host data synchronises that stream first;
 *   - the library uploads its constant tables (and finds the address of its
 *     no-allocation scratch) once per device and process; resetting a device
 *     (cudaDeviceReset) while the library is loaded is not supported.
 */
#ifndef CGL_H
#define CGL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int cgl_status;

#define CGL_OK 0
#define CGL_EINVAL (-1)     /* invalid argument or unsupported combination */
#define CGL_ECUDA (-2)      /* a CUDA call failed (no device, launch error) */
#define CGL_EOOM (-3)       /* device or host allocation failed */
#define CGL_EIDP (-4)       /* a node left the invariant domain beyond rounding */
#define CGL_ENONFINITE (-5) /* a non-finite value was produced */
#define CGL_EDT (-6)        /* the global time step collapsed */
#define CGL_ETIMEOUT (-7)   /* a bounded device-side wait gave up */

/* boundary conditions per direction (applied on both sides) */
#define CGL_BC_PERIODIC 0
#define CGL_BC_OUTFLOW 1    /* external state = internal state: F(u,u;n) = f(u).n */
#define CGL_BC_FIXED 2      /* constant external state cgl_problem.ubc */
#define CGL_BC_WALL 3       /* reflecting wall (Euler, cgl_set_boundary only):
                               u_hat = (rho, m - 2 (m.n) n, E) */

/* flux functions */
#define CGL_FLUX_ADVECTION 0 /* f(u) = (vx, vy) u */
#define CGL_FLUX_BURGERS 1   /* f(u) = (u^2/2, u^2/2) */
#define CGL_FLUX_KPP 2       /* f(u) = (sin u, cos u), Sec. 5.3.2 */
#define CGL_FLUX_EULER 3     /* compressible Euler, ideal gas, Sec. 5.2 */

/* method labels of Sec. 5.3: LO (gamma=beta=0), HO (gamma=beta=1),
   WENO (sensor gamma, beta=1), WENO-L (sensor gamma, limited beta) */
#define CGL_MODE_LO 0
#define CGL_MODE_HO 1
#define CGL_MODE_WENO 2
#define CGL_MODE_WENO_L 3

/* cell-average fluxes: 0 = high-order f^H (eq. (uebar)), 1 = flux-limited
   (eqs. (uelim), (fAlim) / Appendix A), 2 = low-order LLF f^L (eq. (uebar2)) */
#define CGL_FL_NONE 0
#define CGL_FL_LIMITED 1
#define CGL_FL_LOW 2

/* storage / arithmetic precision */
#define CGL_FP64 0        /* everything in float64 */
#define CGL_FP32_MIXED 1  /* bulk (state, sensor, residual, g_h, udot, f_i^e)
                             in float32; cell averages, pseudo time steps,
                             facet fluxes and their limiter, limiter bound gaps,
                             positivity tests, final nodal sums and
                             conservation sums in float64 */

typedef struct cgl_mesh cgl_mesh;
typedef struct cgl_state cgl_state;

/* Uniform mesh of nx x ny squares on [x0,x1] x [y0,y1] (Sec. 2.1, Table 1 of
   the paper). Requires (x1-x0)/nx == (y1-y0)/ny, 1 <= p <= 4, nx, ny >= 1.
   basis: CGL_BASIS_BERNSTEIN (0, the paper's basis) or CGL_BASIS_LGL (1):
   the Lagrange basis at the Legendre-Gauss-Lobatto points, the collocated
   spectral-element basis the paper's concluding section names as the next
   step.  On an LGL mesh the state holds nodal values at the LGL points of
   every element (node gx at x0 + (gx / p + xn[gx % p]) h, xn the Lobatto
   points on [0, 1]); the stage is the same with m_i^e = |K| w_a w_b (the
   LGL weights) in every lumped mass, cell average and face average.  LGL
   meshes run in the FP64 form only and take neither CGL_OPT_SUBCELL_DT (the
   subcell bound of Lemma 1 is stated for Bernstein elements) nor
   CGL_OPT_AEC_Q1 (CGL_EINVAL). */
#define CGL_BASIS_BERNSTEIN 0
#define CGL_BASIS_LGL 1
typedef struct cgl_mesh_desc {
    int32_t nx, ny, p;
    int32_t bc_x, bc_y;
    int32_t basis;
    double x0, x1, y0, y1;
} cgl_mesh_desc;

/* Problem parameters. cgl_problem_defaults() fills the paper's defaults:
   q = 1 (Sec. 5), r = 2 (Sec. 2.2), w_lin = 1e-3 (Sec. 5.4), gamma = 1.4
   (Sec. 5.2), omega_CFL = 0.2, k_g = k_u = 1. */
/* cgl_problem.options.  CGL_OPT_FP64_LIMITER: in the FP32-mixed form, evaluate
 * every Appendix-A positivity factor (facet and nodal limiter) with the float64
 * formula.  By default a float32 evaluation with a rigorous error bound first
 * certifies the factors that equal 1 and only the others are evaluated in
 * float64; the results are identical, the option exists to check that.
 * No effect in the FP64 form or for scalar fluxes. */
#define CGL_OPT_FP64_LIMITER 1
/* cgl_problem.options.  CGL_OPT_UNFUSED_SWEEPS: in the FP32-mixed form on meshes
 * of 2^22 nodes or more, run the right-hand sides of the g_h and udot solves and
 * their first Richardson sweeps as separate kernels.  By default they are
 * fused there (one kernel each); the results are identical, the option exists
 * to check that. */
#define CGL_OPT_UNFUSED_SWEEPS 2
/* cgl_problem.options.  CGL_OPT_SUBCELL_DT: the unlimited-flux variant of the
 * paper's Sec. 4.3 (step 4 with the flux limiter deactivated): the pseudo time
 * steps dt_e are the subcell bound dt_e^max of Lemma 1, eq. (dtmaxsubcell),
 * instead of the macrocell bound of eq. (dtmaxcell); the global dt is
 * omega_CFL min_e dt_e as before.  Requires flux_limiter = CGL_FL_NONE
 * (CGL_EINVAL otherwise).  u_0^e is the mean of the interior coefficients
 * (Q1: the cell average, with s = 2), c_ie = |S|/(p+1) times the summed
 * outward normals of the faces through boundary node i, a zero-speed node
 * term is dropped and the speed sum is floored at lambda_floor |S|. */
#define CGL_OPT_SUBCELL_DT 4
/* cgl_problem.options.  CGL_OPT_AEC_Q1: the element contributions of eq. (aecQ1)
 * (the paper's Sec. 5.3 variant, stated there for Q1, computed here for every p):
 *   f_i^e = gamma_e ( m_i^e (u_i - u^e) - dt_e [ int (phi_i - m_i^e/|K_e|) div f_h
 *                                                + int phi_i (udot^L_h - udot^L_i) ] )
 * with f_h = sum_j f(u_j) phi_j and the low-order time derivative
 * m_i udot^L_i = sum_e m_i^e (ubar^e - u_i)/dt_e of eq. (weak:low2) taken from
 * the stage's intermediate averages ubar^e.  The g_h projection, the target
 * residual and the udot solve are skipped.  The KPP entropy correction of that
 * section is not included.  Batched states (cgl_batch_create) reject this option
 * and CGL_OPT_SUBCELL_DT. */
#define CGL_OPT_AEC_Q1 8
/* cgl_problem.options.  CGL_OPT_DTE_REDUCE: the strategy of the remark after
 * eq. (dtmaxcell) for the unlimited averages of eq. (uebar): where the
 * macrocell dt_e gives ubar^e = u^e - (dt_e/|K_e|) sum |S| f^H outside G,
 * dt_e is decreased to the largest value that brings ubar^e back into G
 * (scalars: the crossed bound solved exactly; Euler: the Appendix-A
 * positivity criterion, margin pos_eps, for u^e moved along the step), and
 * that dt_e enters the element contributions and the SSP weights of the
 * element.  The global dt is not changed: theta = dt/dt_e > 1 is counted in
 * cfl_violations.  Requires flux_limiter = CGL_FL_NONE and neither
 * CGL_OPT_SUBCELL_DT nor CGL_OPT_AEC_Q1 (CGL_EINVAL otherwise); batched
 * states reject it.  Whether or not it is set, cgl_step_info.ubar_outside
 * counts the elements whose unlimited ubar^e left G. */
#define CGL_OPT_DTE_REDUCE 16

typedef struct cgl_problem {
    int32_t flux;          /* CGL_FLUX_* */
    int32_t mode;          /* CGL_MODE_* */
    int32_t flux_limiter;  /* CGL_FL_* */
    int32_t k_g;           /* Richardson sweeps of the g_h projection (>= 0) */
    int32_t k_u;           /* Richardson sweeps of the udot solve (>= 0) */
    int32_t options;       /* CGL_OPT_* bits, 0 by default */
    double vx, vy;         /* advection velocity */
    double gamma_gas;      /* Euler adiabatic constant, 1 < gamma <= 5/3 */
    double umin, umax;     /* scalar invariant domain G = [umin, umax] */
    double pos_eps;        /* Euler positivity margin (rho*, p* >= eps-fraction) */
    double q;              /* sensor steepening exponent, eq. (WENO:alpha) */
    double r;              /* WENO weight exponent */
    double weno_eps;       /* WENO weight epsilon */
    double w_lin;          /* linear weight of each face-neighbour candidate */
    double gamma_eps;      /* regulariser of the sensor ratio */
    double cfl;            /* omega_CFL: dt = cfl * min_e dt_e */
    double lambda_floor;   /* floor of the facet speed sum in eq. (dtmaxcell) */
    double ubc[4];         /* FIXED boundary state (ncomp values) */
} cgl_problem;

typedef struct cgl_step_info {
    double t;              /* time after the call */
    double dt_last;        /* last global time step */
    int64_t steps;         /* SSP-RK3 steps taken by the call */
    int64_t violations;    /* nodes outside G beyond rounding, summed over stages */
    int64_t clamps;        /* nodes clamped into G by rounding, summed over stages */
    int64_t cfl_violations;/* elements with dt > dt_e at a later stage */
    double mass[4];        /* sum_i m_i u_i per component after the call (float64) */
    double umin[4];        /* range of the coefficients after the call */
    double umax[4];
    int64_t ubar_outside;  /* flux limiter off: elements whose ubar^e of eq. (uebar) left G, summed over stages */
    int64_t dte_reduced;   /* CGL_OPT_DTE_REDUCE: elements whose dt_e was decreased, summed over stages */
} cgl_step_info;

/* --- library ------------------------------------------------------------ */

/* Thread-local message of the last failed call ("" if none). */
const char *cgl_last_error(void);

/* Library version string, e.g. "cgl 0.1 sm_103a". Never fails. */
const char *cgl_version(void);

/* Fill *p with the paper's defaults for the given flux kind (Sec. 5). */
cgl_status cgl_problem_defaults(cgl_problem *p, int32_t flux);

/* Export the library's own 1D Bernstein / Gauss tables of degree p (host
   computation, no GPU needed). out receives, in order: M, C, D, Ep, Em
   ((p+1)^2 each, row-major [a][b]), xq, wq (p+2 each), Bq, dBq
   ((p+2)(p+1) each, [q][a]) and the semi-norm matrix A ((p+1)^4, [i][j]).
   n must be at least the total count, returned in *needed. */
cgl_status cgl_debug_tables(int32_t p, double *out, size_t n, size_t *needed);

/* The same export for either basis (CGL_BASIS_BERNSTEIN, Sec. 2.1, or
   CGL_BASIS_LGL, the basis the concluding section names), followed by the
   weights int_0^1 phi_a and the node positions on [0, 1] (p+1 each). */
cgl_status cgl_debug_basis_tables(int32_t p, int32_t basis, double *out, size_t n, size_t *needed);

/* --- mesh ---------------------------------------------------------------- */

/* Validate a mesh description and create a mesh object (host only). */
cgl_status cgl_mesh_create(const cgl_mesh_desc *desc, cgl_mesh **out);
void cgl_mesh_destroy(cgl_mesh *mesh);

/* Node counts per direction and element count. */
cgl_status cgl_mesh_sizes(const cgl_mesh *mesh, int64_t *nnx, int64_t *nny, int64_t *nelem);

/* --- state ----------------------------------------------------------------- */

/* Allocate device storage for ncomp components (1 scalar, 4 Euler) of the
   given precision on the current CUDA device. stream is a cudaStream_t (or
   NULL: the library creates its own non-blocking stream). The mesh must
   outlive the state. Fails with CGL_ECUDA when no GPU is usable. */
cgl_status cgl_state_create(const cgl_mesh *mesh, int32_t ncomp, int32_t precision,
                            void *stream, cgl_state **out);
void cgl_state_destroy(cgl_state *state);

/* As cgl_state_create, but the nodal state itself lives in caller-owned device
   memory: u_device holds ncomp*nny*nnx values of the state's precision
   (float64 for CGL_FP64, float32 for CGL_FP32_MIXED), layout [comp][gy][gx]
   as in cgl_set_state, on the current device, 16-byte aligned, u_bytes at
   least that size.  Every stage reads and writes it in place, so a caller
   (for instance a framework tensor) sees the state without copies.  The
   caller keeps ownership; the memory must outlive the state, and nothing else
   may write it while a step is in flight on the state's stream.  All scratch
   is still allocated by the library.  CGL_EINVAL for a null, misaligned,
   too small or non-device pointer. */
cgl_status cgl_state_create_external(const cgl_mesh *mesh, int32_t ncomp, int32_t precision, void *u_device,
                                     size_t u_bytes, void *stream, cgl_state **out);

/* Set the problem (validated: flux/ncomp match, bounds, exponents, counts). */
cgl_status cgl_set_problem(cgl_state *state, const cgl_problem *prob);

/* Boundary data per side for cgl_set_boundary (Sec. 2 of the paper: the
   boundary flux F(u_h, u_hat; n) with weakly imposed data u_hat; the
   double Mach reflection of Sec. 5.4 combines a reflecting wall, a supersonic
   outlet and time-dependent inflow).  Side k: 0 = W (x = x0), 1 = E (x = x1),
   2 = S (y = y0), 3 = N (y = y1).  A boundary point whose coordinate along
   its side (y on W and E, x on S and N) lies below s_k(t) = s0[k] + s1[k] t
   takes kind_lo[k] / state_lo[k], every other point kind_hi[k] /
   state_hi[k]; t is the time of the SSP-RK stage (t, t + dt, t + dt/2 in
   cgl_step; the state's time in cgl_stage).  s0 = +inf gives one kind on the
   whole side.  Kinds: CGL_BC_OUTFLOW (u_hat = u), CGL_BC_FIXED (u_hat =
   state, ncomp values used), CGL_BC_WALL (u_hat = u with the normal momentum
   reversed; Euler only).  The data are taken at the Gauss points of a face
   in the residual, at the face nodes in the high-order facet fluxes and at
   the face midpoint in the low-order facet fluxes.  Sides on a periodic
   direction must carry CGL_BC_PERIODIC in both kinds. */
typedef struct cgl_boundary {
    int32_t kind_lo[4], kind_hi[4];
    double s0[4], s1[4];
    double state_lo[4][4], state_hi[4][4];
} cgl_boundary;

/* Replace the mesh's per-axis boundary conditions of the state with the
   per-side table b (copied), or restore them with b = NULL.  A table needs
   the problem set first.  CGL_EINVAL for an unknown kind, WALL with a scalar
   flux, a FIXED state outside G (scalar) or with rho <= 0 or p <= 0 (Euler),
   a NaN split or a non-finite s1.  A later cgl_set_problem checks the
   table against the new problem.  States with a table cannot be batched. */
cgl_status cgl_set_boundary(cgl_state *state, const cgl_boundary *b);

/* Copy n = ncomp*nny*nnx float64 coefficients from the host into the state
   (rounded to float32 in FP32_MIXED). The values pass through a float64
   staging buffer on the device (allocated at the first copy, 8 bytes per
   value, kept by the state), where they are checked and converted; a host
   buffer in pinned memory copies fastest. CGL_ENONFINITE (state unchanged)
   if any value is NaN or infinite. Synchronous. */
cgl_status cgl_set_state(cgl_state *state, const double *host, size_t n);

/* Nodal initialisation u_j(0) = u0(x_j) at the Bernstein nodal points x_j
   of the uniform sub-grid (spacing h/p; Sec. 5 sets the initial coefficients
   this way): u0(x, y, comp, ctx) is called on the host for every component
   and node, then the values are copied as by cgl_set_state.  Synchronous. */
cgl_status cgl_set_state_nodal(cgl_state *state, double (*u0)(double x, double y, int32_t comp, void *ctx),
                               void *ctx);

/* Copy the state to the host as float64 (exact widening in FP32_MIXED, on
   the device through the staging buffer). Synchronous. */
cgl_status cgl_get_state(cgl_state *state, double *host, size_t n);

/* Pipelined host copies, for a loop that feeds the state from the host and
   reads it back every step without waiting (an application; not in the
   paper).  cgl_set_state_async enqueues the copy of host (n float64 values,
   the layout of cgl_set_state) into one of two device staging buffers on a
   copy stream of the state, then, on the state's stream after the work
   enqueued before it, the finiteness check and the import; it returns
   without waiting, so the copy overlaps the steps still running.  A copy
   holding a non-finite value leaves the state as it was and is counted.
   cgl_get_state_async enqueues, on the state's stream, the export of the
   state as the work enqueued before it leaves it into one of two staging
   buffers, then its copy into host on a second copy stream, which overlaps
   the steps enqueued after it.  Both need host memory that is page-locked
   (cudaMallocHost, cudaHostRegister, a pinned torch tensor) for the copies
   to overlap, and the caller keeps each host buffer untouched until
   cgl_sync returns.  The staging buffers (4 x 8 n bytes) are allocated at
   the first call. */
cgl_status cgl_set_state_async(cgl_state *state, const double *host, size_t n);
cgl_status cgl_get_state_async(cgl_state *state, double *host, size_t n);

/* Wait for the state's work and its pipelined copies. CGL_ENONFINITE if a
   cgl_set_state_async since the last cgl_sync was refused (the count is
   reset); CGL_ECUDA on a CUDA error. */
cgl_status cgl_sync(cgl_state *state);

/* Set the base state u^n used by cgl_stage (same layout as cgl_set_state). */
cgl_status cgl_set_base_state(cgl_state *state, const double *host, size_t n);

/* Simulation time. */
cgl_status cgl_set_time(cgl_state *state, double t);
cgl_status cgl_get_time(cgl_state *state, double *t);

/* Advance min(nsteps, until t_end) SSP-RK3 steps with dt = cfl*min_e dt_e
   taken from u^n each step (capped at t_end - t). Pass t_end = +inf for a
   fixed step count. Returns CGL_EIDP if a node left G beyond rounding (the
   state is still advanced), CGL_ENONFINITE on NaN/Inf. info may be NULL. */
cgl_status cgl_step(cgl_state *state, int32_t nsteps, double t_end, cgl_step_info *info);

/* Enqueue nsteps SSP-RK3 steps (as cgl_step with the t_end of the last
   cgl_step call, +inf initially) on the state's stream and return without
   waiting or reading diagnostics; a later cgl_step / cgl_get_state /
   cgl_get_counters observes the result. */
cgl_status cgl_step_async(cgl_state *state, int32_t nsteps);

/* Cumulative counters since creation: out4 = {violations, clamps,
   cfl_violations, non-finite values}. Synchronises the stream. */
cgl_status cgl_get_counters(cgl_state *state, int64_t *out4);

/* One SSP stage with a given dt: u <- a u^n + b FE(u), FE(u) the forward
   Euler update eq. (eq:SSPupdate). With a = 0 the input state is also
   stored as the base state u^n (as the first stage of a step does). Used by
   parity tests. */
cgl_status cgl_stage(cgl_state *state, double dt, double a, double b, cgl_step_info *info);

/* Global dt = cfl * min_e dt_e of the current state (eq. (dtmaxcell)). */
cgl_status cgl_time_step(cgl_state *state, double *dt);

/* Per-element intermediates of the last stage, float64 [comp][E] or [E]. */
#define CGL_FIELD_UE 0      /* u^e        (ncomp x E) */
#define CGL_FIELD_DTE 1     /* dt_e       (E)         */
#define CGL_FIELD_UBL 2     /* ubar^{e,L} (ncomp x E) */
#define CGL_FIELD_UBE 3     /* ubar^e     (ncomp x E) */
#define CGL_FIELD_GAMMA 4   /* gamma_e    (E)         */
#define CGL_FIELD_NU 5      /* nu_e       (E)         */
#define CGL_FIELD_BETA 6    /* beta_e     (E)         */
/* Nodal intermediates of the last stage, float64 [v][nny][nnx]. */
#define CGL_FIELD_GX 16     /* g_h x-components (ncomp) */
#define CGL_FIELD_GY 17     /* g_h y-components (ncomp) */
#define CGL_FIELD_R 18      /* target residual r (ncomp) */
#define CGL_FIELD_UDOT 19   /* udot (ncomp); udot^L of eq. (weak:low2) with CGL_OPT_AEC_Q1 */
cgl_status cgl_get_field(cgl_state *state, int32_t field, double *host, size_t n);

/* --- batches ------------------------------------------------------------------ */

/* Many independent scalar instances (uneven sizes, degrees 1..4, own time
   steps) advanced together: per SSP-RK stage one persistent cooperative
   launch for each degree present, over all instances of that degree (a
   kernel compiled for the degree, with its own register budget), all
   launches of a step captured in one CUDA graph. Every state must be FP32_MIXED, scalar (advection, Burgers, KPP),
   on one device, with the same mode, k_g and k_u; the batch uses the first
   state's stream and references (does not copy) the states, which must
   outlive it. A batched instance evolves bitwise like the same state stepped
   alone with cgl_step. The batch copies each state's problem parameters at
   creation: a later cgl_set_problem or cgl_set_boundary on a member state
   is not seen by the batch (create a new batch after changing them). */
typedef struct cgl_batch cgl_batch;
cgl_status cgl_batch_create(cgl_state *const *states, int32_t n, cgl_batch **out);
void cgl_batch_destroy(cgl_batch *batch);

/* nsteps SSP-RK3 steps of every instance; *violations receives the summed
   invariant-domain violation counters of the instances (cumulative).
   CGL_ETIMEOUT if a grid barrier gave up (the instances are then undefined). */
cgl_status cgl_batch_step(cgl_batch *batch, int32_t nsteps, int64_t *violations);

/* Enqueue nsteps steps without waiting. */
cgl_status cgl_batch_step_async(cgl_batch *batch, int32_t nsteps);

/* Launch geometry: the largest persistent grid of the per-degree kernels,
   its block size (also the phase form's element blocks), tile counts
   (summed over the degrees), and how
   a step runs: 1 = a captured CUDA graph, 0 = no step has run yet (the
   graph is captured at the first step), -1 = the capture failed and steps
   run as direct cooperative launches (same results; cgl_last_error() then
   names the CUDA error of the capture). */
cgl_status cgl_batch_info(cgl_batch *batch, int32_t *grid, int32_t *block, int32_t *elem_tiles,
                          int32_t *node_tiles, int32_t *graph);

/* How a batch step runs.  CGL_BATCH_PERSISTENT (the default): per SSP-RK
   stage one persistent cooperative launch for each degree present, its
   phases separated by bounded grid barriers.  CGL_BATCH_PHASES: the same
   phases (the same device functions, so the same bits) as one launch each,
   one block per tile, so that every phase has the register budget of its
   own code; the update and residual phases are split in two launches each
   as in the single-state stage, element tiles take 128-thread blocks and
   node tiles 256-thread blocks; each degree's launches run on a stream of
   their own inside the step's graph, so the degrees overlap.  Changing the form waits for the
   batch's stream and captures a new graph at the next step.  (Batching is an
   application of the stage; the paper has no counterpart.) */
#define CGL_BATCH_PERSISTENT 0
#define CGL_BATCH_PHASES 1
cgl_status cgl_batch_set_form(cgl_batch *batch, int32_t form);
cgl_status cgl_batch_get_form(cgl_batch *batch, int32_t *form);

/* Element-tile length per degree (tile_elems[p], p = 1..4, in [1, 128]). */
cgl_status cgl_batch_set_tiles(cgl_batch *batch, const int32_t *tile_elems);
cgl_status cgl_batch_get_tiles(cgl_batch *batch, int32_t *tile_elems);

/* Autotuner: coordinate search of the tile length of every degree present
   (32, 64, 96, 128), each trial timed over `steps` steps with CUDA events
   (the states advance). Writes {"block", "tile_elems", "ms_per_step"} as
   JSON to json_path unless it is NULL. */
cgl_status cgl_batch_autotune(cgl_batch *batch, int32_t steps, const char *json_path);
cgl_status cgl_batch_load_tuning(cgl_batch *batch, const char *json_path);

/* TEST ONLY, not for production use: every grid barrier waits for
   phantom_blocks arrivals that never come (0 = normal) and gives up after
   spin_limit polls, so the timeout path (CGL_ETIMEOUT) can be exercised
   without any fault.  A batch with phantom_blocks > 0 cannot step; set 0
   and a spin limit again (or create a new batch) to use it. */
cgl_status cgl_batch_debug(cgl_batch *batch, int32_t phantom_blocks, int64_t spin_limit);

/* --- no-allocation entry point --------------------------------------------------- */

/* Lumped gradient projection of a scalar FP64 field, g = M_L^-1 b with
   b_i = sum_e int phi_i grad u_h (the first step of the g_h projection),
   computed without allocating any memory. The paper has no counterpart:
   this entry point exists for callers that cannot allocate device memory
   while they run (host callbacks, allocator hooks, real-time loops,
   embedders that only hand over fixed buffers).

   u: device pointer, nny*nnx float64 coefficients ([gy][gx]) of the mesh.
   g: device pointer, 2*nny*nnx float64 outputs, x-derivatives then
      y-derivatives, same layout; owned and allocated by the caller.
   stream: cudaStream_t or NULL; the call only enqueues work on it.

   The element-vector scratch lives in a fixed device array of 2^21 float64
   (16 MiB) that every GPU loading the library keeps until exit; meshes
   with nx*ny*(p+1)^2 > 2^20 are rejected with CGL_EINVAL. The first call on
   a device does a one-time set-up on that device (table upload, scratch
   address lookup), so make it before any stream capture. All calls share
   the scratch: calls that overlap on the GPU (on different streams, or from
   different threads) race and must be serialised by the caller. No part of
   the scratch needs to start at zero: every value read was written by the
   same call. */
cgl_status cgl_gradient_noalloc(const cgl_mesh *mesh, const double *u, double *g, void *stream);

/* --- measurement ------------------------------------------------------------ */

/* Name of kernel identifier id (identifiers are below 32), "" for an
   unused identifier. */
const char *cgl_kernel_name(int32_t id);

/* Run nsteps (1..1000) SSP-RK3 steps launch by launch (no graph, every
   kernel on the state's stream, the second stream's kernels included, so
   that no two kernels overlap) with CUDA events around every kernel; ms[id] and
   launches[id] receive the summed device time and the launch count per
   kernel identifier (nk >= 32). The state is advanced like cgl_step. */
cgl_status cgl_profile(cgl_state *state, int32_t nsteps, int32_t nk, double *ms, int64_t *launches);

/* Number of kernels one cgl_step step launches with the current problem. */
cgl_status cgl_launches_per_step(cgl_state *state, int64_t *kernels);

/* Arithmetic peaks of the current device, measured with CUDA events: the
   float64 and float32 fused multiply-add rates in FLOP/s (2 per FMA; eight
   independent FMA chains per thread, 8 blocks of 256 threads per SM, best of
   three timed launches after a warm-up).  They are the denominators of the
   arithmetic roofs the benchmark reports beside the HBM roof; the paper has
   no counterpart.  Allocates and frees a small device buffer; synchronises
   the device's default stream.  CGL_ECUDA without a usable GPU. */
cgl_status cgl_measure_peaks(double *fp64_flops, double *fp32_flops);

#ifdef __cplusplus
}
#endif

#endif /* CGL_H */
