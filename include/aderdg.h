/*
 * aderdg.h -- C ABI of the GB300 ADER-DG compressible Navier-Stokes hot path.
 *
 * Method: Krenz, Rannabauer, Bader, "A High-Order Discontinuous Galerkin
 * Solver with Dynamic Adaptive Mesh Refinement to Simulate Cloud Formation
 * Processes" (arXiv 1905.05524).  Sec. 2 (Eqs. 1-7) fixes the PDE: 2D
 * compressible Navier-Stokes with viscous flux, EOS with geopotential and
 * the hydrostatic perturbation split; Sec. 3 fixes the scheme family
 * (ADER-DG predictor/corrector, Rusanov-type viscous flux) and the
 * total-variation refinement indicator (Eqs. 6-8).
 *
 * Conventions (all functions):
 *   - return an int status, ADG_OK (0) on success; nothing throws or aborts;
 *   - adg_last_error() returns a thread-local text of the last failure;
 *   - the library owns each mesh and its device workspace; the caller owns
 *     every array it passes;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); all device work of a call is queued on it; only calls that
 *     return host data synchronise it;
 *   - `on_device` 1 means the pointer is a device pointer on the mesh's
 *     device, 0 means host memory (a get_state into host memory synchronises
 *     `stream`), ADG_COPY_HOST_ASYNC (2) means host memory copied
 *     asynchronously on `stream` without synchronising: the caller keeps the
 *     buffer alive and unchanged until the stream has passed the copy (page-
 *     locked memory makes the copy truly asynchronous); other values are
 *     ADG_EINVAL.
 *
 * State layout (set_state / get_state / adjoint vectors): double u[c][v][j][i]
 * with c = iy*nx + ix (row-major cells), v = rho, rho*u, rho*v, rho*E, and
 * j, i the y- and x-indices of the (N+1) x (N+1) Gauss-Legendre nodes of the
 * cell (nodal values).  count = nx*ny*(N+1)^2*4.
 */
#ifndef ADERDG_H
#define ADERDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define ADG_OK 0
#define ADG_EINVAL 1      /* bad argument (size, range, NULL)                */
#define ADG_ENOMEM 2      /* device or host allocation failed                 */
#define ADG_ECUDA 3       /* a CUDA runtime call failed (text kept)           */
#define ADG_ENONFINITE 4  /* a NaN/Inf was found in the state                 */
#define ADG_ETIMEOUT 5    /* a bounded device wait gave up                    */
#define ADG_ESTATE 6      /* wrong call order (e.g. corrector w/o predictor)  */
#define ADG_EUNSUPPORTED 7 /* option not built for this configuration         */

/* ---- options ---- */
#define ADG_BC_PERIODIC 0
#define ADG_BC_WALL 1       /* slip wall with background ghost (Sec. 4.2, Eq. 10) */
/* bc_y only, FP64 uniform meshes: the mesh is one horizontal strip of a
 * larger domain split across ranks; the marked sides take the neighbour
 * strip's face traces from halo buffers (adg_set_halo_traces) */
#define ADG_BC_EXCHANGE 2       /* south and north faces exchange            */
#define ADG_BC_WALL_EXCHANGE 3  /* south slip wall, north face exchanges     */
#define ADG_BC_EXCHANGE_WALL 4  /* south face exchanges, north slip wall     */
/* FP64 uniform meshes without gravity (the CFD scenarios of Sec. 4.1): */
#define ADG_BC_NOSLIP 5     /* no-slip wall: ghost density and pressure of the
                               interior, velocity 2 v_wall - v, interior
                               gradients, adiabatic; the north wall moves with
                               x-velocity lid_u (lid-driven cavity)            */
#define ADG_BC_ANALYTIC 6   /* the field bc_field imposed on the boundary: ghost
                               = the field's state and flux at the face node,
                               averaged over the step at the Gauss-Legendre
                               time nodes (Taylor-Green vortex)                */

#define ADG_SRC_NONE 0
#define ADG_SRC_STEADY 1    /* steady manufactured source rho = 1 + a sin(2pi(x+y)/L) */
#define ADG_SRC_PAPER 2     /* the paper's time-dependent manufactured solution (Sec. 4.1,
                               Eq. 8) with phi = 2pi/L (x+y) - 2pi t; FP64 uniform meshes */

#define ADG_PREC_FP64 0     /* every operation in FP64                          */
#define ADG_PREC_MIXED 1    /* FP32 predictor on perturbation variables; FP64
                               background split, pressure recovery and update   */
#define ADG_PREC_MIXED_TF32 2 /* ADG_PREC_MIXED with the predictor's derivative
                               contractions as tensor-core MMAs (TF32 operands
                               split in two, three products, FP32 accumulation); uniform
                               meshes of degree 3, 5, 7 (ADG_EUNSUPPORTED
                               otherwise).  Measured slower than ADG_PREC_MIXED
                               on this GPU; kept as the tensor-core form of the
                               contractions.                                     */
#define ADG_PREC_MIXED_BF16X3 3 /* as ADG_PREC_MIXED_TF32 with BF16 operands: each
                               operand split exactly in three BF16 numbers, the
                               six largest products accumulated in FP32 by three
                               m16n8k16 MMAs (a product within about 2^-21 of
                               exact); the same meshes as ADG_PREC_MIXED_TF32. */

#define ADG_TV_RHO 0
#define ADG_TV_THETA 1      /* potential temperature theta = T (p0/p)^(R/cp)  */

#define ADG_MAX_DEGREE 7

#define ADG_COPY_HOST_ASYNC 2 /* on_device value: host memory, asynchronous copy */

typedef struct adg_mesh adg_mesh;

/* Mesh and physics description.  A uniform nx x ny mesh on
 * [x0, x0+Lx] x [y0, y0+Ly]; y is the vertical (z) coordinate of Eqs. 2, 6, 7. */
typedef struct adg_mesh_desc {
    int degree;            /* polynomial degree N, 1..ADG_MAX_DEGREE             */
    int nx, ny;            /* cells per direction, >= 1                          */
    double x0, y0, Lx, Ly; /* domain box                                         */
    int bc_x, bc_y;        /* ADG_BC_* per direction                             */
    double gamma, Pr, R, mu; /* Eqs. 2-5: heat-capacity ratio, Prandtl number,
                                gas constant, viscosity                          */
    int gravity;           /* 1: gravity source -g rho' and hydrostatic split    */
    double g, p0, theta0;  /* gravity, reference pressure, background theta      */
    int source;            /* ADG_SRC_*                                          */
    double src_a, src_L, src_U, src_p; /* parameters of ADG_SRC_STEADY            */
    int precision;         /* ADG_PREC_*                                         */
    int device;            /* CUDA device ordinal                                */
    int max_levels;        /* 0: uniform mesh; 1..4: adaptive 3:1 tree with up to
                              this many refinement levels above the nx x ny base
                              (see adg_adapt); with ADG_PREC_MIXED the predictor
                              runs in FP32 on perturbations and the corrector,
                              hanging faces and TV in FP64                        */
    double lid_u;          /* ADG_BC_NOSLIP: x-velocity of the north wall (the
                              lid of the driven cavity, Sec. 4.1); others rest    */
    int bc_field;          /* ADG_BC_ANALYTIC: the imposed field, ADG_FIELD_*     */
} adg_mesh_desc;

#define ADG_FIELD_NONE 0
#define ADG_FIELD_TAYLOR_GREEN 1 /* Sec. 4.1: rho = 1, v = e^{-2 mu t} (sin x cos y,
                                    -cos x sin y), p = e^{-4 mu t} (cos 2x + cos 2y)/4
                                    + 100/gamma                                     */

#define ADG_SCEN_STEADY 0       /* steady manufactured field of the source above */
#define ADG_SCEN_COSINE 1       /* cosine bubble theta' (Eq. 15, r/a reading)    */
#define ADG_SCEN_TWO_BUBBLES 2  /* Gaussian-tail warm + cold bubbles (Eqs. 12, 14) */
#define ADG_SCEN_BACKGROUND 3   /* unperturbed hydrostatic atmosphere (Eq. 6)     */
#define ADG_SCEN_PAPER 4        /* the Eq. 8 field at the mesh's time             */
#define ADG_SCEN_TAYLOR_GREEN 5 /* the Taylor-Green field at t = 0 (Sec. 4.1)     */
#define ADG_SCEN_CAVITY 6       /* fluid at rest, rho = 1, p = 100/gamma (Sec. 4.1) */

typedef struct adg_scenario {
    int kind;              /* ADG_SCEN_*                                         */
    double A, a, xc, zc;   /* cosine bubble: amplitude, radius, centre           */
} adg_scenario;

/* Create a mesh: allocates the state and workspace on desc->device and builds
 * the basis (Gauss-Legendre nodes, derivative, time-stiffness matrices).
 * Errors: ADG_EINVAL (degree/size/options), ADG_ENOMEM, ADG_ECUDA. */
int adg_create_mesh(const adg_mesh_desc* desc, adg_mesh** out);

/* Free everything owned by the mesh; NULL-safe.  Synchronises the device. */
void adg_destroy_mesh(adg_mesh* m);

/* Number of doubles of the state: nx*ny*(N+1)^2*4. */
size_t adg_state_count(const adg_mesh* m);

/* Copy a state in / out (layout above).  count must equal adg_state_count;
 * ADG_EINVAL otherwise.  get_state with a host pointer synchronises `stream`. */
int adg_set_state(adg_mesh* m, const double* u, size_t count, int on_device, void* stream);
int adg_get_state(adg_mesh* m, double* u, size_t count, int on_device, void* stream);

/* Borrowed device pointer to the mesh's state (layout above, adg_state_count
 * doubles); valid until adg_destroy_mesh or adg_adapt.  NULL for a NULL mesh. */
double* adg_state_ptr(adg_mesh* m);

/* Simulation time carried by the mesh (advanced by adg_step). */
int adg_set_time(adg_mesh* m, double t);
double adg_get_time(const adg_mesh* m);

/* Nodal interpolation of a scenario's initial state (Sec. 4.1, 4.2). */
int adg_init_scenario(adg_mesh* m, const adg_scenario* s, void* stream);

/* Space-time predictor (Sec. 3, ADER-DG): n = N+1 Picard sweeps of the
 * element-local space-time polynomial, then the time-averaged volume
 * residual and the boundary-extrapolated face traces into the workspace. */
int adg_predictor(adg_mesh* m, double dt, void* stream);

/* Corrector: Rusanov-type viscous face flux (Sec. 3), weak-form lift and the
 * FP64 update u += dt * (volume - faces + source).  ADG_ESTATE unless the
 * last call on this mesh was adg_predictor with the same dt. */
int adg_corrector(adg_mesh* m, double dt, void* stream);

/* predictor + corrector; t += dt. */
int adg_step(adg_mesh* m, double dt, void* stream);

/* Largest stable dt for a CFL number (dt = CFL h / (2 (2N+1) max(|v| + c +
 * 2 eta lambda_v))).  Synchronises `stream`. */
int adg_stable_dt(adg_mesh* m, double cfl, double* dt, void* stream);

/* Total-variation refinement indicator of the current state (Sec. 3,
 * Eqs. 6-8): per-cell TV of `var` (ADG_TV_*), mean and population standard
 * deviation over all cells (Chan et al. parallel update, fixed combine
 * order), and flags +1 refine / 0 keep / -1 coarsen.  tv (double[cells]) and
 * flags (int8_t[cells]) are device pointers, either may be NULL; stats (host,
 * double[2] = mean, std) may be NULL; when it is not, `stream` is synchronised. */
int adg_tv_indicator(adg_mesh* m, int var, double T_r, double T_c,
                     double* tv, int8_t* flags, double* stats, void* stream);

/* One step followed by the TV indicator of the new state: the results of
 * adg_step then adg_tv_indicator with the same arguments (bitwise), but on
 * uniform meshes the corrector kernel evaluates the per-cell TV on the state
 * it has just written, saving one pass over the state and one launch
 * (Sec. 3: the indicator is evaluated after every step).  Adaptive meshes
 * run the two calls in turn.  Errors: those of both calls. */
int adg_step_tv(adg_mesh* m, double dt, int var, double T_r, double T_c, double* tv, int8_t* flags,
                double* stats, void* stream);

/* Discrete adjoint of one adg_step (predictor + corrector, FP64) at the
 * state u_n: lam_n = lam_np1 + (d step / d u)^T lam_np1, i.e. the gradient of
 * J(u^{n+1}) with respect to u^n given lam_np1 = dJ/du^{n+1} (the adjoint of
 * the method of Sec. 3, not a separate discretisation).  u_n, lam_np1, lam_n
 * are device arrays in the state layout; lam_n must not alias the inputs.
 * The mesh's own state is not touched; its predictor workspace is
 * (a following adg_corrector needs a new adg_predictor).  Non-smooth points:
 * max(s_L, s_R) takes s_L on ties and |v.n| takes sign(v.n) (0 at 0).
 * FP64 meshes with degree <= 5 (ADG_EUNSUPPORTED otherwise). */
int adg_step_adjoint(adg_mesh* m, double dt, const double* u_n, const double* lam_np1, double* lam_n,
                     void* stream);

/* ---- potential-temperature maps of the sensitivity problem (Sec. 4.2) ----
 *
 * Device arrays, uniform meshes (ADG_EUNSUPPORTED on adaptive ones), FP64,
 * queued on `stream`.  theta' arrays are nodal [c][j][i] (cells*(N+1)^2
 * doubles); states use the state layout above.
 *
 * adg_theta_to_state: the bubble initialisation of Sec. 4.2 (the reading
 *   that fixes pressure at the isentropic background, temperature
 *   (theta0 + theta') pi with the Exner function pi = 1 - g z/(cp theta0),
 *   fluid at rest, rhoE = pbar/(gamma-1) + rho g z), node by node: with the
 *   cosine theta' it is bitwise adg_init_scenario(ADG_SCEN_COSINE).  Needs
 *   gravity (ADG_EINVAL otherwise).
 * adg_theta_to_state_adjoint: lam_theta = (d u / d theta')^T lam_u at theta_p.
 * adg_state_to_theta: theta' = T (p0/p)^(R/cp) - theta0 at the nodes.
 * adg_probe_objective: J = sum_p (theta'(x_p) - target_p)^2, theta'
 *   interpolated by the cell's nodal Lagrange basis at the probe points
 *   probes_xy[2p], probes_xy[2p+1] (device, nprobes pairs; a point outside
 *   the mesh uses the nearest cell), target device [nprobes].  Writes the
 *   residuals theta'(x_p) - target_p to residual (device [nprobes]), J to
 *   *J (device scalar) and, if dJ_du is not NULL, dJ/du (device, state
 *   layout).  Sums run in a fixed order (bitwise reproducible). */
int adg_theta_to_state(adg_mesh* m, const double* theta_p, double* u, void* stream);
int adg_theta_to_state_adjoint(adg_mesh* m, const double* theta_p, const double* lam_u, double* lam_theta,
                               void* stream);
int adg_state_to_theta(adg_mesh* m, const double* u, double* theta_p, void* stream);
int adg_probe_objective(adg_mesh* m, const double* u, int nprobes, const double* probes_xy, const double* target,
                        double* residual, double* J, double* dJ_du, void* stream);

/* Strip decomposition (bc_y = ADG_BC_EXCHANGE*): the one exchange of an
 * ADER-DG step (Sec. 1: the scheme communicates once per step) is the face
 * trace of the cells along a strip edge.  After adg_predictor,
 * adg_get_boundary_traces copies the south-face traces of the first row and
 * the north-face traces of the last row to device arrays of nx*17*(N+1)
 * doubles each ([ix][component][node]; either pointer may be NULL).  The
 * caller sends them to the ranks below and above; adg_set_halo_traces
 * installs the traces received from the strip below (its north traces) and
 * above (its south traces) before adg_corrector.  ADG_EINVAL if bc_y has no
 * exchange side. */
int adg_get_boundary_traces(adg_mesh* m, double* south, double* north, void* stream);
int adg_set_halo_traces(adg_mesh* m, const double* south, const double* north, void* stream);

/* Refinement flags for given statistics: flags[c] from tv[c] against the
 * mean and population deviation of `count` values with sum of squared
 * deviations M2 (Eq. 7; used when the statistics are combined across ranks
 * with Chan's update).  tv, flags: device arrays of the mesh's cells.
 * Synchronises `stream`. */
int adg_tv_flags(adg_mesh* m, const double* tv, double count, double mean, double M2, double T_r, double T_c,
                 int8_t* flags, void* stream);

/* Scan the state for NaN/Inf: ADG_ENONFINITE if any.  Synchronises `stream`. */
int adg_check_finite(adg_mesh* m, void* stream);

/* ---- batched persistent step ----
 *
 * Many independent meshes ("instances", e.g. scenarios of different grid
 * sizes; the paper's method applied per instance, Sec. 3) advanced together:
 * per step one persistent predictor launch and one persistent corrector
 * launch walk a static list of tiles (instance, first cell) across all
 * instances; nsteps steps are captured once into a CUDA graph and replayed.
 * Instances may be uniform or adaptive (desc.max_levels > 0, Sec. 3's
 * dynamic AMR): the tiles of an adaptive instance cover its leaves of every
 * level, which run the adaptive mixed predictor and the FP64 corrector with
 * its hanging faces inside the same persistent launches.  After an
 * adg_adapt of a member, the next adg_batch_step synchronises the device,
 * rebuilds the instance tables and tile lists from the new leaves and
 * captures the graph again.
 * adg_batch_create times the predictor's candidates on the batch -- three
 * tile sizes of the node-per-thread body and, for batches of uniform
 * instances at degrees 3 and 5, the node-pair body (two nodes per thread) --
 * and keeps the fastest, cached per (degree, precision, SM count, size class,
 * number of candidates, adaptive or not) in memory and in a JSON file:
 * $ADG_TUNE_CACHE if set (an empty value keeps the cache in memory only),
 * else tune_cache.json beside the library; an entry found there is used
 * without timing.
 *
 * A batch of ADG_PREC_FP64 members runs the per-mesh FP64 predictor and
 * corrector bodies in the persistent launches, with one tile size (the
 * per-mesh cells per block) and no timing; its members are uniform meshes
 * without the time-dependent source (ADG_SRC_PAPER), analytic sides or strip
 * exchange, since the graph replays fixed arguments (ADG_EUNSUPPORTED).
 *
 *   meshes   k distinct meshes of one degree, device and precision, all
 *            ADG_PREC_MIXED or all ADG_PREC_FP64 (ADG_EINVAL for a mix,
 *            ADG_EUNSUPPORTED for the tensor-core precisions); they stay owned by
 *            the caller and must outlive the batch; their states are
 *            advanced in place
 *   dt       host array of k time steps (> 0), one per instance
 *   nsteps   steps per call (>= 1); each instance's time += nsteps * dt
 *   info     adg_batch_info fills up to n of: predictor tiles, cells per
 *            predictor tile, predictor grid, corrector tiles, cells per
 *            corrector tile, corrector grid, tuned time of candidates 0..2
 *            (ns; 0 when the cache decided), chosen candidate, where the
 *            choice came from (0 timed now, 2 cache), adaptive instances,
 *            tuned time of candidate 3 (ns)
 * adg_batch_step synchronises `stream` only when the dt array changed or a
 * member adapted. */
typedef struct adg_batch adg_batch;
int adg_batch_create(adg_mesh* const* meshes, int k, adg_batch** out);
int adg_batch_step(adg_batch* b, const double* dt, int nsteps, void* stream);
int adg_batch_info(const adg_batch* b, int* info, int n);
/* Pins the predictor's candidate (0, 1 or 2: half, default and double the
 * per-mesh node-per-thread cells per block; 3: the node-pair body with its
 * per-mesh cells per block at degrees 3 and 5 in a batch without adaptive
 * instances, candidate 1 otherwise) instead of the timed choice, e.g. to
 * reproduce a run or to test every candidate.  Synchronises the device
 * (the previous tile list may be in use by a launched step), rebuilds the
 * tile list and drops the captured graph.  ADG_EINVAL for a NULL batch or a
 * candidate outside 0..3; ADG_EUNSUPPORTED for an FP64 batch. */
int adg_batch_set_candidate(adg_batch* b, int cand);
void adg_batch_destroy(adg_batch* b);

/* ---- allocation-free step (the paper has no counterpart) ----
 *
 * One FP64 step (predictor + corrector, the same kernels as adg_step, so
 * the same results up to FP64 rounding of the background tables) on a
 * caller-owned device state, with no mesh object and no device allocation.  Meant for callers that must not call cudaMalloc: an
 * application whose pool allocator already owns the device memory, a
 * latency-critical loop that cannot take cudaMalloc's implicit device-wide
 * synchronisation, or a plug-in whose host forbids allocator calls.
 *
 *   desc   mesh/physics description (as for adg_create_mesh); precision must
 *          be ADG_PREC_FP64 and max_levels 0 (ADG_EUNSUPPORTED otherwise);
 *          at most 2^26 cells
 *   u      device pointer to the state (layout above), updated in place;
 *          count must equal nx*ny*(N+1)^2*4
 *   dt     time step (> 0)
 *
 * Scratch (background tables, volume residual, face traces) lives in a
 * fixed file-scope device array of ADG_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library holds until exit; meshes needing more scratch are
 * rejected with ADG_EINVAL and a message giving both sizes (at N = 5 about
 * 7,500 cells fit).  A call on a stream that is not capturing looks the
 * array's device address up (again, so a device reset cannot leave a stale
 * address); a call on a capturing stream reuses the address of the last
 * uncaptured call on that device, so the first call on a device must come
 * before any stream capture (ADG_ESTATE otherwise).  The work runs on
 * desc->device; the caller's current device is restored before returning,
 * and `stream` must belong to desc->device.  All calls share the array, so
 * calls whose work overlaps on the GPU (different streams, or different
 * threads on one device) race; serialise them.  Every scratch entry is
 * written before it is read within a call, so no state carries over between
 * calls. */
#define ADG_NOALLOC_SCRATCH_BYTES (32u << 20)
int adg_step_noalloc(const adg_mesh_desc* desc, double* u, size_t count, double dt, void* stream);

/* ---- adaptive mesh (desc.max_levels > 0) ----
 *
 * Refinement criterion of Sec. 3 (Eq. 7 flags from adg_tv_indicator) applied
 * on a 3:1 tree as in Sec. 4.2.  Leaves are ordered by (level, iy, ix); the
 * state, tv and flags arrays follow that order and their length changes with
 * every adaptation (adg_leaf_count).  Refinement: children = the parent
 * polynomial at their nodes; coarsening (all 9 siblings flagged -1, as the
 * paper requires): L2 projection; neighbours differ by at most one level,
 * refinement wins; hanging faces: the coarse side receives the L2 restriction
 * of the three fine numerical fluxes (conservative).
 *
 * adg_adapt: flags = device int8 per leaf (+1 refine, -1 coarsen, 0 keep);
 *   rebuilds the leaf list, transfers the state, reallocates the workspace;
 *   synchronises `stream`; writes the new leaf count to *leaves_out (may be
 *   NULL).  ADG_EINVAL on a uniform mesh.
 * adg_leaf_info: host int[3 * leaves] = (level, ix, iy) per leaf, ix/iy in
 *   units of that level's cells (a uniform mesh reports level 0). */
size_t adg_leaf_count(const adg_mesh* m);
int adg_leaf_info(const adg_mesh* m, int* out, size_t count);
int adg_adapt(adg_mesh* m, const int8_t* flags, int* leaves_out, void* stream);

/* ---- local time stepping across the levels of an adaptive mesh ----
 * (not in the paper, whose runs take one global dt from the finest cells)
 *
 * One cycle: the leaves of level l advance by dt * 3^(L-l), L the finest
 * level present, so the cycle advances the mesh by dt * 3^(L-l0) (l0 the
 * coarsest level), written to *cycle (host, may be NULL) and added to the
 * mesh time.  A level's step is its predictor over its whole step, three
 * steps of the next finer level, then its corrector.  At a hanging face the
 * fine side takes the coarse predictor's trace averaged over the third of
 * the coarse step its own step covers; the coarse side receives, per
 * spatial third of the face, the average of the fine numerical fluxes of its
 * three sub-steps (their L2 restriction, as for a global step) -- so the
 * scheme stays conservative.  On a mesh with one level present it is
 * adg_step.  dt is the finest level's step (from adg_stable_dt).  FP64
 * adaptive meshes of degree >= 2 (ADG_EUNSUPPORTED otherwise; ADG_EINVAL on
 * uniform meshes).  Queued on `stream`. */
int adg_step_lts(adg_mesh* m, double dt, double* cycle, void* stream);

/* ---- MUSCL-Hancock finite volumes (the paper's second scheme, Sec. 3) ----
 *
 * Unsplit MUSCL-Hancock on cell averages with the van Albada limiter, run
 * without viscosity as in the colliding-bubbles run of Sec. 4.2 ("as we use
 * limiting, we do not need any viscosity"): slopes of the perturbation from
 * the hydrostatic background (the atmosphere at rest is kept exactly), a
 * half-step evolution of the face states, Rusanov fluxes (s = |v.n| + c),
 * the perturbation form of Eq. 7 and slip walls with background ghosts.
 * The descriptor supplies nx, ny, the box, bc_x / bc_y (periodic or
 * ADG_BC_WALL), gamma, R, gravity, g, p0, theta0, precision and device; mu
 * must be 0.  precision ADG_PREC_FP64: FP64 throughout; ADG_PREC_MIXED: FP64
 * state, FP32 arithmetic on perturbations of the background (with gravity it
 * needs bc_y = ADG_BC_WALL, else ADG_EUNSUPPORTED).
 * State: double[4][ny][nx] cell averages of (rho, rho u, rho v, rho E).
 * adg_fv_step: one step of fixed dt (FP64: two kernels, face states at the
 *   half step, then fluxes and update; mixed: one fused kernel writing the
 *   second state buffer, which becomes the state, so a device pointer to the
 *   state is not stable across steps, and the FP32 perturbations of the new
 *   state for the next step; after adg_fv_set_state or adg_fv_init_scenario
 *   one more kernel first splits the state).  adg_fv_stable_dt: cfl / (max(|u| + c)/hx
 *   + max(|v| + c)/hy); synchronises `stream`.  adg_fv_init_scenario: cell
 *   centre values of ADG_SCEN_COSINE, ADG_SCEN_TWO_BUBBLES or
 *   ADG_SCEN_BACKGROUND (gravity on).  Errors as for adg_mesh. */
typedef struct adg_fv adg_fv;
int adg_fv_create(const adg_mesh_desc* desc, adg_fv** out);
void adg_fv_destroy(adg_fv* f);
size_t adg_fv_state_count(const adg_fv* f);
int adg_fv_set_state(adg_fv* f, const double* u, size_t count, int on_device, void* stream);
int adg_fv_get_state(adg_fv* f, double* u, size_t count, int on_device, void* stream);
int adg_fv_init_scenario(adg_fv* f, const adg_scenario* s, void* stream);
int adg_fv_step(adg_fv* f, double dt, void* stream);
int adg_fv_stable_dt(adg_fv* f, double cfl, double* dt, void* stream);

/* ---- Three dimensions (the ABC flow of Sec. 4.1, the 3D cosine bubble of
 * Sec. 4.2) ----
 *
 * The ADER-DG scheme above on a uniform nx x ny x nz mesh of degree N:
 * n = N+1 Picard sweeps of the space-time predictor, time-averaged
 * volume term and face traces, the Rusanov-type viscous flux and the FP64
 * update (one predictor and one corrector kernel per step).  z is the
 * vertical: gravity, the isentropic background (Eq. 6) and the perturbation
 * form (Eq. 7) act along z.
 *   desc   supplies degree (1..ADG_MAX_DEGREE_3D), nx, ny, x0, y0, Lx, Ly,
 *          bc_x, bc_y, gamma, Pr, R, mu, gravity, g, p0, theta0, device and
 *          bc_field; precision ADG_PREC_FP64 or ADG_PREC_MIXED (the predictor
 *          in FP32 on perturbations of the background, the corrector and the
 *          state in FP64); source ADG_SRC_NONE, max_levels 0
 *          (ADG_EUNSUPPORTED otherwise).
 *   nz, z0, Lz, bc_z   the vertical cells, origin, extent and boundary.
 * Boundaries per direction: periodic, ADG_BC_WALL (slip wall: background
 * rho, rhoE with gravity, reflected momentum, interior gradient, the
 * background heat flux of Eq. 10) or ADG_BC_ANALYTIC with bc_field
 * ADG_FIELD_ABC (no gravity; the field's state and flux averaged over the
 * step at the Gauss-Legendre time nodes).
 * State: double[nz*ny*nx][5][n][n][n], cell c = (iz*ny + iy)*nx + ix,
 * variables (rho, rho u, rho v, rho w, rho E), nodes [l (z)][j (y)][i (x)].
 * adg3_step: nsteps steps of fixed dt, advancing the mesh time.
 * adg3_stable_dt: cfl h_min / (3 (2N+1) max(|v| + c + 2 eta lambda_v));
 *   synchronises `stream`.
 * adg3_init_scenario: ADG_SCEN_COSINE (centre (xc, xc, zc): the paper sets
 *   yc = xc), ADG_SCEN_BACKGROUND (gravity on) or ADG_SCEN_ABC (the ABC field
 *   at the mesh time).  Errors as for adg_mesh. */
#define ADG_MAX_DEGREE_3D 4
#define ADG_FIELD_ABC 2         /* Sec. 4.1: rho = 1, v = e^{-mu t} (sin z + cos y,
                                   sin x + cos z, sin y + cos x), p = -e^{-2 mu t}
                                   (cos x sin y + sin x cos z + sin z cos y) + 100/gamma */
#define ADG_SCEN_ABC 7          /* the ABC field (3D meshes)                      */
typedef struct adg_mesh3 adg_mesh3;
int adg3_create(const adg_mesh_desc* desc, int nz, double z0, double Lz, int bc_z, adg_mesh3** out);
void adg3_destroy(adg_mesh3* m);
size_t adg3_state_count(const adg_mesh3* m);
int adg3_set_state(adg_mesh3* m, const double* u, size_t count, int on_device, void* stream);
int adg3_get_state(adg_mesh3* m, double* u, size_t count, int on_device, void* stream);
int adg3_set_time(adg_mesh3* m, double t);
double adg3_get_time(const adg_mesh3* m);
int adg3_init_scenario(adg_mesh3* m, const adg_scenario* s, void* stream);
int adg3_step(adg_mesh3* m, double dt, int nsteps, void* stream);
int adg3_stable_dt(adg_mesh3* m, double cfl, double* dt, void* stream);

/* Text of the last error on the calling thread ("" if none). */
const char* adg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ADERDG_H */
