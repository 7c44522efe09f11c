/*
 * liblskum: the per-iteration hot path of the implicit q-LSKUM 2D Euler solver
 * with the modified (exact-AD) LU-SGS scheme, on one GB300 GPU.
 *
 * The calls follow the statement of the problem in the paper (Verma, Mamidi,
 * Nemili, "GPU Accelerated Implicit Kinetic Meshfree Method based on Modified
 * LU-SGS", 2024): a point cloud with neighbour lists and point types (Sec. 4,
 * Alg. 1-3: wall, interior and outer points; Alg. 5: connectivity) and the
 * free-stream Mach number and angle of attack (Sec. 5) go in; the flow state
 * (Sec. 5), the density-residual history (Sec. 5.1) and the lift and drag
 * coefficients (Sec. 5.2, Table 5) come out.
 *
 * Conventions shared by every call:
 *  - All pointers are HOST pointers unless a name ends in _dev.
 *  - Inputs are copied; the caller keeps ownership of its arrays.
 *  - Point arrays are in the caller's point order; the library's internal
 *    (colour-sorted) order never leaks out.
 *  - Every call returns a status; no call aborts the process.  After a
 *    non-OK status the context stays valid for lskum_get_* (last good state),
 *    lskum_last_error and lskum_destroy.
 *  - A context is bound to the CUDA device current at lskum_create and to the
 *    stream given there (NULL = the legacy default stream).  Calls on one
 *    context must not overlap in time; different contexts are independent.
 */
#ifndef LSKUM_H
#define LSKUM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lskum_ctx lskum_ctx; /* opaque, owned by the library */

typedef enum {
    LSKUM_OK = 0,
    LSKUM_ERR_ARG = -1,         /* bad argument (NULL, size, flag value, option) */
    LSKUM_ERR_STENCIL = -2,     /* a point's (split) stencil is degenerate */
    LSKUM_ERR_NONPOSITIVE = -3, /* an update produced rho <= 0, p <= 0 or a non-finite value */
    LSKUM_ERR_DIVERGED = -4,    /* the residual norm became non-finite */
    LSKUM_ERR_CUDA = -5,        /* a CUDA runtime call failed */
    LSKUM_ERR_TIMEOUT = -6,     /* a bounded device wait gave up */
    LSKUM_ERR_OOM = -7          /* device or host allocation failed */
} lskum_status;

/* Point types (Alg. 2, 4): */
enum { LSKUM_INTERIOR = 0, LSKUM_WALL = 1, LSKUM_OUTER = 2 };

/* Jacobian-vector products in the LU-SGS sweeps: */
enum {
    LSKUM_JVP_EXACT = 0,    /* forward-mode derivative of the split fluxes (Sec. 3, Listing 3) */
    LSKUM_JVP_INCREMENT = 1 /* split-flux increments, Eq. 28 */
};

/* Fields readable with lskum_get_field (caller order; [N][4] row-major unless noted): */
enum {
    LSKUM_FIELD_U = 0,   /* conserved state [rho, rho u, rho v, rho e] (Eq. 2) */
    LSKUM_FIELD_Q = 1,   /* q-variables (Eq. 14) of the current state */
    LSKUM_FIELD_QX = 2,  /* x-derivatives of q of the last iteration (Eq. 16) */
    LSKUM_FIELD_QY = 3,  /* y-derivatives of q of the last iteration */
    LSKUM_FIELD_R = 4,   /* flux residual of the last iteration (Eq. 11-12, 19) */
    LSKUM_FIELD_D = 5,   /* scalar diagonal D of the last iteration, [N] (Eq. 26, 33-34) */
    LSKUM_FIELD_DUS = 6, /* forward-sweep increment dU* of the last iteration (Eq. 27) */
    LSKUM_FIELD_DU = 7   /* backward-sweep increment dU of the last iteration (Eq. 27) */
};

/*
 * The point cloud (all host pointers, copied at create):
 *   n_points  N >= 1
 *   x, y      f64[N] coordinates
 *   flag      u8[N]  LSKUM_INTERIOR / LSKUM_WALL / LSKUM_OUTER
 *   nx, ny    f64[N] unit normals: at wall points into the fluid; at outer
 *             points out of the domain (read there only under
 *             LSKUM_FARFIELD_KINETIC); read nowhere else.  Both NULL: the
 *             library computes them from the closed polygon of the wall
 *             points (and of the outer points) in caller order -- the
 *             central-difference tangent (next minus previous point)
 *             rotated to its right for a counter-clockwise polygon (to its
 *             left for a clockwise one): into the fluid at the wall, out of
 *             the domain at the far field (LSKUM_ERR_ARG for fewer than 3
 *             such points or a zero tangent)
 *   nbr_off   i32[N+1] CSR offsets, nbr_off[0] = 0, non-decreasing
 *   nbr_idx   i32[nbr_off[N]] neighbour indices: 0-based, < N, no self, no
 *             duplicates within a row.  The order within a row is the
 *             summation order of every neighbour sum.
 */
typedef struct {
    int32_t n_points;
    const double *x, *y;
    const uint8_t *flag;
    const double *nx, *ny;
    const int32_t *nbr_off, *nbr_idx;
} lskum_cloud;

/*
 * Solver options:
 *   mach, aoa_deg    free stream (rho = 1, p = 1/gamma, gamma = 1.4)
 *   cfl              local time-step factor (> 0)
 *   cfl_ramp_iters   if > 0, the CFL of iteration n (1-based) is
 *                    cfl * min(1, n / cfl_ramp_iters)
 *   inner_iters      K >= 0 defect-correction inner iterations of the
 *                    q-derivatives (Eq. 16)
 *   jvp              LSKUM_JVP_EXACT or LSKUM_JVP_INCREMENT
 *   precision        0 = FP64 everywhere; 1 = mixed: the LU-SGS sweeps and
 *                    their Jacobian products in FP32, the residual (with
 *                    compensated neighbour sums), norm and update in FP64
 *   first_order_iters  iterations n <= first_order_iters (counted since the
 *                    last set_state / create) use the first-order residual
 *                    (q~ = q: no defect correction); a start-up aid, >= 0
 *   scheme           LSKUM_SCHEME_LUSGS (0, the implicit solver) or
 *                    LSKUM_SCHEME_EXPLICIT (1, the paper's explicit solver:
 *                    forward Euler with the same local time step, no sweeps;
 *                    stable for cfl <= ~0.3; precision must be 0)
 *   lusgs            implicit solver's LU-SGS form (Sec. 3):
 *                    LSKUM_LUSGS_ANANDH (0): the scalar diagonal of the
 *                    split-flux spectral radii (Eq. 34), with the dominance
 *                    bound sum_s rho_s sum_i |w_i|;
 *                    LSKUM_LUSGS_MANISH (1): the revised form of Manish et
 *                    al.: Jameson's splitting gives D = 1/dt + sum_s
 *                    (|u_d| + a)|LS_s(1)|/2, and the term S_0 = -1/2 sum_s
 *                    LS_s(1) A_d(U_0) dU_0 of the previous iteration's
 *                    increment (exact unsplit Jacobian products) joins the
 *                    right-hand side as -R - S (the sign the algebra of the
 *                    split diagonal gives); converges faster at cfl ~ 2-3,
 *                    diverges at cfl >= ~7.  The lag restarts from dU = 0
 *                    after every new state.
 *   ordering         the LU-SGS sweep order: LSKUM_ORDER_COLOUR (0; all
 *                    points of a colour together, Alg. 6) or
 *                    LSKUM_ORDER_WALL_FIRST (1; the wall points colour by
 *                    colour, then the interior points colour by colour,
 *                    Alg. 4; the backward sweep is the exact reverse) or
 *                    LSKUM_ORDER_SERIAL (2; the serial sweeps of Alg. 2:
 *                    wall, interior and outer points, each in caller order,
 *                    no colouring; executed level by level over the
 *                    dependency graph this order induces -- a point's level
 *                    is one more than the highest among its earlier
 *                    neighbours -- which reproduces the sequential sweeps
 *                    exactly; as many levels as the longest dependency chain)
 *   farfield         the outer (far-field) points: LSKUM_FARFIELD_FREESTREAM
 *                    (0) holds them at the free stream (Dirichlet; they are
 *                    not swept); LSKUM_FARFIELD_KINETIC (1) makes them
 *                    unknowns like the others (the paper's sweeps visit them,
 *                    Alg. 2 and 4; it states no formula): in the frame (t, n),
 *                    n the outward normal, their residual is the t+, t- and
 *                    n+ split derivatives over their neighbours plus the
 *                    n- derivative against free-stream ghost points at the
 *                    mirror images of the n+ neighbours, LS_3(1)
 *                    (G_n^-(U_inf) - G_n^-(U_0)) with LS_3(1) = -LS_2(1):
 *                    molecules entering the domain carry the free-stream
 *                    Maxwellian (supersonic inflow and outflow alike).  They
 *                    are swept (last among equal colours, or after the
 *                    interior points in LSKUM_ORDER_WALL_FIRST), updated and
 *                    counted in the residual norms.
 */
enum { LSKUM_SCHEME_LUSGS = 0, LSKUM_SCHEME_EXPLICIT = 1 };
enum { LSKUM_LUSGS_ANANDH = 0, LSKUM_LUSGS_MANISH = 1 };
enum { LSKUM_ORDER_COLOUR = 0, LSKUM_ORDER_WALL_FIRST = 1, LSKUM_ORDER_SERIAL = 2 };
enum { LSKUM_FARFIELD_FREESTREAM = 0, LSKUM_FARFIELD_KINETIC = 1 };
typedef struct {
    double mach, aoa_deg, cfl, cfl_ramp_iters;
    int32_t inner_iters, jvp, precision, first_order_iters, scheme, lusgs, ordering, farfield;
} lskum_opts;

/*
 * Validate and copy the cloud, colour it (Alg. 5 on the symmetrised
 * neighbour graph), order points by colour (the LU-SGS sweep order, Alg. 6-7),
 * precompute stencil geometry, allocate device memory and set the free-stream
 * state (normal momentum removed at wall points).
 *   cloud, opts   host structures (not kept)
 *   cuda_stream   a cudaStream_t of the current device, or NULL
 *   out           receives the context; set to NULL on failure
 * Errors: LSKUM_ERR_ARG (bad input, with the offending point in
 * lskum_last_error(NULL)), LSKUM_ERR_STENCIL (a degenerate split sub-stencil),
 * LSKUM_ERR_OOM, LSKUM_ERR_CUDA.
 */
lskum_status lskum_create(const lskum_cloud *cloud, const lskum_opts *opts, void *cuda_stream,
                          lskum_ctx **out);

/*
 * Dry run (no counterpart in the paper): validate the clouds and options
 * exactly as lskum_batch_create does (n_cases = 1: as lskum_create), build
 * the host layout (colouring, sweep order and levels, slot lists) and check
 * its invariants: the sweep order is a permutation, every wall or interior
 * point (and every outer point under LSKUM_FARFIELD_KINETIC) lies in one
 * sweep level and frozen outer points in none, each level's sweep
 * orders are permutations of it, no two coupled points share a level, and
 * the lower / upper slot lists hold exactly the coupling slots of earlier /
 * later levels.  No device call is made.  n_colours, n_levels (may be NULL)
 * receive the counts.  Errors as lskum_create (LSKUM_ERR_ARG also for a
 * failed invariant, with the reason in lskum_last_error(NULL)).
 */
lskum_status lskum_validate(const lskum_cloud *clouds, const lskum_opts *opts, int32_t n_cases, int32_t *n_colours,
                            int32_t *n_levels);

/*
 * Batched solves (a serving extension; no counterpart in the paper): n_cases
 * independent flow problems, each with its own cloud and free stream, solved
 * together.  The context holds the disjoint union of the clouds (caller point
 * order: case 0's points, then case 1's, ...); one iteration launch covers
 * every case, colour level by colour level.  Each case keeps its own residual
 * history and drop test: a case that reaches the target stops updating while
 * the others continue, and lskum_run returns when all have stopped (or after
 * max_iters).  A case whose norm is not finite or whose update is
 * non-physical fails alone: it keeps its last good state, its status
 * (lskum_get_case_info) says why, and the others go on; lskum_run still
 * returns LSKUM_OK.  A failed case stays frozen until a new state is set.
 * opts[b] may differ only in mach and aoa_deg (LSKUM_ERR_ARG otherwise).
 * The single-case calls act on the whole union (state, fields) or on case 0
 * (residuals, forces).  Errors as lskum_create.
 */
lskum_status lskum_batch_create(const lskum_cloud *clouds, const lskum_opts *opts, int32_t n_cases, void *cuda_stream,
                                lskum_ctx **out);

/* Case cs (0 <= cs < n_cases): its residual history (as lskum_get_residuals),
 * its Cl and Cd (with its own Mach and AoA), and its first point in the
 * caller order of the union, its point count, the norms recorded, whether it
 * has stopped (target reached or failed) in the last run, its status
 * (LSKUM_OK, or LSKUM_ERR_DIVERGED / LSKUM_ERR_NONPOSITIVE for a failed case)
 * and, for LSKUM_ERR_NONPOSITIVE, the offending point (caller order of the
 * union; else -1).  Pointers other than the context may be NULL in
 * lskum_get_case_info. */
lskum_status lskum_get_case_residuals(lskum_ctx *ctx, int32_t cs, double *hist, int32_t cap, int32_t *n);
/* As lskum_get_case_residuals for the norms of all four residual components
 * (mass, x and y momentum, energy): hist4 f64[cap][4], n receives the count;
 * column 0 is the density history the drop test uses. */
lskum_status lskum_get_case_residuals4(lskum_ctx *ctx, int32_t cs, double *hist4, int32_t cap, int32_t *n);
lskum_status lskum_get_case_forces(lskum_ctx *ctx, int32_t cs, double *cl, double *cd);
lskum_status lskum_get_case_info(lskum_ctx *ctx, int32_t cs, int32_t *first_point, int32_t *n_points, int32_t *iters,
                                 int32_t *stopped, int32_t *status, int32_t *bad_point);

/* Device-pointer variants (no counterpart in the paper; for callers that keep
 * the state in device memory, e.g. torch tensors' data_ptr()):
 *   lskum_get_field_dev: like lskum_get_field into out_dev (device, caller
 *     order, same shapes), asynchronous: ordered after the work on
 *     cuda_stream, and cuda_stream is ordered after the copy (NULL = the
 *     legacy default stream).
 *   lskum_set_conserved_dev: like lskum_set_conserved from U_dev (device,
 *     f64[N][4], caller order, read after the work on cuda_stream); returns
 *     when the state is set, with cuda_stream ordered after it.
 * Errors as the host versions. */
lskum_status lskum_get_field_dev(lskum_ctx *ctx, int32_t field, double *out_dev, void *cuda_stream);
lskum_status lskum_set_conserved_dev(lskum_ctx *ctx, const double *U_dev, void *cuda_stream);

/* Host-array transfers (no counterpart in the paper).  Where the device can
 * read and write pageable host memory directly (cudaDevAttrPageableMemoryAccess,
 * as on a GPU attached to a Grace CPU), the calls that take or fill host
 * arrays (lskum_set_state, lskum_set_conserved, lskum_get_field,
 * lskum_get_state) reorder between the caller's array and the device layout
 * in one kernel, with no staging copy; otherwise one copy each way goes
 * through a device buffer.  Both give the same bits.  lskum_set_host_io
 * chooses: direct = 1 (LSKUM_ERR_ARG where it is not supported) or 0 (the
 * copies); a context starts with 0: on GB300 with a Grace host the direct
 * kernels read 4.7 MB in 0.12 ms (the copy path 0.13 ms) but write a fresh
 * array in 0.13 ms (0.05 ms), the device's first touches of new host pages
 * being faults.  lskum_get_host_io reports the mode in use and whether
 * direct access is supported (either pointer may be NULL). */
lskum_status lskum_set_host_io(lskum_ctx *ctx, int32_t direct);
lskum_status lskum_get_host_io(lskum_ctx *ctx, int32_t *direct, int32_t *supported);

/* Replace the state by primitive fields (f64[N] each, caller order); the wall
 * projection is applied and the residual history is cleared.
 * Errors: LSKUM_ERR_ARG (NULL), LSKUM_ERR_NONPOSITIVE (rho or p <= 0 or not
 * finite; state unchanged), LSKUM_ERR_CUDA. */
lskum_status lskum_set_state(lskum_ctx *ctx, const double *rho, const double *u, const double *v,
                             const double *p);

/* Replace the state by conserved variables U f64[N][4] (caller order), keeping
 * the residual history (resume from a checkpoint).  U is taken as given, with
 * no wall projection, so a state read with lskum_get_field(LSKUM_FIELD_U)
 * resumes bit for bit (re-projecting a projected state can move its last
 * bit); every update projects the wall points it moves.  Same errors as
 * above. */
lskum_status lskum_set_conserved(lskum_ctx *ctx, const double *U);

/*
 * Run up to max_iters pseudo-time iterations of Alg. 1 on the device:
 * q-derivatives (K inner iterations), flux residual and diagonal, density
 * residual norm, forward and backward sweeps, state update.  After iteration n
 * the run stops early if norm_n / norm_1 <= target_drop (norm_1 = the first
 * norm since the last set_state / create); target_drop <= 0 runs all
 * iterations.  iters_done (may be NULL) receives the number of iterations run.
 * Errors: LSKUM_ERR_NONPOSITIVE (an update produced a non-physical state; the
 * state of the last good iteration is kept), LSKUM_ERR_DIVERGED,
 * LSKUM_ERR_ARG, LSKUM_ERR_CUDA.
 */
lskum_status lskum_run(lskum_ctx *ctx, int32_t max_iters, double target_drop, int32_t *iters_done);

/* The two halves of lskum_run.  lskum_enqueue validates, then enqueues
 * max_iters iterations (one CUDA graph launch each) on the context's stream
 * and returns at once; lskum_wait blocks until they finish and reports the
 * status and the iterations run exactly as lskum_run does.  Between the two,
 * every other call on the context except lskum_stream returns LSKUM_ERR_ARG. */
lskum_status lskum_enqueue(lskum_ctx *ctx, int32_t max_iters, double target_drop);
lskum_status lskum_wait(lskum_ctx *ctx, int32_t *iters_done);

/* The context's internal cudaStream_t (work is enqueued there; the caller's
 * stream given at create is ordered before and after each call). */
void *lskum_stream(lskum_ctx *ctx);

/* Primitive state, f64[N] each, caller order. */
lskum_status lskum_get_state(lskum_ctx *ctx, double *rho, double *u, double *v, double *p);

/* One field (LSKUM_FIELD_*), caller order, into a caller buffer of N*4 (N for D) doubles. */
lskum_status lskum_get_field(lskum_ctx *ctx, int32_t field, double *out);

/* Density-residual norms of every iteration since the last set_state/create
 * (absolute, not divided by norm_1; case 0 of a batch).  Copies min(cap, count) entries; *n gets
 * the count. */
lskum_status lskum_get_residuals(lskum_ctx *ctx, double *hist, int32_t cap, int32_t *n);

/* Lift and drag coefficients of the current state (wall pressure integrated
 * over the wall polygon, wall points taken in caller index order). */
lskum_status lskum_get_forces(lskum_ctx *ctx, double *cl, double *cd);

/* The colouring and sweep order: colour i32[N] (1-based, caller order),
 * order i32[N] (caller index at each sweep position, as opts.ordering
 * defines it), n_colours. Any may be NULL. */
lskum_status lskum_get_order(lskum_ctx *ctx, int32_t *colour, int32_t *order, int32_t *n_colours);

/* Measure: run `reps` iterations with each phase launched directly (not as a
 * graph) between CUDA events on the context's stream; ms[6] receives the mean
 * device time per iteration of the phases 0 q-derivatives (all K+1 passes),
 * 1 residual + diagonal, 2 norm, 3 forward sweep (all levels), 4 backward
 * sweep, 5 update.  The iterations are real: the state advances by reps
 * iterations and the history grows.  Errors as lskum_run. */
lskum_status lskum_time_phases(lskum_ctx *ctx, int32_t reps, double *ms);

/* Autotune the launch shape (no counterpart in the paper; the kernels'
 * results do not depend on it beyond the order of floating-point sums): for
 * every threads-per-point count {1,2,4,8} of the q-derivative and residual
 * kernels and lanes-per-point count {2,4,8} of the sweep kernels, plus the
 * packed sweep form (sweep_lanes = 32: each point forms the axis Jacobian
 * products of its new increment once and interior points gather their
 * neighbours' products, four lanes per interior point; wall points, and
 * outer points under the kinetic far field, form their products per slot in
 * their own frame, one lane per list slot with whole points packed into
 * warps; available when no point has more than 32 lower or upper
 * neighbours), re-capture
 * the iteration graphs, run one warm-up iteration and time `trial_iters`
 * iterations between CUDA events on the context's stream; keep the fastest
 * shape.  The state, the per-case counters, stop flags and histories are
 * saved before and restored after every trial, so the caller sees the
 * context as before, only faster.  Outputs (each may be NULL): the chosen
 * threads per point, lanes per point and its mean device time per iteration
 * in ms.  Errors as lskum_run (the launch shape is then left unchanged). */
lskum_status lskum_autotune(lskum_ctx *ctx, int32_t trial_iters, int32_t *tpp, int32_t *sweep_lanes,
                            double *ms_per_iter);

/* Set the launch shape directly (e.g. one found by lskum_autotune for the
 * same cloud earlier): tpp in {1, 2, 4, 8} threads per point of the
 * q-derivative and residual kernels, sweep_lanes in {2, 4, 8} lanes per point
 * of the sweep kernels or 32 for the packed form.  The iteration graphs are
 * re-captured.  Errors: LSKUM_ERR_ARG (other values, the packed form where
 * it is not available, or a run not waited for), LSKUM_ERR_CUDA. */
lskum_status lskum_set_launch_shape(lskum_ctx *ctx, int32_t tpp, int32_t sweep_lanes);

/* Number of points, of colours and of kernel launches one iteration makes. */
lskum_status lskum_get_info(lskum_ctx *ctx, int32_t *n_points, int32_t *n_colours, int32_t *launches_per_iter);

/*
 * Density-residual norm without any device allocation (no counterpart in the
 * paper: a service for callers that cannot allocate device memory, e.g. hosts
 * whose device memory all belongs to their own pool allocator, loops that must
 * not take the synchronisation an allocation or free can cause, or deployments
 * that forbid runtime allocation).
 *   r_rho_dev  device pointer to n doubles (density residuals; the order does
 *              not matter; zeros may be included)
 *   n          0 <= n <= 134,217,728 (8192 partial sums x 256 threads x 64
 *              elements per thread); larger n returns LSKUM_ERR_ARG
 *   norm_dev   device pointer to one double: receives sqrt(sum r^2), the
 *              quantity lskum_get_residuals reports for the solver's own R
 *   cuda_stream  stream of the current device (NULL = legacy default); the
 *              result is ready when that stream reaches it
 * The scratch is a fixed 64 KiB device array inside the library, held by every
 * GPU that loads it until the process exits; no cudaMalloc/cudaFree or other
 * allocating call is made.  The first call on each device performs a one-time
 * set-up (it looks up that array's device address with that device current),
 * so make that first call before any stream capture.  The address is cached
 * per device number for the life of the process: after cudaDeviceReset (or
 * any other teardown of the device's primary context) the library's module
 * may load elsewhere, so do not call this entry point again in that process
 * (a failed launch drops the cached address, the next call looks it up
 * again).  All calls share the array: calls that overlap on the GPU race and
 * must be serialised by the caller.  Errors: LSKUM_ERR_ARG (NULL pointer, n out of range),
 * LSKUM_ERR_CUDA (set-up or launch failed).
 */
lskum_status lskum_density_norm_noalloc(const double *r_rho_dev, int32_t n, double *norm_dev, void *cuda_stream);

/*
 * Self-test of the kernels' integer-pipe FP64 arithmetic (no counterpart in
 * the paper: GB300-specific implementation of the method's operations).  On
 * the current device, for k < n, out[k] =
 *   op 0: a[k] * b[k] by the integer multiply the residual and the update
 *         use (correctly rounded, the FP64 multiply's bits);
 *   op 1: exp(a[k]) by the fixed-point exp behind exp(-S^2) in the split
 *         fluxes (Eq. 11-13) and rho in the inverse of Eq. 14 (Tang's
 *         table-driven method);
 *   op 2: erfcx(min(|a[k]|, 9))/2 by the fixed-point Horner evaluation
 *         behind A = (1 +- erf S)/2 of Eq. 11-13;
 *   op 3: a[k] * b[k] by the FP64 unit.
 * a, b, out: host arrays of n doubles (b may be NULL for ops 1 and 2); the
 * call allocates, copies and synchronises (a test and diagnostics service,
 * not for a hot path).  Errors: LSKUM_ERR_ARG (op not 0-3, n < 0, NULL
 * array), LSKUM_ERR_CUDA.
 */
lskum_status lskum_selftest_fpint(int32_t op, const double *a, const double *b, double *out, int32_t n);

/* Message of the last failure of ctx (or of the last failed create when ctx
 * is NULL); never NULL; valid until the next call on the same context. */
const char *lskum_last_error(const lskum_ctx *ctx);

/* Free everything; NULL is allowed. */
void lskum_destroy(lskum_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LSKUM_H */
