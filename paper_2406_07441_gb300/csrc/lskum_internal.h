// Device data layout and the launch interface between the host orchestration
// (lskum_host.cpp) and the kernels (lskum_kernels.cu).
//
// Layout in HBM (all in the internal order: points sorted by colour, then by
// type wall < interior < outer, then by caller index):
//  - per-point fields are structure-of-arrays with a row stride `ld`
//    (N rounded up to a multiple of 32): field f of point k at a[f * ld + k];
//  - neighbour lists are sliced ELLPACK: slice s holds points 32s..32s+31,
//    neighbour slot j of point k sits at slice_off[k / 32] + 32 j + k % 32, so
//    the 32 threads of a warp reading slot j of consecutive points touch one
//    contiguous 128-byte (i32) or 256-byte (f64) span.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lskum {

constexpr int kInterior = 0;
constexpr int kWall = 1;
constexpr int kOuter = 2;

// Device-resident control block: lets many iterations be enqueued (CUDA
// graph launches) without host synchronisation; every kernel of an
// iteration returns at once when the run has stopped.  A context holds one
// or several independent cases (a batch: the disjoint union of their
// clouds); each case has its own residual history and stopping state.
// kReachedTarget and kFailedNow finish their iteration (the sweeps and the
// update run; kFailedNow's update is undone by k_repair) and become
// kStopped / kFailed at the next k_begin.  Stopped and failed cases are
// frozen: their points keep their state while the batch's other cases run.
enum CaseState { kRunning = 0, kReachedTarget = 1, kStopped = 2, kFailedNow = 3, kFailed = 4 };

struct Ctrl {
    int32_t stop;        // 1: every case stopped or a failure: skip all further work
    int32_t error;       // lskum_status of a device-detected failure (0 = none)
    int32_t bad_point;   // smallest internal index of a non-physical update
    int32_t it;          // iterations started since the last reset (k_begin counts)
    int32_t it_start;    // it when the current run was enqueued
    int32_t hist_cap;    // capacity of each case's history
    int32_t n_cases;
    double target;       // drop target of the current run (<= 0: none)
    int32_t *case_state; // [n_cases] CaseState; kReachedTarget finishes the
                         // iteration, the next k_begin makes it kStopped
    int32_t *case_it;    // [n_cases] norms recorded
    double *case_hist0;  // [n_cases] first norm (drop reference); <= 0 = not set
    double *hist;        // [n_cases][hist_cap] residual-norm histories (density)
    double *hist4;       // [n_cases][hist_cap][4] norms of the four residual components
    int32_t *case_err;   // [n_cases] lskum_status of a failed case of a batch (0 = none)
    int32_t *case_bad;   // [n_cases] smallest internal index of its non-physical update
};

// Per-point geometry rows (fields of `geo`, stride ld).
enum GeoField {
    G_E1X, G_E1Y, G_E2X, G_E2Y,          // frame: (1,0),(0,1), or (t, n) at wall and kinetic outer points
    G_LS1_0, G_LS1_1, G_LS1_2, G_LS1_3,  // LS_s(1) of the four split sub-stencils (kinetic
                                         // outer points: LS_3(1) = -LS_2(1), the ghosts)
    G_ABS_0, G_ABS_1, G_ABS_2, G_ABS_3,  // sum_i |w_i| of each split sub-stencil
    G_DMIN,                              // min_i |r_i - r_0|
    G_SXX, G_SXY, G_SYX, G_SYY,          // sums over the stencil of wgx dx, wgx dy, wgy dx, wgy dy
    G_NFIELDS
};

// Per-point primal quantities of the current state used by the sweeps'
// Jacobian products: array of structures, point k's record at
// prim[k * kPrimStride + field], so that one neighbour's record is two
// cache lines instead of one line per field.
enum PrimField {
    P_RHO, P_IRHO, P_U, P_V, P_P, P_BETA, P_SB, P_ISB, P_I2P, P_Q2, P_E1, P_E2,
    P_BSX, P_APX, P_AMX, P_EKX, P_BX,  // direction (1,0): 2 B S, A+, A-, exp(-S^2)/sqrt(pi), B
    P_BSY, P_APY, P_AMY, P_EKY, P_BY,  // direction (0,1)
    P_UE1, P_VE1,                      // u e1, v e1
    P_NFIELDS
};
constexpr int kPrimStride = 24;

// Packed sweep form: lanes per interior point (each takes every kLanesPerPoint-th
// slot of the point's list and forms one of its four axis products), and so
// interior points per warp.
constexpr int kLanesPerPoint = 4;
constexpr int kPointsPerWarp = 32 / kLanesPerPoint;
static_assert(P_NFIELDS <= kPrimStride, "prim record too small");

struct StateSet {
    double *U;     // [4][ld] conserved variables
    double *q;     // [4][ld] q-variables
    double *prim;  // [ld][kPrimStride]
    float *primf;  // [ld][kPrimStride] FP32 copy (mixed precision only, else null)
};

struct Dev {
    int32_t n, ld, n_slices;
    // cloud
    const uint8_t *flag;     // [n]
    const double *wnx, *wny; // [n] wall normals (and outer normals under the kinetic far field)
    const double *geo;       // [G_NFIELDS][ld]
    // sliced ELL neighbour slots
    const int32_t *slice_off; // [n_slices + 1]
    const int32_t *deg;       // [n]
    const int32_t *nbr;       // neighbour (internal index)
    const uint8_t *memb;      // bits 0/1: e1 sub-stencil +/-, bits 2/3: e2 sub-stencil +/-
    const double *nhx, *nhy;  // (x_i - x_0)/2, (y_i - y_0)/2
    const double *w1, *w2;    // LS weight of the slot in its e1 / e2 split sub-stencil (0 if none)
    const double *wgx, *wgy;  // full-stencil LS weights of d/dx and d/dy (Eq. 10, 16)
    const double *gxx, *gxy, *gyx, *gyy;  // wgx dx, wgx dy, wgy dx, wgy dy (inner iterations)
    // iteration buffers
    StateSet set[2];
    double *gq[2];           // double-buffered q-derivatives, [ld][8]: point k's
                             // (dq/dx 0..3, dq/dy 0..3) at 8k, one 64-byte record
    double *g1x, *g1y;       // first-order LS derivatives (the fixed part of Eq. 16)
    double *R;               // [4][ld]
    double *D;               // [ld]
    double *iD;              // [ld] 1/D (explicit scheme: the local time step)
    double *dUs, *dU;        // [ld][4] (array of structures: one 32-byte gather per neighbour)
    // LU-SGS slot lists (CSR over the internal index): the slots of each point
    // whose neighbour comes earlier (lo) or later (up) in the sweep order,
    // outer neighbours and slots in no split sub-stencil left out
    const int32_t *lo_off, *lo_nbr, *up_off, *up_nbr;
    const uint8_t *lo_mb, *up_mb;
    const double *lo_w1, *lo_w2, *up_w1, *up_w2;
    // mixed precision (precision = 1): FP32 increments ([ld][4]) and weights;
    // null in FP64 mode
    float *dUsf, *dUf;
    const float *lo_w1f, *lo_w2f, *up_w1f, *up_w2f;
    // per colour level, its swept points ordered by decreasing list length
    // (forward: lower list, backward: upper list), so a warp's groups share a
    // trip count
    const int32_t *sw_fwd, *sw_bwd;
    // packed sweep form, [0] forward (lower lists), [1] backward (upper
    // lists), for the points in a (t, n) frame: warp w's 32 lanes hold slots
    // 32w .. 32w+31, each with the sweep position of its point (-1: padding),
    // neighbour, membership and weights; a point's slots are consecutive
    // lanes of one warp (null when a list is longer than 32)
    const int32_t *pk_pt[2], *pk_nbr[2];
    const uint8_t *pk_mb[2];
    const uint8_t *pk_steps[2];  // per warp: steps of its segmented sum, ceil(log2(longest list))
    const double *pk_w1[2], *pk_w2[2];
    const float *pk_w1f[2], *pk_w2f[2];
    // and for the interior points: kLanesPerPoint lanes per point, in groups
    // of kPointsPerWarp points (by decreasing list length): point p of group g
    // is lp_k[kPointsPerWarp g + p] (-1: none), with lp_len[...] slots, slot j
    // at lp_goff[g] + 32 (j / kLanesPerPoint) + kLanesPerPoint p + j % kLanesPerPoint
    // (lane kLanesPerPoint p + s takes the slots j = s (mod kLanesPerPoint))
    const int32_t *lp_k[2], *lp_len[2], *lp_goff[2], *lp_nbr[2];
    const uint8_t *lp_mb[2];
    const double *lp_w1[2], *lp_w2[2];
    const float *lp_w1f[2], *lp_w2f[2];
    // packed form: per point, the axis split-flux Jacobian products of its
    // latest increment, [ld][4 products: x+, x-, y+, y-][4]: written when the
    // point's increment is formed, gathered by the later levels' interior
    // points (FP64, or FP32 for the mixed-precision sweeps; the other is null)
    double *jc;
    float *jcf;
    // packed form, exact Jacobian products of the points in a (t, n) frame:
    // the Jacobians of the split fluxes depend only on the state of the
    // iteration, not on the increments, so they are formed for the whole
    // level set before the forward sweep (k_framed_jac) and the sweeps'
    // framed chains reduce to matrix-vector products.  pk_jm[dir]: per packed
    // slot lane, M = w1 dG_e1/dU + w2 dG_e2/dU at the neighbour's state, 16
    // values (row c, column j at 4 c + j); fj: per framed point f, its four
    // axis Jacobians (x+, x-, y+, y-) at its own state, [nf][4][16]; fidx[k]
    // = f or -1.  FP64, or FP32 for the mixed-precision sweeps.
    double *pk_jm[2], *fj;
    float *pk_jmf[2], *fjf;
    const int32_t *fidx, *fpt;  // fpt[f] = internal index of framed point f
    int32_t pk_lanes[2], nf;
    // per-case residual norm: stage 1 sums R_rho^2 over blocks of up to 256
    // points of one case (caller order), stage 2 adds each case's blocks
    double *blk;             // [n_blk][4] partial sums of the four components
    const int32_t *blk_pos;  // [n_blk + 1] caller-order start of each block
    const int32_t *blk_case; // [n_blk] case of each block
    const int32_t *case_blk; // [n_cases + 1] first block of each case
    const int32_t *inv;      // [n] caller index -> internal index
    const int32_t *case_of;  // [ld] internal index -> case
    int32_t n_blk, n_cases;
    Ctrl *ctrl;
    const int32_t *case_state;  // = ctrl->case_state (read per point)
    // options
    double cfl, ramp, u_inf[4];
    int32_t K, jvp;
    int32_t first_order;  // iterations n <= first_order use q~ = q
    int32_t precision;    // 0 FP64; 1 FP32 sweeps, compensated FP64 residual sums
    int32_t scheme;       // 0 implicit LU-SGS; 1 explicit (forward Euler, no sweeps)
    int32_t lusgs;        // 0 Anandhanarayanan's diagonal; 1 the revised form of Manish et al.
    int32_t farfield;     // 0 outer points frozen at the free stream; 1 the kinetic far field
    const double *case_uinf;  // [n_cases][4] free-stream conserved state of each case
};

// Kernel launch wrappers (lskum_kernels.cu).  `cur` is the state set read by
// this iteration; the update writes set 1 - cur.
struct Launch {
    int tpp;          // threads per point of the gradient and residual kernels (1, 2, 4, 8)
    int res_block;    // threads per block of the residual kernel
    int sweep_lanes;  // lanes per point of the sweep kernels (2, 4, 8), or 32: the packed form
    const int32_t *pk_lw[2];  // packed form: host arrays [n_levels + 1], first framed-point warp of each level
    const int32_t *lp_lg[2];  // packed form: host arrays [n_levels + 1], first interior group of each level
    // optional side branch of a captured iteration: the framed points'
    // Jacobians (k_framed_jac) run on `side` between the `fork` after k_begin
    // and the `join` before the forward sweep, beside the q-derivatives and
    // the residual; null: inline, before the forward sweep
    cudaStream_t side;
    cudaEvent_t fork, join;
};

cudaError_t launch_iteration(const Dev &d, const Launch &L, int cur, int n_levels, const int32_t *lvl_beg,
                             const int32_t *lvl_act_end, const int32_t *lvl_end, cudaStream_t s,
                             int *launches);
// One phase of an iteration (0 q-derivatives, 1 residual, 2 norm, 3 forward
// sweep, 4 backward sweep, 5 update), launched directly on s.
cudaError_t launch_phase(const Dev &d, const Launch &L, int cur, int phase, int n_levels, const int32_t *lvl_beg,
                         const int32_t *lvl_act_end, const int32_t *lvl_end, cudaStream_t s);
// Derive q and the per-point records of a new state in set cur (with the
// wall projection of the state when project).
cudaError_t launch_init_state(const Dev &d, int cur, bool project, cudaStream_t s);
// Fill the global copy of the function tables the sweeps read (idempotent).
cudaError_t launch_init_math(cudaStream_t s);
// The integer-pipe FP64 arithmetic on n device values (lskum_selftest_fpint).
cudaError_t launch_selftest_fpint(int op, const double *a, const double *b, double *out, int n, cudaStream_t s);
cudaError_t launch_reset_ctrl(Ctrl *c, cudaStream_t s);
// Prepare the control block for a run, on the device: flags cleared, drop
// target set, it_start = it, stopped cases running again (failed ones stay).
cudaError_t launch_prep_run(Ctrl *c, double target, cudaStream_t s);
// Device-side reordering between the internal and the caller's point order
// (source layout [c][ld] for stride 0, else point k's values at stride * k).
cudaError_t launch_to_caller(const double *src, const float *srcf, int comps, int stride, int ld, int n,
                             const int32_t *inv, double *out, cudaStream_t s);
cudaError_t launch_from_caller(const double *in, int ld, int n, const int32_t *inv, double *U, cudaStream_t s);

}  // namespace lskum
