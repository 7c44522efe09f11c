// sm_103a kernels of one implicit q-LSKUM pseudo-time iteration (Alg. 1):
//   k_grad      least-squares q-derivatives, first order + K inner iterations (Eq. 10, 16)
//   k_residual  defect-corrected kinetic split-flux residual (Eq. 11-15), local time
//               step and scalar LU-SGS diagonal (Eq. 26, 33-34), density-norm partials
//   k_norm_*    per-case residual norms, histories and stopping tests
//   k_sweep     one colour level of the forward or backward LU-SGS sweep (Eq. 27) with
//               exact (forward-mode AD) or increment (Eq. 28) Jacobian-vector products;
//               k_sweep_packed: the same level with each point's axis products formed
//               once and gathered by its neighbours
//   k_update    U += dU, wall projection, q-variables and the per-point primal
//               quantities the next iteration's sweeps need
//
// GB300 has 62x more FP32 than FP64 throughput (1.2 FP64 TFLOP/s measured), so
// the FP64 path is bound by FP64 instruction issue, not HBM.  The kernels are
// shaped to issue as few FP64 instructions as possible: every geometric
// quantity (LS weights, frames, stencil membership) is precomputed per
// neighbour slot; the inverse of Eq. 14 uses beta^(-5/2) instead of a log;
// the sweeps' Jacobian products reuse erf/exp of each point's own state,
// computed once per iteration by k_update, so an exact product has no
// transcendental call at all, and a neighbour's product along an axis is
// formed once and gathered; exp and A = (1 + s erf S)/2 are the kernels' own
// (lskum_fastmath.cuh), which share exp(-S^2) and keep index work off the
// FP64 pipe, as are signs and multiplications by 2 and 1/2 (integer steps).
// exp and erfcx run in fixed point on the integer pipes (lskum_fixmath.cuh),
// and the multiplications of the split fluxes and of the update on the
// integer pipes too (mul_i, lskum_intmul.cuh: correctly rounded, the same
// bits), which leaves the FP64 unit the fused multiply-adds, the additions
// and the multiplications on the residual's critical path (q to primitives);
// the sweeps, bound by the latency of their dependent chains rather than by
// FP64 issue, keep the FP64 multiply.
#include "lskum_internal.h"

#include <cstdint>

#include "lskum_fastmath.cuh"

namespace lskum {

namespace {

constexpr double kGm1 = 0.4;                              // gamma - 1 (gamma = 1.4)
constexpr double kInv2SqrtPi = 0.28209479177387814347;    // 1 / (2 sqrt(pi))
constexpr double kInvSqrtPi = 0.56418958354775628695;     // 1 / sqrt(pi)
constexpr unsigned kFull = 0xffffffffu;

// Every kernel returns at once after a stop or a failure.  When a case
// reaches its drop target, k_norm marks it kReachedTarget, so the sweeps and
// the update of that iteration still run; the next k_begin makes it
// kStopped, after which its points are left alone (a batch keeps iterating
// its other cases) and, once every case has stopped, sets stop.  In a batch
// a failure (non-finite norm, non-physical update) fails only its own case,
// which keeps its last good state; a single case fails the context.
__device__ __forceinline__ bool halted(const Ctrl *c)
{
    const volatile Ctrl *v = c;
    return (v->stop | v->error) != 0;
}

// Is point k's case stopped?  (Only batches have cases that stop while
// others run; a single case stops the whole context.)
__device__ __forceinline__ bool frozen_state(int32_t st)
{
    return st == kStopped || st == kFailed;
}

__device__ __forceinline__ bool frozen(const Dev &d, int k)
{
    return d.n_cases > 1 && frozen_state(((const volatile int32_t *)d.case_state)[d.case_of[k]]);
}

// One copy of the function tables in global memory, for kernels that need
// them only at a few points (the sweeps: wall and outer points); kernels that
// evaluate them at every point stage them in shared memory instead.
__device__ MathTables g_math;

__global__ void k_init_math()
{
    load_math_tables(g_math);
}

// x with its sign flipped unless pos: an integer XOR of the sign bit, so a
// selected sign costs no FP64 (or FP32) instruction.
__device__ __forceinline__ double signed_by(double x, bool pos)
{
    return __hiloint2double(__double2hiint(x) ^ (pos ? 0 : (int)0x80000000), __double2loint(x));
}
__device__ __forceinline__ float signed_by(float x, bool pos)
{
    return __int_as_float(__float_as_int(x) ^ (pos ? 0 : (int)0x80000000));
}

// x / 2 and 2 x as a step of the exponent field on the integer pipe: the same
// bits as the FP64 multiplication whenever both x and the result are normal
// (a multiplication by a power of two is exact there).  Zeros and
// non-finite values come back unchanged, which is again the exact result;
// only magnitudes below 2^-1021 (halving: the result would be subnormal),
// subnormal inputs (doubling: returned as they are) and magnitudes above
// 2^1023 (doubling) differ, far outside what any quantity of the solver
// reaches.  FP32 keeps
// its multiplication (its pipe is not the bottleneck).
__device__ __forceinline__ double half_of(double x)
{
    const int hi = __double2hiint(x);
    const unsigned ex = ((unsigned)hi >> 20) & 0x7ffu;
    return __hiloint2double(ex - 2u < 0x7fdu ? hi - 0x00100000 : hi, __double2loint(x));
}
__device__ __forceinline__ double twice(double x)
{
    const int hi = __double2hiint(x);
    const unsigned ex = ((unsigned)hi >> 20) & 0x7ffu;
    return __hiloint2double(ex - 1u < 0x7fdu ? hi + 0x00100000 : hi, __double2loint(x));
}
__device__ __forceinline__ float half_of(float x) { return 0.5f * x; }
__device__ __forceinline__ float twice(float x) { return 2.0f * x; }

// Primitive state carried through the residual.
struct Prim {
    double rho, u, v, p, sb, isb, e1, e2;  // sb = sqrt(beta), isb = 1/sb,
                                           // e1 = 3.5 p + rho|u|^2/2, e2 = 3 p + rho|u|^2/2
    double bk;                             // 1 / (2 sqrt(pi beta)): B = exp(-S^2) bk
};

// Inverse of Eq. 14: beta = -q4/2, u = q2/(2 beta), v = q3/(2 beta),
// rho = exp(q1 + beta |u|^2) beta^(-1/(gamma-1)) with 1/(gamma-1) = 5/2,
// p = rho/(2 beta).  One reciprocal square root and one exp.  Its
// multiplications stay on the FP64 unit: every split flux of the slot waits
// for these primitives, and on that critical path the integer multiply's
// longer dependency chain costs more than the FP64 issue it would free
// (measured: the residual is 8% faster this way than with the integer
// multiply here, and 20% slower with every multiplication of the split flux
// on the FP64 unit too).
__device__ __forceinline__ Prim q_to_prim(const MathTables &T, const double q[4])
{
    Prim P;
    const double beta = signed_by(half_of(q[3]), false);  // -q4/2, the sign by XOR
    P.isb = rsqrt(beta);
    const double ib = P.isb * P.isb;   // 1/beta
    const double r = ib * ib * P.isb;  // beta^(-5/2)
    const double i2b = half_of(ib);    // 1/(2 beta)
    P.sb = beta * P.isb;
    P.u = q[1] * i2b;
    P.v = q[2] * i2b;
    const double q2 = fma(P.u, P.u, P.v * P.v);
    P.rho = exp_t(T, fma(beta, q2, q[0])) * r;
    P.p = P.rho * i2b;
    const double k = half_of(P.rho * q2);
    P.e1 = fma(3.5, P.p, k);
    P.e2 = fma(3.0, P.p, k);
    P.bk = kInv2SqrtPi * P.isb;
    return P;
}

// Kinetic split flux G_d^sg (half-range moments of the Maxwellian; sg = +1
// if pos, else -1, applied by negation) in unit direction d: (dx, dy) in a
// (t, n) frame (framed), else the x axis (xdir) or the y axis, where the
// axis components are selected on the integer pipe instead of multiplied by
// 0 and 1.  One body for every frame and axis keeps the residual's loop
// small enough for the instruction cache.
__device__ __forceinline__ void split_flux(const MathTables &T, const Prim &P, bool framed, bool xdir, double dx,
                                          double dy, bool pos, double G[4])
{
    const double ua = xdir ? P.u : P.v, uo = xdir ? P.v : P.u;  // along and across the axis
    const double ud = framed ? fma(P.u, dx, mul_i(P.v, dy)) : ua;
    const double S = ud * P.sb;  // FP64 unit: heads the exp/erfcx path (measured faster)
    double A, eS;
    split_A(T, S, pos, A, eS);
    const double B = mul_i(eS, P.bk);
    const double sB = signed_by(B, pos);
    const double M1 = fma(ud, A, sB);
    const double rm = mul_i(P.rho, M1);
    const double pA = mul_i(P.p, A);
    G[0] = rm;
    if (framed) {
        G[1] = fma(rm, P.u, mul_i(pA, dx));
        G[2] = fma(rm, P.v, mul_i(pA, dy));
    } else {
        const double ga = fma(rm, ua, pA), go = mul_i(rm, uo);
        G[1] = xdir ? ga : go;
        G[2] = xdir ? go : ga;
    }
    G[3] = fma(mul_i(ud, P.e1), A, mul_i(P.e2, sB));
}

// Primal quantities of a conserved state for the Jacobian products (FP64,
// or FP32 for the mixed-precision sweeps).
template <typename T>
struct PrimT {
    T rho, irho, u, v, p, beta, sb, isb, i2p, q2, e1, e2;
};
using PrimU = PrimT<double>;

__device__ __forceinline__ PrimU prim_from_cons(const double U[4])
{
    PrimU P;
    P.rho = U[0];
    P.irho = 1.0 / U[0];
    P.u = mul_i(U[1], P.irho);
    P.v = mul_i(U[2], P.irho);
    P.q2 = fma(P.u, P.u, mul_i(P.v, P.v));
    const double hr = half_of(P.rho);
    P.p = mul_i(kGm1, fma(-hr, P.q2, U[3]));
    const double k = mul_i(hr, P.q2);  // rho |u|^2 / 2
    P.i2p = 0.5 / P.p;
    P.beta = mul_i(P.rho, P.i2p);
    P.sb = sqrt(P.beta);
    P.isb = 1.0 / P.sb;
    P.e1 = fma(3.5, P.p, k);
    P.e2 = fma(3.0, P.p, k);
    return P;
}

template <typename T>
__device__ __forceinline__ PrimT<T> load_prim(const T *__restrict__ pr, int i)
{
    const T *r = pr + (size_t)i * kPrimStride;
    PrimT<T> P;
    P.rho = r[P_RHO];
    P.irho = r[P_IRHO];
    P.u = r[P_U];
    P.v = r[P_V];
    P.p = r[P_P];
    P.beta = r[P_BETA];
    P.sb = r[P_SB];
    P.isb = r[P_ISB];
    P.i2p = r[P_I2P];
    P.q2 = r[P_Q2];
    P.e1 = r[P_E1];
    P.e2 = r[P_E2];
    return P;
}

// Exact product A_d^sg(U) dl by forward-mode differentiation of
// U -> (rho, u, v, p) -> (beta, S, A, B) -> G_d^sg.  S, A = (1 + sg erf S)/2,
// exp(-S^2) and B of the state are inputs (precomputed per point for d = x, y).
// The direction-independent part of the tangent: derivatives of the
// primitive quantities along dl (shared by a neighbour's x and y split
// sub-stencils, computed once per neighbour).
template <typename T>
struct JvpBase {
    T drho, du, dv, dk, dp, dsb;
    T dsbi, de1, de2;  // dsb / sqrt(beta), d(3.5 p + k), d(3 p + k)
};

template <typename T>
__device__ __forceinline__ JvpBase<T> jvp_base(const PrimT<T> &P, const T dl[4])
{
    JvpBase<T> b;
    b.drho = dl[0];
    b.du = (dl[1] - P.u * b.drho) * P.irho;
    b.dv = (dl[2] - P.v * b.drho) * P.irho;
    const T dq2 = twice(P.u * b.du + P.v * b.dv);
    b.dk = half_of(b.drho * P.q2 + P.rho * dq2);  // d(rho |u|^2 / 2)
    b.dp = T(kGm1) * (dl[3] - b.dk);
    const T dbeta = (b.drho - twice(P.beta) * b.dp) * P.i2p;
    b.dsb = half_of(dbeta) * P.isb;
    b.dsbi = b.dsb * P.isb;
    b.de1 = T(3.5) * b.dp + b.dk;
    b.de2 = T(3.0) * b.dp + b.dk;
    return b;
}

// Tangent of the split flux in direction (dx, dy) with sign sg, given the
// primal S, A, exp(-S^2), B of that direction.
template <typename T>
__device__ __forceinline__ void jvp_dir(const PrimT<T> &P, const JvpBase<T> &b, T dx, T dy, T sg, T S, T A, T eS,
                                        T B, T out[4])
{
    const T ud = P.u * dx + P.v * dy;
    const T dud = b.du * dx + b.dv * dy;
    const T dS = dud * P.sb + ud * b.dsb;
    const T dA = sg * eS * dS * T(kInvSqrtPi);
    const T dB = -B * (T(2.0) * S * dS + b.dsbi);
    const T M1 = ud * A + sg * B;
    const T dM1 = dud * A + ud * dA + sg * dB;
    const T de1 = b.de1;
    const T de2 = b.de2;
    const T drm = b.drho * M1 + P.rho * dM1;  // d(rho M1)
    const T rm = P.rho * M1;
    out[0] = drm;
    out[1] = drm * P.u + rm * b.du + (b.dp * A + P.p * dA) * dx;
    out[2] = drm * P.v + rm * b.dv + (b.dp * A + P.p * dA) * dy;
    out[3] = (dud * P.e1 + ud * de1) * A + ud * P.e1 * dA + sg * (de2 * B + P.e2 * dB);
}

// The same product along an axis (DIR 0: d = (1,0), DIR 1: (0,1)) from the
// point's record: A, exp(-S^2)/sqrt(pi) (ek), B, 2 B S and u_d e1 precomputed
// per point, the direction-free tangents in the base, signs applied by
// negation (no multiplication by 0, 1 or +-1 is left to the FP64 pipe).
template <int DIR, typename T>
__device__ __forceinline__ void jvp_axis(const PrimT<T> &P, const JvpBase<T> &b, bool pos, T A, T ek, T B, T B2S,
                                         T ude1, T out[4])
{
    const T ud = DIR == 0 ? P.u : P.v;
    const T dud = DIR == 0 ? b.du : b.dv;
    const T dS = fma(dud, P.sb, ud * b.dsb);
    const T dA = signed_by(ek * dS, pos);
    const T sB = signed_by(B, pos);
    const T sdB = signed_by(fma(B2S, dS, B * b.dsbi), !pos);  // sg times the tangent of B
    const T M1 = fma(ud, A, sB);
    const T dM1 = fma(dud, A, fma(ud, dA, sdB));
    const T rm = P.rho * M1;
    const T drm = fma(b.drho, M1, P.rho * dM1);
    const T pA = fma(b.dp, A, P.p * dA);  // tangent of p A
    out[0] = drm;
    if (DIR == 0) {
        out[1] = fma(drm, P.u, fma(rm, b.du, pA));
        out[2] = fma(drm, P.v, rm * b.dv);
    } else {
        out[1] = fma(drm, P.u, rm * b.du);
        out[2] = fma(drm, P.v, fma(rm, b.dv, pA));
    }
    const T t1 = fma(dud, P.e1, ud * b.de1);
    const T t3 = fma(b.de2, sB, P.e2 * sdB);
    out[3] = fma(t1, A, fma(ude1, dA, t3));  // ude1 = u_d e1, from the record
}

// The same product with the axis chosen at run time (xdir: d = (1,0), else
// (0,1)) without a branch: the axis-dependent operands are selected on the
// integer pipe, so the lanes of a warp that form x- and y-products issue one
// FP64 sequence together.  Equal to jvp_axis<0 or 1> except that a pressure
// term of zero is added as +0 (an exactly zero product then has sign +).
template <typename T>
__device__ __forceinline__ void jvp_axis_sel(const PrimT<T> &P, const JvpBase<T> &b, bool xdir, bool pos, T A, T ek,
                                             T B, T B2S, T ude1, T out[4])
{
    const T ud = xdir ? P.u : P.v;
    const T dud = xdir ? b.du : b.dv;
    const T dS = fma(dud, P.sb, ud * b.dsb);
    const T dA = signed_by(ek * dS, pos);
    const T sB = signed_by(B, pos);
    const T sdB = signed_by(fma(B2S, dS, B * b.dsbi), !pos);
    const T M1 = fma(ud, A, sB);
    const T dM1 = fma(dud, A, fma(ud, dA, sdB));
    const T rm = P.rho * M1;
    const T drm = fma(b.drho, M1, P.rho * dM1);
    const T pA = fma(b.dp, A, P.p * dA);
    const T zero = T(0);
    out[0] = drm;
    out[1] = fma(drm, P.u, fma(rm, b.du, xdir ? pA : zero));
    out[2] = fma(drm, P.v, fma(rm, b.dv, xdir ? zero : pA));
    const T t1 = fma(dud, P.e1, ud * b.de1);
    const T t3 = fma(b.de2, sB, P.e2 * sdB);
    out[3] = fma(t1, A, fma(ude1, dA, t3));
}

// Unsplit Euler-flux Jacobian product A_d(U) dU in direction d = (dx, dy)
// (the tangent of G_d = (rho u_d, rho u u_d + p dx, rho v u_d + p dy,
// (E + p) u_d) along dU; the revised LU-SGS's S term).
__device__ __forceinline__ void euler_jvp(double rho, double u, double v, double p, const double dU[4], double dx,
                                          double dy, double out[4])
{
    const double irho = 1.0 / rho;
    const double ud = u * dx + v * dy;
    const double du = (dU[1] - u * dU[0]) * irho, dv = (dU[2] - v * dU[0]) * irho;
    const double dud = du * dx + dv * dy;
    const double dk = u * dU[1] + v * dU[2] - 0.5 * (u * u + v * v) * dU[0];  // d(rho |u|^2 / 2)
    const double dp = kGm1 * (dU[3] - dk);
    const double E = p / kGm1 + 0.5 * rho * (u * u + v * v);
    out[0] = dU[1] * dx + dU[2] * dy;
    out[1] = dU[1] * ud + rho * u * dud + dp * dx;
    out[2] = dU[2] * ud + rho * v * dud + dp * dy;
    out[3] = (dU[3] + dp) * ud + (E + p) * dud;
}

__device__ __forceinline__ void flux_cons(const MathTables &T, const double U[4], double dx, double dy, bool pos,
                                          double G[4])
{
    const PrimU P = prim_from_cons(U);
    const double ud = P.u * dx + P.v * dy;
    const double S = ud * P.sb;
    double A, eS;
    split_A(T, S, pos, A, eS);
    const double B = eS * kInv2SqrtPi * P.isb;
    const double sB = signed_by(B, pos);
    const double M1 = fma(ud, A, sB);
    const double rm = P.rho * M1;
    const double pA = P.p * A;
    G[0] = rm;
    G[1] = fma(rm, P.u, pA * dx);
    G[2] = fma(rm, P.v, pA * dy);
    G[3] = fma(ud * P.e1, A, P.e2 * sB);
}

template <int TPP, typename T>
__device__ __forceinline__ T group_sum(T v)
{
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// q-derivatives: first order (Eq. 10), then Jacobi inner iterations of Eq. 16
// ---------------------------------------------------------------------------
// An inner iteration's right-hand side sum_i w_i (Delta q_i - Delta r_i .
// (grad q_i - grad q_0)/2) splits into the first-order term g1 = sum_i w_i
// Delta q_i, fixed across iterations, and
//   sum_i (w_i dx_i) px_i + (w_i dy_i) py_i - px_0 sum_i w_i dx_i - py_0 sum_i w_i dy_i
// with per-slot products w dx, w dy precomputed: 4 FMAs per component and
// slot instead of 7 FP64 instructions.
// The q-derivatives live in 64-byte records ([ld][8]), so a neighbour's
// previous iterate is two 32-byte sectors instead of eight scattered ones.
template <int TPP, bool CORR>
__global__ void __launch_bounds__(256) k_grad(Dev d, const double *__restrict__ q, const double *__restrict__ pg,
                                              double *__restrict__ g)
{
    if (halted(d.ctrl)) return;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = gt / TPP, sub = gt % TPP;
    const bool active = k < d.n;
    const int kk = active ? k : d.n - 1;
    const int ld = d.ld;
    double q0[4], sx[4], sy[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        if (!CORR) q0[c] = q[c * ld + kk];
        sx[c] = 0.0;
        sy[c] = 0.0;
    }
    const int deg = d.deg[kk];
    const int base = d.slice_off[kk >> 5] + (kk & 31);
    for (int j = sub; j < deg; j += TPP) {
        const int e = base + 32 * j;
        const int i = d.nbr[e];
        if (!CORR) {
            const double wx = d.wgx[e], wy = d.wgy[e];
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const double dq = q[c * ld + i] - q0[c];
                sx[c] = fma(wx, dq, sx[c]);
                sy[c] = fma(wy, dq, sy[c]);
            }
        } else {
            const double axx = d.gxx[e], axy = d.gxy[e], ayx = d.gyx[e], ayy = d.gyy[e];
            const double2 *r = reinterpret_cast<const double2 *>(pg + 8 * (size_t)i);
            const double2 a01 = r[0], a23 = r[1], b01 = r[2], b23 = r[3];
            const double a[4] = {a01.x, a01.y, a23.x, a23.y}, b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
            for (int c = 0; c < 4; c++) {
                sx[c] = fma(axx, a[c], fma(axy, b[c], sx[c]));
                sy[c] = fma(ayx, a[c], fma(ayy, b[c], sy[c]));
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        sx[c] = group_sum<TPP>(sx[c]);
        sy[c] = group_sum<TPP>(sy[c]);
    }
    if (active && sub == 0) {
        if (!CORR) {
#pragma unroll
            for (int c = 0; c < 4; c++) {
                d.g1x[c * ld + k] = g[8 * (size_t)k + c] = sx[c];
                d.g1y[c * ld + k] = g[8 * (size_t)k + 4 + c] = sy[c];
            }
        } else {
            const double cxx = d.geo[G_SXX * ld + k], cxy = d.geo[G_SXY * ld + k];
            const double cyx = d.geo[G_SYX * ld + k], cyy = d.geo[G_SYY * ld + k];
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const double a0 = pg[8 * (size_t)k + c], b0 = pg[8 * (size_t)k + 4 + c];
                const double rx = sx[c] - fma(cxx, a0, cxy * b0);
                const double ry = sy[c] - fma(cyx, a0, cyy * b0);
                g[8 * (size_t)k + c] = fma(-0.5, rx, d.g1x[c * ld + k]);
                g[8 * (size_t)k + 4 + c] = fma(-0.5, ry, d.g1y[c * ld + k]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// flux residual, time step, diagonal, norm partials
// ---------------------------------------------------------------------------
// R += y with Kahan's compensated summation (W. Kahan, "Further remarks on
// reducing truncation errors", CACM 8(1), 1965): c carries the negated
// rounding error of the running sum into the next term.  The caller forms y
// as the terms of a group of four slots less c, the weighted flux
// differences of their split sub-stencils folded in by FMAs, so one
// compensated addition serves the group (a quarter of the per-slot
// additions' FP64 instructions; R changed by at most 6e-17 relative).  The
// final sum is R - c.
__device__ __forceinline__ void comp_add(double &R, double &c, double y)
{
    const double t = R + y;
    c = (t - R) - y;  // what the addition lost (negated)
    R = t;
}

// The sign of x with magnitude 0 (what 0 * x gives), on the integer pipe.
__device__ __forceinline__ double zero_like(double x)
{
    return __hiloint2double(__double2hiint(x) & (int)0x80000000, 0);
}

template <int TPP, bool COMP>
// Blocks of the residual kept resident per SM: 4 x 128 threads caps it at
// 128 registers without spills (5 spills and runs slower; with no cap the
// integer multiplies take it to 139 registers and 3 blocks).
#ifndef LSKUM_RES_MIN_BLOCKS
#define LSKUM_RES_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(128, LSKUM_RES_MIN_BLOCKS) k_residual(Dev d, StateSet st, const double *__restrict__ g)
{
    __shared__ MathTables T;
    if (halted(d.ctrl)) return;
    load_math_tables(T);
    __syncthreads();
    const int n1 = ((const volatile Ctrl *)d.ctrl)->it;  // this iteration, counted by k_begin
    const double cfl = (d.ramp > 0.0 && (double)n1 < d.ramp) ? d.cfl * ((double)n1 / d.ramp) : d.cfl;
    const bool second = n1 > d.first_order;  // first-order start: q~ = q
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = gt / TPP, sub = gt % TPP;
    const bool active = k < d.n;
    const int kk = active ? k : d.n - 1;
    const int ld = d.ld;
    const int fl = d.flag[kk];
    const bool work = active && (fl != kOuter || d.farfield == 1) && !frozen(d, kk);
    const bool framed = fl != kInterior;  // (t, n) frame: wall and kinetic outer points
    const double *__restrict__ q = st.q;
    double R[4] = {0.0, 0.0, 0.0, 0.0};
    double Rc[4] = {0.0, 0.0, 0.0, 0.0};  // compensation terms (COMP)
    const double e1x = d.geo[G_E1X * ld + kk], e1y = d.geo[G_E1Y * ld + kk];
    const double e2x = d.geo[G_E2X * ld + kk], e2y = d.geo[G_E2Y * ld + kk];
    if (work) {
        double q0[4], gx0[4], gy0[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            q0[c] = q[c * ld + kk];
            gx0[c] = g[8 * (size_t)kk + c];
            gy0[c] = g[8 * (size_t)kk + 4 + c];
        }
        const int deg = d.deg[kk];
        const int base = d.slice_off[kk >> 5] + (kk & 31);
        // (COMP) the terms of a group of four slots are summed by FMAs into y,
        // which starts as the negated carried error; each group then enters R
        // by one compensated addition, and a last partial group after the loop
        double y[4] = {0.0, 0.0, 0.0, 0.0};
        int ng = 0;  // (COMP) slots in the current group
        for (int j = sub; j < deg; j += TPP) {
            const int e = base + 32 * j;
            const int mb = d.memb[e];
            if (!mb) continue;
            const int i = d.nbr[e];
            const double hx = d.nhx[e], hy = d.nhy[e];  // half offsets
            double qi[4], q0t[4];
            const double2 *gr = reinterpret_cast<const double2 *>(g + 8 * (size_t)i);
            const double2 x01 = gr[0], x23 = gr[1], y01 = gr[2], y23 = gr[3];
            const double gxi[4] = {x01.x, x01.y, x23.x, x23.y}, gyi[4] = {y01.x, y01.y, y23.x, y23.y};
            const double hdx = second ? hx : zero_like(hx), hdy = second ? hy : zero_like(hy);
#pragma unroll
            for (int c = 0; c < 4; c++) {
                qi[c] = fma(-hdx, gxi[c], fma(-hdy, gyi[c], q[c * ld + i]));
                q0t[c] = fma(-hdx, gx0[c], fma(-hdy, gy0[c], q0[c]));
            }
            const Prim Pi = q_to_prim(T, qi);
            const Prim P0 = q_to_prim(T, q0t);
            // the slot's sub-stencils (x then y, or t then n): one loop body
#pragma unroll 1
            for (int sb = 0; sb < 2; sb++) {
                const int m = sb == 0 ? (mb & 3) : (mb >> 2);
                if (!m) continue;
                const bool pos = m & 1, xdir = sb == 0;
                const double w = xdir ? d.w1[e] : d.w2[e];
                const double dx = xdir ? e1x : e2x, dy = xdir ? e1y : e2y;
                double Gi[4], G0[4];
                split_flux(T, Pi, framed, xdir, dx, dy, pos, Gi);
                split_flux(T, P0, framed, xdir, dx, dy, pos, G0);
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    if (COMP) y[c] = fma(w, Gi[c] - G0[c], y[c]);
                    else R[c] = fma(w, Gi[c] - G0[c], R[c]);
                }
            }
            if (COMP && ++ng == 4) {
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    comp_add(R[c], Rc[c], y[c]);
                    y[c] = -Rc[c];
                }
                ng = 0;
            }
        }
        if (COMP && ng > 0) {
#pragma unroll
            for (int c = 0; c < 4; c++) comp_add(R[c], Rc[c], y[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        if (COMP) R[c] -= Rc[c];
        R[c] = group_sum<TPP>(R[c]);
    }
    if (work && sub == 0) {
        if (fl == kOuter) {
            // kinetic far field: the n- side is free-stream ghosts at the mirror
            // images of the inside neighbours, LS_3(1) (G_n^-(U_inf) - G_n^-(U_0))
            // with LS_3(1) = -LS_2(1); first order (the point's own state)
            const double *ui = d.case_uinf + 4 * d.case_of[k];
            double U0[4], Ui[4];
            bool same = true;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                U0[c] = st.U[c * ld + k];
                Ui[c] = ui[c];
                same = same && U0[c] == Ui[c];
            }
            if (!same) {  // (equal states give exactly 0)
                double Gi[4], G0[4];
                flux_cons(T, Ui, e2x, e2y, false, Gi);
                flux_cons(T, U0, e2x, e2y, false, G0);
                const double l3 = d.geo[G_LS1_3 * ld + k];
#pragma unroll
                for (int c = 0; c < 4; c++) R[c] = fma(l3, Gi[c] - G0[c], R[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < 4; c++) d.R[c * ld + k] = R[c];
        // local time step (reading: CFL min_i|dr| / (|u| + a)) and the scalar
        // diagonal of Eq. 26 with the spectral radii of Eq. 34, kept at least
        // sum_s rho_s sum_i |w_i| so that it bounds the off-diagonal blocks
        const double *pr = st.prim + (size_t)k * kPrimStride;
        const double u = pr[P_U], v = pr[P_V];
        const double a = sqrt(1.4 * pr[P_P] * pr[P_IRHO]);
        const double dt = cfl * d.geo[G_DMIN * ld + k] / (sqrt(u * u + v * v) + a);
        // D and 1/D: the sweeps multiply by 1/D (one division per point here
        // instead of one per point in each sweep)
        if (d.scheme == 1) {  // explicit: D = 1/dt, the step is -dt R
            d.D[k] = 1.0 / dt;
            d.iD[k] = dt;
            return;
        }
        if (d.lusgs == 1) {  // revised LU-SGS: Jameson's splitting, rho(A_d) = |u_d| + a
            const double u1 = fabs(u * e1x + v * e1y) + a, u2 = fabs(u * e2x + v * e2y) + a;
            const double Dm = 1.0 / dt +
                              0.5 * (u1 * (fabs(d.geo[G_LS1_0 * ld + k]) + fabs(d.geo[G_LS1_1 * ld + k])) +
                                     u2 * (fabs(d.geo[G_LS1_2 * ld + k]) + fabs(d.geo[G_LS1_3 * ld + k])));
            d.D[k] = Dm;
            d.iD[k] = 1.0 / Dm;
            return;
        }
        double Dp = 1.0 / dt, Ddom = 0.0;
        const double u1 = u * e1x + v * e1y, u2 = u * e2x + v * e2y;
        const double r0 = fmax(u1 + a, 0.0), r1 = fmax(a - u1, 0.0);
        const double r2 = fmax(u2 + a, 0.0), r3 = fmax(a - u2, 0.0);
        Dp -= r0 * d.geo[G_LS1_0 * ld + k];
        Dp += r1 * d.geo[G_LS1_1 * ld + k];
        Dp -= r2 * d.geo[G_LS1_2 * ld + k];
        Dp += r3 * d.geo[G_LS1_3 * ld + k];
        Ddom = r0 * d.geo[G_ABS_0 * ld + k] + r1 * d.geo[G_ABS_1 * ld + k] + r2 * d.geo[G_ABS_2 * ld + k]
             + r3 * d.geo[G_ABS_3 * ld + k];
        const double Da = Dp > Ddom ? Dp : Ddom;
        d.D[k] = Da;
        d.iD[k] = 1.0 / Da;
    }
}

// ---------------------------------------------------------------------------
// per-case residual norms, histories and stopping tests (two stages)
// ---------------------------------------------------------------------------
// Stage 1: block j sums R_rho^2 over caller positions [blk_pos[j], blk_pos[j+1]),
// all of one case (frozen outer points hold R = 0).  Fixed order: warp butterfly,
// then warp 0.
__global__ void __launch_bounds__(256) k_norm_partials(Dev d)
{
    __shared__ double red[4][8];
    if (halted(d.ctrl)) return;
    const int j = blockIdx.x;
    const int p = d.blk_pos[j] + threadIdx.x;
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    if (p < d.blk_pos[j + 1]) {
        const int k = d.inv[p];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const double r = d.R[c * d.ld + k];
            t[c] = r * r;
        }
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t[c] += __shfl_xor_sync(kFull, t[c], o);
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = t[c];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            double s = threadIdx.x < 8 ? red[c][threadIdx.x] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
            if (threadIdx.x == 0) d.blk[4 * j + c] = s;
        }
    }
}

// Stage 2: one block per case adds the case's partials in a fixed order,
// records the norm and applies the stopping test.
__global__ void __launch_bounds__(256) k_norm_cases(Dev d)
{
    __shared__ double red[4][8];
    if (halted(d.ctrl)) return;
    const int b = blockIdx.x;
    Ctrl *c = d.ctrl;
    if (frozen_state(((volatile int32_t *)c->case_state)[b])) return;  // block-uniform
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = d.case_blk[b] + threadIdx.x; j < d.case_blk[b + 1]; j += blockDim.x)
#pragma unroll
        for (int q = 0; q < 4; q++) t[q] += d.blk[4 * j + q];
#pragma unroll
    for (int q = 0; q < 4; q++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t[q] += __shfl_xor_sync(kFull, t[q], o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = t[q];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double sq[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            sq[q] = threadIdx.x < 8 ? red[q][threadIdx.x] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sq[q] += __shfl_xor_sync(kFull, sq[q], o);
        }
        const double s = sq[0];
        if (threadIdx.x == 0) {
            const int n0 = c->case_it[b];
            if (n0 < c->hist_cap)
#pragma unroll
                for (int q = 0; q < 4; q++) c->hist4[((size_t)b * c->hist_cap + n0) * 4 + q] = sqrt(sq[q]);
            const double nrm = sqrt(s);
            const int n = c->case_it[b];
            if (n < c->hist_cap) c->hist[(size_t)b * c->hist_cap + n] = nrm;
            if (!(c->case_hist0[b] > 0.0)) c->case_hist0[b] = nrm;
            c->case_it[b] = n + 1;
            if (!isfinite(nrm)) {
                if (c->n_cases > 1) {  // this case only: frozen from its sweeps on
                    c->case_state[b] = kFailed;
                    c->case_err[b] = -4;  // LSKUM_ERR_DIVERGED
                } else {
                    atomicExch(&c->error, -4);
                    atomicMin(&c->bad_point, -1 - b);
                }
            } else if (c->target > 0.0 && nrm / c->case_hist0[b] <= c->target) {
                c->case_state[b] = kReachedTarget;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// LU-SGS sweep, one colour level; G lanes per point
// ---------------------------------------------------------------------------
// Positions [lb, le) of the level's point order (sw_fwd / sw_bwd).  The
// forward sweep sums over each point's lower list (neighbours earlier in the
// sweep order, whose dU* this sweep already produced), the backward sweep
// over its upper list (neighbours later in the order, dU already final).
// T is the sweep arithmetic: double, or float in the mixed-precision mode
// (increments, weights, primal records and Jacobian products in FP32; R and
// D are read in FP64 and rounded once per point).
template <typename T>
struct SweepBufs {
    T *dUs, *dU;
    const T *lo_w1, *lo_w2, *up_w1, *up_w2, *prim;
    T *jc;  // packed form's per-point axis products
};

template <typename T>
__device__ __forceinline__ SweepBufs<T> sweep_bufs(const Dev &d, const StateSet &st);

template <>
__device__ __forceinline__ SweepBufs<double> sweep_bufs<double>(const Dev &d, const StateSet &st)
{
    return {d.dUs, d.dU, d.lo_w1, d.lo_w2, d.up_w1, d.up_w2, st.prim, d.jc};
}

template <>
__device__ __forceinline__ SweepBufs<float> sweep_bufs<float>(const Dev &d, const StateSet &st)
{
    return {d.dUsf, d.dUf, d.lo_w1f, d.lo_w2f, d.up_w1f, d.up_w2f, st.primf, d.jcf};
}

// One slot of a point's lower / upper list: acc += w_s J_s(U_i) dW_i over the
// split sub-stencils s the slot joins (exact AD or increment products).
template <int JVP, typename T>
__device__ __forceinline__ void sweep_slot(const Dev &d, const StateSet &st, const MathTables &Tb,
                                           const T *__restrict__ dW, const T *__restrict__ pr, bool framed,
                                           double e1x, double e1y, double e2x, double e2y, int i, int mb, T w1,
                                           T w2, T acc[4])
{
    T dl[4];
#pragma unroll
    for (int c = 0; c < 4; c++) dl[c] = dW[4 * i + c];
    if (JVP == 0 && !framed) {
        // interior frame: d = (1,0) or (0,1); A+-, exp(-S^2)/sqrt(pi), B,
        // 2 B S and u_d e1 precomputed per point
        const PrimT<T> P = load_prim(pr, i);
        const T *rec = pr + (size_t)i * kPrimStride;
        const JvpBase<T> jb = jvp_base(P, dl);
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const int m = s == 0 ? (mb & 3) : (mb >> 2);
            if (!m) continue;
            const bool pos = m & 1;
            T J[4];
            if (s == 0)
                jvp_axis<0, T>(P, jb, pos, rec[pos ? P_APX : P_AMX], rec[P_EKX], rec[P_BX], rec[P_BSX], rec[P_UE1],
                               J);
            else
                jvp_axis<1, T>(P, jb, pos, rec[pos ? P_APY : P_AMY], rec[P_EKY], rec[P_BY], rec[P_BSY], rec[P_VE1],
                               J);
            const T w = s == 0 ? w1 : w2;
#pragma unroll
            for (int c = 0; c < 4; c++) acc[c] = fma(w, J[c], acc[c]);
        }
    } else {
        // (t, n) frames and the increment form: evaluated in FP64
        double dld[4];
#pragma unroll
        for (int c = 0; c < 4; c++) dld[c] = (double)dl[c];
        const int ld = d.ld;
        double Ui[4], Up[4];
        PrimU P;
        JvpBase<double> jb{};
        if (JVP == 0) {
            P = load_prim(st.prim, i);
            jb = jvp_base(P, dld);
        } else {
#pragma unroll
            for (int c = 0; c < 4; c++) {
                Ui[c] = st.U[c * ld + i];
                Up[c] = Ui[c] + dld[c];
            }
        }
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const int m = s == 0 ? (mb & 3) : (mb >> 2);
            if (!m) continue;
            const bool pos = m & 1;
            const double sg = pos ? 1.0 : -1.0;
            const double ddx = s == 0 ? e1x : e2x, ddy = s == 0 ? e1y : e2y;
            double J[4];
            if (JVP == 0) {
                const double S = (P.u * ddx + P.v * ddy) * P.sb;
                double A, eS;
                split_A(Tb, S, pos, A, eS);
                jvp_dir(P, jb, ddx, ddy, sg, S, A, eS, eS * kInv2SqrtPi * P.isb, J);
            } else {
                double G1[4], G0[4];
                flux_cons(Tb, Up, ddx, ddy, pos, G1);
                flux_cons(Tb, Ui, ddx, ddy, pos, G0);
#pragma unroll
                for (int c = 0; c < 4; c++) J[c] = G1[c] - G0[c];
            }
            const T w = s == 0 ? w1 : w2;
#pragma unroll
            for (int c = 0; c < 4; c++) acc[c] = fma(w, (T)J[c], acc[c]);
        }
    }
}

// Point k's new increment from its list sum acc: forward dU*_k = -(R_k (+ S_k)
// + acc) / D_k, backward dU_k = dU*_k - acc / D_k; normal momentum removed at
// wall points.  Stored, and returned in w.
template <bool FWD, typename T>
__device__ __forceinline__ void sweep_point(const Dev &d, const StateSet &st, const SweepBufs<T> &sb, int k,
                                            bool wall, double e1x, double e1y, double e2x, double e2y,
                                            const T acc[4], T w[4])
{
    const int ld = d.ld;
    const T iD = (T)d.iD[k];
    if (FWD) {
        double rhs[4];
#pragma unroll
        for (int c = 0; c < 4; c++) rhs[c] = d.R[c * ld + k];
        if (d.lusgs == 1) {
            // revised LU-SGS: -R - S with S_0 = -1/2 sum_s LS_s(1) A_d(U_0) dU_0 of
            // the previous iteration's increment (still in dU: the backward
            // sweep of this iteration has not run)
            double dp[4];
#pragma unroll
            for (int c = 0; c < 4; c++) dp[c] = d.dUf ? (double)d.dUf[4 * k + c] : d.dU[4 * k + c];
            const double *pk = st.prim + (size_t)k * kPrimStride;
            double J1[4], J2[4];
            euler_jvp(pk[P_RHO], pk[P_U], pk[P_V], pk[P_P], dp, e1x, e1y, J1);
            euler_jvp(pk[P_RHO], pk[P_U], pk[P_V], pk[P_P], dp, e2x, e2y, J2);
            const double l1 = d.geo[G_LS1_0 * ld + k] + d.geo[G_LS1_1 * ld + k];
            const double l2 = d.geo[G_LS1_2 * ld + k] + d.geo[G_LS1_3 * ld + k];
#pragma unroll
            for (int c = 0; c < 4; c++) rhs[c] -= 0.5 * (l1 * J1[c] + l2 * J2[c]);  // R + S
        }
#pragma unroll
        for (int c = 0; c < 4; c++) w[c] = -((T)rhs[c] + acc[c]) * iD;
    } else {
#pragma unroll
        for (int c = 0; c < 4; c++) w[c] = fma(-acc[c], iD, sb.dUs[4 * k + c]);
    }
    if (wall) {
        const T nx = (T)d.wnx[k], ny = (T)d.wny[k];
        const T mn = w[1] * nx + w[2] * ny;
        w[1] -= mn * nx;
        w[2] -= mn * ny;
    }
    T *out = FWD ? sb.dUs : sb.dU;
#pragma unroll
    for (int c = 0; c < 4; c++) out[4 * k + c] = w[c];
}

// The frame of point k: (1,0), (0,1), or (t, n) at wall and kinetic outer points.
__device__ __forceinline__ void point_frame(const Dev &d, int k, bool framed, double &e1x, double &e1y, double &e2x,
                                            double &e2y)
{
    e1x = 1.0, e1y = 0.0, e2x = 0.0, e2y = 1.0;
    if (framed) {
        const int ld = d.ld;
        e1x = d.geo[G_E1X * ld + k];
        e1y = d.geo[G_E1Y * ld + k];
        e2x = d.geo[G_E2X * ld + k];
        e2y = d.geo[G_E2Y * ld + k];
    }
}

// G lanes per point over the point's list, butterfly reduction.
template <int JVP, bool FWD, int G, typename T>
__global__ void __launch_bounds__(256) k_sweep(Dev d, StateSet st, int lb, int le)
{
    const MathTables &Tb = g_math;  // wall and outer points only: no per-block copy
    if (halted(d.ctrl)) return;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    if (lb + (gt & ~31) / G >= le) return;  // the whole warp is past the level
    const int pos = lb + gt / G, sub = gt % G;
    const bool active = pos < le;
    const int k = (FWD ? d.sw_fwd : d.sw_bwd)[active ? pos : le - 1];
    const bool live = active && !frozen(d, k);
    const SweepBufs<T> sb = sweep_bufs<T>(d, st);
    const int32_t *__restrict__ off = FWD ? d.lo_off : d.up_off;
    const int32_t *__restrict__ nbr = FWD ? d.lo_nbr : d.up_nbr;
    const uint8_t *__restrict__ mbs = FWD ? d.lo_mb : d.up_mb;
    const T *__restrict__ w1s = FWD ? sb.lo_w1 : sb.up_w1;
    const T *__restrict__ w2s = FWD ? sb.lo_w2 : sb.up_w2;
    const T *__restrict__ dW = FWD ? sb.dUs : sb.dU;
    const int fk = d.flag[k];
    const bool wall = fk == kWall, framed = fk != kInterior;
    double e1x, e1y, e2x, e2y;
    point_frame(d, k, framed, e1x, e1y, e2x, e2y);
    T acc[4] = {T(0), T(0), T(0), T(0)};
    const int beg = off[k], end = live ? off[k + 1] : beg;
    for (int e = beg + sub; e < end; e += G)
        sweep_slot<JVP, T>(d, st, Tb, dW, sb.prim, framed, e1x, e1y, e2x, e2y, nbr[e], mbs[e], w1s[e], w2s[e], acc);
#pragma unroll
    for (int c = 0; c < 4; c++) acc[c] = group_sum<G>(acc[c]);
    T w[4];
    if (live && sub == 0) sweep_point<FWD, T>(d, st, sb, k, wall, e1x, e1y, e2x, e2y, acc, w);
}

// Four consecutive values from 16-byte-aligned storage (one point's product).
__device__ __forceinline__ void load4(const double *__restrict__ p, double v[4])
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
__device__ __forceinline__ void load4(const float *__restrict__ p, float v[4])
{
    const float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
}

__device__ __forceinline__ void store4(double *p, const double v[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void store4(float *p, const float v[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// Axis product cb (0: x+, 1: x-, 2: y+, 3: y-) of point k's new increment w
// in the increment form, G_d(U_k + w) - G_d(U_k) in FP64 (the value an
// interior point whose list holds k would form for that sub-stencil),
// stored once for every later level to gather.  (The exact products are
// formed by jvp_axis_sel from the point's record, or from the framed
// points' precomputed Jacobians.)
template <typename T>
__device__ __forceinline__ void store_increment_product(const Dev &d, const StateSet &st, const MathTables &Tb,
                                                        const SweepBufs<T> &sb, const T w[4], int k, int cb)
{
    const bool pos = !(cb & 1);
    const int ld = d.ld;
    double Ui[4], Up[4], G1[4], G0[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        Ui[c] = st.U[c * ld + k];
        Up[c] = Ui[c] + (double)w[c];
    }
    const double ddx = cb < 2 ? 1.0 : 0.0, ddy = cb < 2 ? 0.0 : 1.0;
    flux_cons(Tb, Up, ddx, ddy, pos, G1);
    flux_cons(Tb, Ui, ddx, ddy, pos, G0);
    T J[4];
#pragma unroll
    for (int c = 0; c < 4; c++) J[c] = (T)(G1[c] - G0[c]);
    store4(sb.jc + 16 * (size_t)k + 4 * cb, J);
}

// Threads per block of the packed sweeps: a level is only a few thousand
// warps, so small blocks spread them evenly over the SMs (whole blocks of
// eight warps left half the SMs with one block and half with two).
#ifndef LSKUM_SWEEP_BLOCK
#define LSKUM_SWEEP_BLOCK 64
#endif
constexpr int kSweepBlock = LSKUM_SWEEP_BLOCK;
static_assert(kSweepBlock % 32 == 0 && kSweepBlock <= 256, "sweep block");

// Packed form of a level.  A neighbour's Jacobian product along an axis
// depends only on the neighbour, the axis and the sub-stencil's sign, so a
// point forms the four axis products of its new increment once, and
// interior points gather them: 8 FMAs per slot instead of ~70 FP64
// instructions.  A point's sum depends only on its own list, in a fixed
// order, so a batch still equals its single solves bit for bit.
// - wf warps for the points in a (t, n) frame, their slots packed whole into
//   warps (at create, by best fit; a point with an empty list takes one idle
//   slot), one lane per slot.  Exact products: the lane applies the slot's
//   weighted Jacobian, formed for the whole iteration by k_framed_jac (16
//   FMAs); increments: the split fluxes per slot in the point's frame.  A
//   segmented suffix sum over the lanes of each point (fixed tree order, no
//   atomics) leaves the point's sum in its first lane, which finishes the
//   point; the point's lanes share its four axis products (exact: its
//   precomputed axis Jacobians).  Packed warps [wb, wb + wf) are the
//   level's; they are spread evenly over the grid (every S-th warp).
// - ng warps for the interior points, kLanesPerPoint lanes per point,
//   kPointsPerWarp points of similar list length per warp (groups
//   [g0, g0 + ng) are the level's), in the other warp positions in order.
//   A level is a chain of dependent loads (list, gathers, the point's own
//   record) and a short FP64 sequence per lane, so the point's own loads
//   are issued before the gathers, and the x- and y-products of a warp's
//   lanes share one branch-free FP64 sequence (jvp_axis_sel).
template <int JVP, bool FWD, typename T>
__global__ void __launch_bounds__(kSweepBlock) k_sweep_packed(Dev d, StateSet st, int wb, int wf, int g0, int ng)
{
    const MathTables &Tb = g_math;  // framed points only: no per-block copy
    if (halted(d.ctrl)) return;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (gw >= wf + ng) return;  // whole warps (blocks are whole warps)
    const int lane = threadIdx.x & 31;
    const int dir = FWD ? 0 : 1;
    const SweepBufs<T> sb = sweep_bufs<T>(d, st);
    const T *__restrict__ dW = FWD ? sb.dUs : sb.dU;  // earlier levels' increments
    const T *__restrict__ jn = sb.jc;                 // earlier levels' axis products
    T acc[4] = {T(0), T(0), T(0), T(0)};
    T w[4] = {T(0), T(0), T(0), T(0)};
    const int S = max(1, (wf + ng) / max(wf, 1)), q = gw / S;  // framed warp q at position q S
    if (wf > 0 && gw % S == 0 && q < wf) {
        const int fw = wb + q;
        const size_t e = (size_t)fw * 32 + lane;
        const int pos = d.pk_pt[dir][e];  // sweep position of the slot's point, -1: padding
        const int k = pos >= 0 ? (FWD ? d.sw_fwd : d.sw_bwd)[pos] : 0;
        const bool live = pos >= 0 && !frozen(d, k);
        const int fk = d.flag[k];
        const bool wall = fk == kWall, framed = fk != kInterior;
        double e1x, e1y, e2x, e2y;
        point_frame(d, k, framed, e1x, e1y, e2x, e2y);
        const int mb = d.pk_mb[dir][e];
        if (live && mb) {
            if (JVP == 0) {
                // the slot's weighted Jacobian, formed before the sweeps: acc += M dW_i
                const T *__restrict__ M = (sizeof(T) == 4 ? (const T *)d.pk_jmf[dir] : (const T *)d.pk_jm[dir]) + 16 * e;
                T dl[4];
                load4(dW + 4 * (size_t)d.pk_nbr[dir][e], dl);
#pragma unroll
                for (int c = 0; c < 4; c++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[c] = fma(M[4 * c + j], dl[j], acc[c]);
            } else {
                const T w1 = sizeof(T) == 4 ? (T)d.pk_w1f[dir][e] : (T)d.pk_w1[dir][e];
                const T w2 = sizeof(T) == 4 ? (T)d.pk_w2f[dir][e] : (T)d.pk_w2[dir][e];
                sweep_slot<JVP, T>(d, st, Tb, dW, sb.prim, framed, e1x, e1y, e2x, e2y, d.pk_nbr[dir][e], mb, w1,
                                   w2, acc);
            }
        }
        // segmented suffix sum: lane l adds lane l + o when both hold the same
        // point; the warp's longest list bounds the steps (warp-uniform)
        const int steps = d.pk_steps[dir][fw];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            if (o >= (1 << steps)) break;
            const int p2 = __shfl_down_sync(kFull, pos, o);
            T v[4];
#pragma unroll
            for (int c = 0; c < 4; c++) v[c] = __shfl_down_sync(kFull, acc[c], o);
            if (lane + o < 32 && p2 == pos) {
#pragma unroll
                for (int c = 0; c < 4; c++) acc[c] += v[c];
            }
        }
        // the point's lanes (consecutive; padding lanes form their own group):
        // the first finishes the point, then lane r of the point's seg lanes
        // forms the products r, r + seg, ... of the new increment
        const unsigned m = __match_any_sync(kFull, pos);
        const int head = __ffs(m) - 1, seg = __popc(m), r = lane - head;
        if (live && r == 0) sweep_point<FWD, T>(d, st, sb, k, wall, e1x, e1y, e2x, e2y, acc, w);
#pragma unroll
        for (int c = 0; c < 4; c++) w[c] = __shfl_sync(kFull, w[c], head);
        if (live) {
            if (JVP == 0) {
                // the point's axis Jacobians, formed before the sweeps
                const T *__restrict__ F =
                    (sizeof(T) == 4 ? (const T *)d.fjf : (const T *)d.fj) + 64 * (size_t)d.fidx[k];
                for (int cb = r; cb < 4; cb += seg) {
                    T J[4];
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        J[c] = F[16 * cb + 4 * c] * w[0];
#pragma unroll
                        for (int j = 1; j < 4; j++) J[c] = fma(F[16 * cb + 4 * c + j], w[j], J[c]);
                    }
                    store4(sb.jc + 16 * (size_t)k + 4 * cb, J);
                }
            } else {
                for (int cb = r; cb < 4; cb += seg) store_increment_product<T>(d, st, Tb, sb, w, k, cb);
            }
        }
        return;
    }
    // interior points: kLanesPerPoint lanes per point, lane s taking the
    // point's slots j = s (mod kLanesPerPoint) in order; a butterfly over the
    // point's lanes gives every one of them the same sum (each addition has
    // the same two operands in either order)
    const int g = g0 + gw - min(wf, q + 1);  // the framed positions up to gw left out
    const int p = lane / kLanesPerPoint, s = lane % kLanesPerPoint;
    const int k = d.lp_k[dir][kPointsPerWarp * g + p];
    const bool live = k >= 0 && !frozen(d, k);
    const int len = live ? d.lp_len[dir][kPointsPerWarp * g + p] : 0;
    const int kk = k >= 0 ? k : 0;  // index for the loads of a slot without a point
    // loads that depend only on the point, issued before the gathers so that
    // their latency overlaps theirs: this lane's entries of the point's
    // primal record (its axis product s: 0 x+, 1 x-, 2 y+, 3 y-) and, in the
    // point's first lane, the right-hand side (R forward, dU* backward) and 1/D
    const bool xdir = s < 2, psg = !(s & 1);
    PrimT<T> P{};
    T rA = T(0), rEK = T(0), rB = T(0), rBS = T(0), rUE = T(0);
    if (JVP == 0) {
        P = load_prim(sb.prim, kk);
        const T *rec = sb.prim + (size_t)kk * kPrimStride;
        rA = rec[xdir ? (psg ? P_APX : P_AMX) : (psg ? P_APY : P_AMY)];
        rEK = rec[xdir ? P_EKX : P_EKY];
        rB = rec[xdir ? P_BX : P_BY];
        rBS = rec[xdir ? P_BSX : P_BSY];
        rUE = rec[xdir ? P_UE1 : P_VE1];
    }
    const bool plain = d.lusgs == 0;  // the revised LU-SGS adds its lagged term in sweep_point
    double rhs[4] = {0.0, 0.0, 0.0, 0.0};
    T iDk = T(0);
    if (s == 0 && plain) {
        iDk = (T)d.iD[kk];
        if (FWD) {
            const int ld = d.ld;
#pragma unroll
            for (int c = 0; c < 4; c++) rhs[c] = d.R[c * ld + kk];
        } else {
            T v[4];
            load4(sb.dUs + 4 * (size_t)kk, v);
#pragma unroll
            for (int c = 0; c < 4; c++) rhs[c] = (double)v[c];
        }
    }
    const size_t base = (size_t)d.lp_goff[dir][g] + lane;
#pragma unroll 4
    for (int j = s; j < len; j += kLanesPerPoint) {
        const size_t e = base + 32 * (size_t)(j / kLanesPerPoint);
        const int i = d.lp_nbr[dir][e], mb = d.lp_mb[dir][e];
        T J[4];
        if (mb & 3) {
            const T w1 = sizeof(T) == 4 ? (T)d.lp_w1f[dir][e] : (T)d.lp_w1[dir][e];
            load4(jn + 16 * (size_t)i + ((mb & 1) ? 0 : 4), J);
#pragma unroll
            for (int c = 0; c < 4; c++) acc[c] = fma(w1, J[c], acc[c]);
        }
        if (mb & 12) {
            const T w2 = sizeof(T) == 4 ? (T)d.lp_w2f[dir][e] : (T)d.lp_w2[dir][e];
            load4(jn + 16 * (size_t)i + ((mb & 4) ? 8 : 12), J);
#pragma unroll
            for (int c = 0; c < 4; c++) acc[c] = fma(w2, J[c], acc[c]);
        }
    }
#pragma unroll
    for (int o = 1; o < kLanesPerPoint; o <<= 1) {
#pragma unroll
        for (int c = 0; c < 4; c++) acc[c] += __shfl_xor_sync(kFull, acc[c], o);
    }
    // the point's first lane finishes it (forward dU* = -(R + acc) / D,
    // backward dU = dU* - acc / D); each of its lanes then forms one of the
    // four axis products of the new increment
#pragma unroll
    for (int c = 0; c < 4; c++) w[c] = T(0);
    if (live && s == 0) {
        if (plain) {
#pragma unroll
            for (int c = 0; c < 4; c++) w[c] = FWD ? -((T)rhs[c] + acc[c]) * iDk : fma(-acc[c], iDk, (T)rhs[c]);
            store4((FWD ? sb.dUs : sb.dU) + 4 * (size_t)k, w);
        } else {
            sweep_point<FWD, T>(d, st, sb, k, false, 1.0, 0.0, 0.0, 1.0, acc, w);
        }
    }
#pragma unroll
    for (int c = 0; c < 4; c++) w[c] = __shfl_sync(kFull, w[c], lane - s);
    if (live) {
        if (JVP == 0) {
            const JvpBase<T> jb = jvp_base(P, w);
            T J[4];
            jvp_axis_sel<T>(P, jb, xdir, psg, rA, rEK, rB, rBS, rUE, J);
            store4(sb.jc + 16 * (size_t)k + 4 * s, J);
        } else {
            store_increment_product<T>(d, st, Tb, sb, w, k, s);
        }
    }
}

// Jacobians of the framed points' products for the packed sweeps (exact
// products).  The split-flux Jacobian A_d^+-(U_i) is the derivative of
// G_d^+- at the state of this iteration and does not depend on the sweeps'
// increments, so every matrix that the two sweeps apply at the points in a
// (t, n) frame is formed here, all in parallel, before the forward sweep;
// inside the levels the framed points' chains are then matrix-vector
// products.  One thread per (slot lane, column) of pk_jm -- M = w1 A_e1 +
// w2 A_e2 at the neighbour's state in the point's frame -- and per (framed
// point, axis product, column) of fj -- A_x+-, A_y+- at the point's own
// state.  Column j is the forward-mode tangent along the unit vector e_j,
// evaluated in FP64 by the functions of the per-slot form (stored as T).
template <typename T>
__global__ void __launch_bounds__(256) k_framed_jac(Dev d, StateSet st)
{
    __shared__ MathTables Tb;
    if (halted(d.ctrl)) return;
    load_math_tables(Tb);
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int n0 = 4 * d.pk_lanes[0], n1 = 4 * d.pk_lanes[1], nfj = 16 * d.nf;
    if (t >= n0 + n1 + nfj) return;
    const int j = t & 3;  // n0 and n1 are multiples of 4
    double dl[4];
#pragma unroll
    for (int c = 0; c < 4; c++) dl[c] = c == j ? 1.0 : 0.0;  // the unit vector e_j
    if (t < n0 + n1) {
        const int dir = t < n0 ? 0 : 1;
        const int e = (t - (dir ? n0 : 0)) >> 2;
        T *M = (sizeof(T) == 4 ? (T *)d.pk_jmf[dir] : (T *)d.pk_jm[dir]) + 16 * (size_t)e;
        const int pos = d.pk_pt[dir][e];
        const int mb = d.pk_mb[dir][e];
        double col[4] = {0.0, 0.0, 0.0, 0.0};
        if (pos >= 0 && mb) {
            const int k = (dir == 0 ? d.sw_fwd : d.sw_bwd)[pos];
            double e1x, e1y, e2x, e2y;
            point_frame(d, k, true, e1x, e1y, e2x, e2y);
            const PrimU P = load_prim(st.prim, d.pk_nbr[dir][e]);
            const JvpBase<double> jb = jvp_base(P, dl);
#pragma unroll
            for (int s = 0; s < 2; s++) {
                const int m = s == 0 ? (mb & 3) : (mb >> 2);
                if (!m) continue;
                const bool pos_s = m & 1;
                const double sg = pos_s ? 1.0 : -1.0;
                const double ddx = s == 0 ? e1x : e2x, ddy = s == 0 ? e1y : e2y;
                const double S = (P.u * ddx + P.v * ddy) * P.sb;
                double A, eS, J[4];
                split_A(Tb, S, pos_s, A, eS);
                jvp_dir(P, jb, ddx, ddy, sg, S, A, eS, eS * kInv2SqrtPi * P.isb, J);
                const double w = s == 0 ? d.pk_w1[dir][e] : d.pk_w2[dir][e];
#pragma unroll
                for (int c = 0; c < 4; c++) col[c] = fma(w, J[c], col[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < 4; c++) M[4 * c + j] = (T)col[c];
        return;
    }
    const int u = t - n0 - n1;
    const int f = u >> 4, cb = (u >> 2) & 3;
    const int k = d.fpt[f];
    const PrimU P = load_prim(st.prim, k);
    const double *rec = st.prim + (size_t)k * kPrimStride;
    const JvpBase<double> jb = jvp_base(P, dl);
    const bool pos = !(cb & 1);
    double J[4];
    if (cb < 2)
        jvp_axis<0, double>(P, jb, pos, rec[pos ? P_APX : P_AMX], rec[P_EKX], rec[P_BX], rec[P_BSX], rec[P_UE1], J);
    else
        jvp_axis<1, double>(P, jb, pos, rec[pos ? P_APY : P_AMY], rec[P_EKY], rec[P_BY], rec[P_BSY], rec[P_VE1], J);
    T *F = (sizeof(T) == 4 ? (T *)d.fjf : (T *)d.fj) + 64 * (size_t)f + 16 * cb;
#pragma unroll
    for (int c = 0; c < 4; c++) F[4 * c + j] = (T)J[c];
}

// ---------------------------------------------------------------------------
// state update (set cur -> set 1-cur) and per-point quantities of the new state
// ---------------------------------------------------------------------------
__global__ void k_begin(Ctrl *c)
{
    if (c->stop | c->error) return;
    int running = 0;
    for (int b = 0; b < c->n_cases; b++) {
        if (c->case_state[b] == kReachedTarget) c->case_state[b] = kStopped;
        if (c->case_state[b] == kFailedNow) c->case_state[b] = kFailed;
        running += !frozen_state(c->case_state[b]);
    }
    if (running == 0) c->stop = 1;
    else c->it += 1;
}

// One kernel for both uses (inc: after an iteration, set cur -> 1 - cur; not
// inc: a new state in set cur), so that q and the per-point records of a
// given U come from the same instructions either way: a resumed checkpoint
// continues bit for bit.
__global__ void __launch_bounds__(256) k_update(Dev d, int cur, bool inc, bool project)
{
    __shared__ MathTables T;
    if (inc && halted(d.ctrl)) return;
    load_math_tables(T);
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    const int ld = d.ld;
    const StateSet src = d.set[cur];
    const StateSet dst = d.set[inc ? 1 - cur : cur];
    const int fl = d.flag[k];
    double U[4];
#pragma unroll
    for (int c = 0; c < 4; c++) U[c] = src.U[c * ld + k];
    const bool moves = inc && (fl != kOuter || d.farfield == 1) && !frozen(d, k);
    if (moves) {
#pragma unroll
        for (int c = 0; c < 4; c++) U[c] += d.dUf ? (double)d.dUf[4 * k + c] : d.dU[4 * k + c];
    }
    // wall projection of a moved point, or of a new state built from
    // primitives or predicted (project): re-projecting a projected state
    // could change its last bits, and a stopped case must keep its state
    if (fl == kWall && (moves || (!inc && project))) {
        const double nx = d.wnx[k], ny = d.wny[k];
        const double mn = U[1] * nx + U[2] * ny;
        U[1] -= mn * nx;
        U[2] -= mn * ny;
    }
    const PrimU P = prim_from_cons(U);
    const bool ok = P.rho > 0.0 && P.p > 0.0 && isfinite(P.rho) && isfinite(P.p) && isfinite(P.u) &&
                    isfinite(P.v);
    if (!ok) {
        if (inc && d.n_cases > 1) {  // fail this case only; k_repair restores its state
            const int b = d.case_of[k];
            atomicExch(&d.ctrl->case_state[b], (int32_t)kFailedNow);
            atomicExch(&d.ctrl->case_err[b], -3);  // LSKUM_ERR_NONPOSITIVE
            atomicMin(&d.ctrl->case_bad[b], k);
        } else {
            atomicMin(&d.ctrl->bad_point, k);
            atomicExch(&d.ctrl->error, -3);
        }
        return;
    }
#pragma unroll
    for (int c = 0; c < 4; c++) dst.U[c * ld + k] = U[c];
    // q1 = ln rho + 2.5 ln beta - beta |u|^2 with one logarithm: ln(rho beta^2 sqrt(beta))
    dst.q[0 * ld + k] = fma(-P.beta, P.q2, log(mul_i(mul_i(P.rho, mul_i(P.beta, P.beta)), P.sb)));
    dst.q[1 * ld + k] = mul_i(twice(P.beta), P.u);
    dst.q[2 * ld + k] = mul_i(twice(P.beta), P.v);
    dst.q[3 * ld + k] = signed_by(twice(P.beta), false);
    // the per-point record, assembled in registers and stored as 16-byte
    // vectors (and, in mixed precision, its FP32 copy from the same registers)
    double rec[P_NFIELDS];
    rec[P_RHO] = P.rho;
    rec[P_IRHO] = P.irho;
    rec[P_U] = P.u;
    rec[P_V] = P.v;
    rec[P_P] = P.p;
    rec[P_BETA] = P.beta;
    rec[P_SB] = P.sb;
    rec[P_ISB] = P.isb;
    rec[P_I2P] = P.i2p;
    rec[P_Q2] = P.q2;
    rec[P_E1] = P.e1;
    rec[P_E2] = P.e2;
    const double sx = mul_i(P.u, P.sb), sy = mul_i(P.v, P.sb);
    double Ex, ex, Ey, ey;
    split_E(T, sx, Ex, ex);
    split_E(T, sy, Ey, ey);
    const double bk = mul_i(kInv2SqrtPi, P.isb);
    const double bx = mul_i(ex, bk), by = mul_i(ey, bk);
    rec[P_BSX] = mul_i(twice(bx), sx);
    rec[P_APX] = sx >= 0.0 ? 1.0 - Ex : Ex;
    rec[P_AMX] = sx >= 0.0 ? Ex : 1.0 - Ex;
    rec[P_EKX] = mul_i(ex, kInvSqrtPi);
    rec[P_BX] = bx;
    rec[P_BSY] = mul_i(twice(by), sy);
    rec[P_APY] = sy >= 0.0 ? 1.0 - Ey : Ey;
    rec[P_AMY] = sy >= 0.0 ? Ey : 1.0 - Ey;
    rec[P_EKY] = mul_i(ey, kInvSqrtPi);
    rec[P_BY] = by;
    rec[P_UE1] = mul_i(P.u, P.e1);
    rec[P_VE1] = mul_i(P.v, P.e1);
    static_assert(P_NFIELDS == kPrimStride && kPrimStride % 4 == 0, "record stored as whole vectors");
    double2 *pr2 = reinterpret_cast<double2 *>(dst.prim + (size_t)k * kPrimStride);
#pragma unroll
    for (int f = 0; f < P_NFIELDS / 2; f++) pr2[f] = make_double2(rec[2 * f], rec[2 * f + 1]);
    if (dst.primf) {  // mixed precision: the sweeps' FP32 copy of the record
        float4 *pf4 = reinterpret_cast<float4 *>(dst.primf + (size_t)k * kPrimStride);
#pragma unroll
        for (int f = 0; f < P_NFIELDS / 4; f++)
            pf4[f] = make_float4((float)rec[4 * f], (float)rec[4 * f + 1], (float)rec[4 * f + 2], (float)rec[4 * f + 3]);
    }
}

// Explicit scheme (the paper's solver (e)): dU = -dt R = -R / D at wall and
// interior points (and outer points under the kinetic far field), normal
// momentum removed at wall points; frozen outer points 0.
__global__ void __launch_bounds__(256) k_explicit(Dev d)
{
    if (halted(d.ctrl)) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    const int ld = d.ld;
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    const int fl = d.flag[k];
    if ((fl != kOuter || d.farfield == 1) && !frozen(d, k)) {
        const double dt = d.iD[k];
#pragma unroll
        for (int c = 0; c < 4; c++) w[c] = -dt * d.R[c * ld + k];
        if (fl == kWall) {
            const double nx = d.wnx[k], ny = d.wny[k];
            const double mn = w[1] * nx + w[2] * ny;
            w[1] -= mn * nx;
            w[2] -= mn * ny;
        }
    }
#pragma unroll
    for (int c = 0; c < 4; c++) d.dU[4 * k + c] = w[c];
}

// Batches: undo this iteration's update of the cases that failed in it (the
// new state set gets the old set's values), so a failed case keeps its last
// good state.
__global__ void __launch_bounds__(256) k_repair(Dev d, int cur)
{
    if (halted(d.ctrl)) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    if (((const volatile int32_t *)d.case_state)[d.case_of[k]] != kFailedNow) return;
    const int ld = d.ld;
    const StateSet src = d.set[cur], dst = d.set[1 - cur];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        dst.U[c * ld + k] = src.U[c * ld + k];
        dst.q[c * ld + k] = src.q[c * ld + k];
    }
    for (int f = 0; f < kPrimStride; f++) dst.prim[(size_t)k * kPrimStride + f] = src.prim[(size_t)k * kPrimStride + f];
    if (src.primf)
        for (int f = 0; f < kPrimStride; f++)
            dst.primf[(size_t)k * kPrimStride + f] = src.primf[(size_t)k * kPrimStride + f];
}

__global__ void k_reset_ctrl(Ctrl *c)
{
    c->stop = 0;
    c->error = 0;
    c->bad_point = 0x7fffffff;
}

__global__ void k_prep_run(Ctrl *c, double target)
{
    c->stop = 0;
    c->error = 0;
    c->bad_point = 0x7fffffff;
    c->target = target;
    c->it_start = c->it;
    for (int b = 0; b < c->n_cases; b++)
        c->case_state[b] = (c->case_state[b] == kFailed || c->case_state[b] == kFailedNow) ? kFailed : kRunning;
}

template <int TPP>
cudaError_t enqueue_grad(const Dev &d, int cur, cudaStream_t s, int *launches)
{
    const int gb = (d.n * TPP + 255) / 256;
    const StateSet st = d.set[cur];
    k_grad<TPP, false><<<gb, 256, 0, s>>>(d, st.q, nullptr, d.gq[0]);
    (*launches)++;
    for (int it = 1; it <= d.K; it++) {
        const int a = (it - 1) & 1, b = it & 1;
        k_grad<TPP, true><<<gb, 256, 0, s>>>(d, st.q, d.gq[a], d.gq[b]);
        (*launches)++;
    }
    return cudaGetLastError();
}

template <int TPP>
cudaError_t enqueue_res(const Dev &d, const Launch &L, int cur, cudaStream_t s, int *launches)
{
    const int fin = d.K & 1;
    const int rb = (d.n * TPP + L.res_block - 1) / L.res_block;
    if (d.precision) k_residual<TPP, true><<<rb, L.res_block, 0, s>>>(d, d.set[cur], d.gq[fin]);
    else k_residual<TPP, false><<<rb, L.res_block, 0, s>>>(d, d.set[cur], d.gq[fin]);
    (*launches)++;
    return cudaGetLastError();
}

cudaError_t enqueue_grad_res(const Dev &d, const Launch &L, int cur, cudaStream_t s, int *launches, bool grad,
                             bool res)
{
    cudaError_t e = cudaSuccess;
    switch (L.tpp) {
    case 1:
        if (grad) e = enqueue_grad<1>(d, cur, s, launches);
        if (res && e == cudaSuccess) e = enqueue_res<1>(d, L, cur, s, launches);
        break;
    case 2:
        if (grad) e = enqueue_grad<2>(d, cur, s, launches);
        if (res && e == cudaSuccess) e = enqueue_res<2>(d, L, cur, s, launches);
        break;
    case 4:
        if (grad) e = enqueue_grad<4>(d, cur, s, launches);
        if (res && e == cudaSuccess) e = enqueue_res<4>(d, L, cur, s, launches);
        break;
    case 8:
        if (grad) e = enqueue_grad<8>(d, cur, s, launches);
        if (res && e == cudaSuccess) e = enqueue_res<8>(d, L, cur, s, launches);
        break;
    default: return cudaErrorInvalidValue;
    }
    return e;
}

template <int JVP, int G>
void enqueue_sweeps_g(const Dev &d, int cur, int n_levels, const int32_t *lvl_beg, const int32_t *lvl_act_end,
                      cudaStream_t s, int *launches, bool fwd, bool bwd)
{
    const StateSet st = d.set[cur];
    for (int l = 0; fwd && l < n_levels; l++) {
        const int np = lvl_act_end[l] - lvl_beg[l];
        if (np <= 0) continue;
        const int blocks = (np * G + 255) / 256;
        if (d.precision) k_sweep<JVP, true, G, float><<<blocks, 256, 0, s>>>(d, st, lvl_beg[l], lvl_act_end[l]);
        else k_sweep<JVP, true, G, double><<<blocks, 256, 0, s>>>(d, st, lvl_beg[l], lvl_act_end[l]);
        (*launches)++;
    }
    for (int l = n_levels - 1; bwd && l >= 0; l--) {
        const int np = lvl_act_end[l] - lvl_beg[l];
        if (np <= 0) continue;
        const int blocks = (np * G + 255) / 256;
        if (d.precision) k_sweep<JVP, false, G, float><<<blocks, 256, 0, s>>>(d, st, lvl_beg[l], lvl_act_end[l]);
        else k_sweep<JVP, false, G, double><<<blocks, 256, 0, s>>>(d, st, lvl_beg[l], lvl_act_end[l]);
        (*launches)++;
    }
}

// The packed exact sweeps apply precomputed framed-point Jacobians.
bool needs_framed_jac(const Dev &d, const Launch &L)
{
    return d.scheme == 0 && d.jvp == 0 && L.sweep_lanes == 32 && (d.pk_jm[0] || d.pk_jmf[0]) &&
           4 * (d.pk_lanes[0] + d.pk_lanes[1]) + 16 * d.nf > 0;
}

void enqueue_framed_jac(const Dev &d, int cur, cudaStream_t s, int *launches)
{
    const int items = 4 * (d.pk_lanes[0] + d.pk_lanes[1]) + 16 * d.nf;
    if (d.precision) k_framed_jac<float><<<(items + 255) / 256, 256, 0, s>>>(d, d.set[cur]);
    else k_framed_jac<double><<<(items + 255) / 256, 256, 0, s>>>(d, d.set[cur]);
    (*launches)++;
}

template <int JVP>
void enqueue_sweeps_packed(const Dev &d, const Launch &L, int cur, int n_levels, cudaStream_t s, int *launches,
                           bool fwd, bool bwd)
{
    const StateSet st = d.set[cur];
    if (fwd && needs_framed_jac(d, L)) {
        if (L.side) cudaStreamWaitEvent(s, L.join, 0);  // formed on the side branch
        else enqueue_framed_jac(d, cur, s, launches);
    }
    for (int l = 0; fwd && l < n_levels; l++) {
        const int wb = L.pk_lw[0][l], wf = L.pk_lw[0][l + 1] - wb;
        const int g0 = L.lp_lg[0][l], ng = L.lp_lg[0][l + 1] - g0;
        if (wf + ng <= 0) continue;
        const int blocks = ((wf + ng) * 32 + kSweepBlock - 1) / kSweepBlock;
        if (d.precision) k_sweep_packed<JVP, true, float><<<blocks, kSweepBlock, 0, s>>>(d, st, wb, wf, g0, ng);
        else k_sweep_packed<JVP, true, double><<<blocks, kSweepBlock, 0, s>>>(d, st, wb, wf, g0, ng);
        (*launches)++;
    }
    for (int l = n_levels - 1; bwd && l >= 0; l--) {
        const int wb = L.pk_lw[1][l], wf = L.pk_lw[1][l + 1] - wb;
        const int g0 = L.lp_lg[1][l], ng = L.lp_lg[1][l + 1] - g0;
        if (wf + ng <= 0) continue;
        const int blocks = ((wf + ng) * 32 + kSweepBlock - 1) / kSweepBlock;
        if (d.precision) k_sweep_packed<JVP, false, float><<<blocks, kSweepBlock, 0, s>>>(d, st, wb, wf, g0, ng);
        else k_sweep_packed<JVP, false, double><<<blocks, kSweepBlock, 0, s>>>(d, st, wb, wf, g0, ng);
        (*launches)++;
    }
}

template <int JVP>
cudaError_t enqueue_sweeps(const Dev &d, const Launch &L, int cur, int n_levels, const int32_t *lvl_beg,
                           const int32_t *lvl_act_end, cudaStream_t s, int *launches, bool fwd, bool bwd)
{
    switch (L.sweep_lanes) {
    case 2: enqueue_sweeps_g<JVP, 2>(d, cur, n_levels, lvl_beg, lvl_act_end, s, launches, fwd, bwd); break;
    case 4: enqueue_sweeps_g<JVP, 4>(d, cur, n_levels, lvl_beg, lvl_act_end, s, launches, fwd, bwd); break;
    case 8: enqueue_sweeps_g<JVP, 8>(d, cur, n_levels, lvl_beg, lvl_act_end, s, launches, fwd, bwd); break;
    case 32:
        if (!d.pk_pt[0] || !L.pk_lw[0] || !L.lp_lg[0] || !(d.precision ? (void *)d.jcf : (void *)d.jc))
            return cudaErrorInvalidValue;
        if (JVP == 0 && !(d.precision ? (void *)d.pk_jmf[0] : (void *)d.pk_jm[0])) return cudaErrorInvalidValue;
        enqueue_sweeps_packed<JVP>(d, L, cur, n_levels, s, launches, fwd, bwd);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t enqueue_phase(const Dev &d, const Launch &L, int cur, int ph, int n_levels, const int32_t *lvl_beg,
                          const int32_t *lvl_act_end, const int32_t *lvl_end, cudaStream_t s, int *launches)
{
    switch (ph) {
    case 0:
        k_begin<<<1, 1, 0, s>>>(d.ctrl);
        (*launches)++;
        if (L.side && needs_framed_jac(d, L)) {
            // the framed points' Jacobians depend only on the state: a side
            // branch beside the q-derivatives and the residual
            cudaError_t e = cudaEventRecord(L.fork, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(L.side, L.fork, 0);
            if (e != cudaSuccess) return e;
            enqueue_framed_jac(d, cur, L.side, launches);
            e = cudaEventRecord(L.join, L.side);
            if (e != cudaSuccess) return e;
        }
        return enqueue_grad_res(d, L, cur, s, launches, true, false);
    case 1: return enqueue_grad_res(d, L, cur, s, launches, false, true);
    case 2:
        k_norm_partials<<<d.n_blk, 256, 0, s>>>(d);
        k_norm_cases<<<d.n_cases, 256, 0, s>>>(d);
        (*launches) += 2;
        return cudaGetLastError();
    case 3:
    case 4:
        if (d.scheme == 1) {  // explicit: one step kernel instead of the two sweeps
            if (ph == 3) {
                k_explicit<<<(d.n + 255) / 256, 256, 0, s>>>(d);
                (*launches)++;
            }
            return cudaGetLastError();
        }
        if (d.jvp == 0) return enqueue_sweeps<0>(d, L, cur, n_levels, lvl_beg, lvl_act_end, s, launches, ph == 3, ph == 4);
        return enqueue_sweeps<1>(d, L, cur, n_levels, lvl_beg, lvl_act_end, s, launches, ph == 3, ph == 4);
    case 5:
        k_update<<<(d.n + 255) / 256, 256, 0, s>>>(d, cur, true, true);
        (*launches)++;
        if (d.n_cases > 1) {
            k_repair<<<(d.n + 255) / 256, 256, 0, s>>>(d, cur);
            (*launches)++;
        }
        return cudaGetLastError();
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_iteration(const Dev &d, const Launch &L, int cur, int n_levels, const int32_t *lvl_beg,
                             const int32_t *lvl_act_end, const int32_t *lvl_end, cudaStream_t s, int *launches)
{
    for (int ph = 0; ph < 6; ph++) {
        cudaError_t e = enqueue_phase(d, L, cur, ph, n_levels, lvl_beg, lvl_act_end, lvl_end, s, launches);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_phase(const Dev &d, const Launch &L, int cur, int phase, int n_levels, const int32_t *lvl_beg,
                         const int32_t *lvl_act_end, const int32_t *lvl_end, cudaStream_t s)
{
    int launches = 0;
    Launch Li = L;  // one phase at a time: the framed Jacobians inline, in the forward sweep's phase
    Li.side = nullptr;
    return enqueue_phase(d, Li, cur, phase, n_levels, lvl_beg, lvl_act_end, lvl_end, s, &launches);
}

cudaError_t launch_init_state(const Dev &d, int cur, bool project, cudaStream_t s)
{
    k_update<<<(d.n + 255) / 256, 256, 0, s>>>(d, cur, false, project);
    return cudaGetLastError();
}

namespace {

// Internal order (structure of arrays [c][ld] for stride 0, else point k's
// values at stride * k; FP64 or FP32) -> caller order [p][comps] on the device.
__global__ void k_to_caller(const double *src, const float *srcf, int comps, int stride, int ld, int n,
                            const int32_t *inv, double *out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int k = inv[p];
    for (int c = 0; c < comps; c++) {
        const size_t i = stride ? (size_t)stride * k + c : (size_t)c * ld + k;
        out[(size_t)comps * p + c] = srcf ? (double)srcf[i] : src[i];
    }
}

// Caller order [p][4] -> internal structure of arrays [c][ld].
__global__ void k_from_caller(const double *in, int ld, int n, const int32_t *inv, double *U)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int k = inv[p];
#pragma unroll
    for (int c = 0; c < 4; c++) U[(size_t)c * ld + k] = in[(size_t)4 * p + c];
}

}  // namespace

cudaError_t launch_to_caller(const double *src, const float *srcf, int comps, int stride, int ld, int n,
                             const int32_t *inv, double *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_to_caller<<<(n + 255) / 256, 256, 0, s>>>(src, srcf, comps, stride, ld, n, inv, out);
    return cudaGetLastError();
}

cudaError_t launch_from_caller(const double *in, int ld, int n, const int32_t *inv, double *U, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_from_caller<<<(n + 255) / 256, 256, 0, s>>>(in, ld, n, inv, U);
    return cudaGetLastError();
}

// The integer-pipe FP64 arithmetic on the device, for the self-test entry
// (op 0: a * b by mul_i; 1: exp(a) in fixed point; 2: erfcx(|a|)/2 in fixed
// point after the kernels' clamp of |a| to 9; 3: a * b on the FP64 unit).
__global__ void __launch_bounds__(256) k_selftest_fpint(int op, const double *a, const double *b, double *out, int n)
{
    __shared__ MathTables T;
    load_math_tables(T);
    __syncthreads();
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double r;
        if (op == 0) {
            r = mul_i(a[k], b[k]);
        } else if (op == 1) {
            r = exp_t(T, a[k]);
        } else if (op == 2) {
            constexpr int kNineHi = 0x40220000;
            const int hs = __double2hiint(a[k]) & 0x7fffffff;
            const bool clamp = hs >= kNineHi;
            const int ha = clamp ? kNineHi : hs, la = clamp ? 0 : __double2loint(a[k]);
            const int iv = erfcx_interval(ha);
            r = erfcx_half_fx<kErfcxDeg>((uint32_t)ha, (uint32_t)la, iv, (const int64_t *)T.ecx[iv], T.esh[iv]);
        } else {
            r = a[k] * b[k];
        }
        out[k] = r;
    }
}

cudaError_t launch_selftest_fpint(int op, const double *a, const double *b, double *out, int n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    k_selftest_fpint<<<blocks, 256, 0, s>>>(op, a, b, out, n);
    return cudaGetLastError();
}

cudaError_t launch_init_math(cudaStream_t s)
{
    k_init_math<<<1, 256, 0, s>>>();
    return cudaGetLastError();
}

cudaError_t launch_prep_run(Ctrl *c, double target, cudaStream_t s)
{
    k_prep_run<<<1, 1, 0, s>>>(c, target);
    return cudaGetLastError();
}

cudaError_t launch_reset_ctrl(Ctrl *c, cudaStream_t s)
{
    k_reset_ctrl<<<1, 1, 0, s>>>(c);
    return cudaGetLastError();
}

}  // namespace lskum
