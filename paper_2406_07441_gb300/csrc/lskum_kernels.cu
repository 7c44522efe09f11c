// sm_103a kernels of one implicit q-LSKUM pseudo-time iteration (Alg. 1):
//   k_grad      least-squares q-derivatives, first order + K inner iterations (Eq. 10, 16)
//   k_residual  defect-corrected kinetic split-flux residual (Eq. 11-15), local time
//               step and scalar LU-SGS diagonal (Eq. 26, 33-34), density-norm partials
//   k_norm      residual norm, history and stopping test
//   k_sweep     one colour level of the forward or backward LU-SGS sweep (Eq. 27) with
//               exact (forward-mode AD) or increment (Eq. 28) Jacobian-vector products
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
// transcendental call at all; exp and A = (1 + s erf S)/2 are the kernels' own
// (lskum_fastmath.cuh), which share exp(-S^2) and keep index work off the
// FP64 pipe.
#include "lskum_internal.h"

#include <cstdint>

#include "lskum_fastmath.cuh"

namespace lskum {

namespace {

constexpr double kGm1 = 0.4;                              // gamma - 1 (gamma = 1.4)
constexpr double kInv2SqrtPi = 0.28209479177387814347;    // 1 / (2 sqrt(pi))
constexpr double kInvSqrtPi = 0.56418958354775628695;     // 1 / sqrt(pi)
constexpr unsigned kFull = 0xffffffffu;

// Every kernel returns at once after a stop or a failure.  k_norm only sets
// stop_after, so the sweeps and the update of the iteration that reached the
// drop target still run; k_begin turns it into stop at the start of the next.
__device__ __forceinline__ bool halted(const Ctrl *c)
{
    const volatile Ctrl *v = c;
    return (v->stop | v->error) != 0;
}

// Primitive state carried through the residual.
struct Prim {
    double rho, u, v, p, sb, isb, e1, e2;  // sb = sqrt(beta), isb = 1/sb,
                                           // e1 = 3.5 p + rho|u|^2/2, e2 = 3 p + rho|u|^2/2
};

// Inverse of Eq. 14: beta = -q4/2, u = q2/(2 beta), v = q3/(2 beta),
// rho = exp(q1 + beta |u|^2) beta^(-1/(gamma-1)) with 1/(gamma-1) = 5/2,
// p = rho/(2 beta).  One reciprocal square root and one exp.
__device__ __forceinline__ Prim q_to_prim(const MathTables &T, const double q[4])
{
    Prim P;
    const double beta = -0.5 * q[3];
    P.isb = rsqrt(beta);
    const double ib = P.isb * P.isb;   // 1/beta
    const double r = ib * ib * P.isb;  // beta^(-5/2)
    const double i2b = 0.5 * ib;       // 1/(2 beta)
    P.sb = beta * P.isb;
    P.u = q[1] * i2b;
    P.v = q[2] * i2b;
    const double q2 = P.u * P.u + P.v * P.v;
    P.rho = exp_t(T, fma(beta, q2, q[0])) * r;
    P.p = P.rho * i2b;
    const double k = 0.5 * P.rho * q2;
    P.e1 = fma(3.5, P.p, k);
    P.e2 = fma(3.0, P.p, k);
    return P;
}

// Kinetic split flux G_d^sg (half-range moments of the Maxwellian, sg = +-1)
// in unit direction d: DIR 0 is (1,0), DIR 1 is (0,1), DIR 2 is (dx, dy).
template <int DIR>
__device__ __forceinline__ void split_flux(const MathTables &T, const Prim &P, double dx, double dy, double sg,
                                          double G[4])
{
    const double ud = DIR == 0 ? P.u : (DIR == 1 ? P.v : P.u * dx + P.v * dy);
    const double S = ud * P.sb;
    double A, eS;
    split_A(T, S, sg, A, eS);
    const double B = eS * kInv2SqrtPi * P.isb;
    const double M1 = fma(ud, A, sg * B);
    const double rm = P.rho * M1;
    const double pA = P.p * A;
    G[0] = rm;
    if (DIR == 0) {
        G[1] = fma(rm, P.u, pA);
        G[2] = rm * P.v;
    } else if (DIR == 1) {
        G[1] = rm * P.u;
        G[2] = fma(rm, P.v, pA);
    } else {
        G[1] = fma(rm, P.u, pA * dx);
        G[2] = fma(rm, P.v, pA * dy);
    }
    G[3] = fma(ud * P.e1, A, sg * P.e2 * B);
}

// Primal quantities of a conserved state for the Jacobian products.
struct PrimU {
    double rho, irho, u, v, p, beta, sb, isb, i2p, q2, e1, e2;
};

__device__ __forceinline__ PrimU prim_from_cons(const double U[4])
{
    PrimU P;
    P.rho = U[0];
    P.irho = 1.0 / U[0];
    P.u = U[1] * P.irho;
    P.v = U[2] * P.irho;
    P.q2 = P.u * P.u + P.v * P.v;
    P.p = kGm1 * (U[3] - 0.5 * P.rho * P.q2);
    P.i2p = 0.5 / P.p;
    P.beta = P.rho * P.i2p;
    P.sb = sqrt(P.beta);
    P.isb = 1.0 / P.sb;
    const double k = 0.5 * P.rho * P.q2;
    P.e1 = 3.5 * P.p + k;
    P.e2 = 3.0 * P.p + k;
    return P;
}

__device__ __forceinline__ PrimU load_primu(const double *__restrict__ pr, int ld, int i)
{
    PrimU P;
    P.rho = pr[P_RHO * ld + i];
    P.irho = pr[P_IRHO * ld + i];
    P.u = pr[P_U * ld + i];
    P.v = pr[P_V * ld + i];
    P.p = pr[P_P * ld + i];
    P.beta = pr[P_BETA * ld + i];
    P.sb = pr[P_SB * ld + i];
    P.isb = pr[P_ISB * ld + i];
    P.i2p = pr[P_I2P * ld + i];
    P.q2 = pr[P_Q2 * ld + i];
    P.e1 = pr[P_E1 * ld + i];
    P.e2 = pr[P_E2 * ld + i];
    return P;
}

// Exact product A_d^sg(U) dl by forward-mode differentiation of
// U -> (rho, u, v, p) -> (beta, S, A, B) -> G_d^sg.  S, A = (1 + sg erf S)/2,
// exp(-S^2) and B of the state are inputs (precomputed per point for d = x, y).
__device__ __forceinline__ void jvp_exact(const PrimU &P, double dx, double dy, double sg, double S, double A,
                                          double eS, double B, const double dl[4], double out[4])
{
    const double drho = dl[0];
    const double du = (dl[1] - P.u * drho) * P.irho;
    const double dv = (dl[2] - P.v * drho) * P.irho;
    const double dq2 = 2.0 * (P.u * du + P.v * dv);
    const double dk = 0.5 * (drho * P.q2 + P.rho * dq2);  // d(rho |u|^2 / 2)
    const double dp = kGm1 * (dl[3] - dk);
    const double dbeta = (drho - 2.0 * P.beta * dp) * P.i2p;
    const double ud = P.u * dx + P.v * dy;
    const double dud = du * dx + dv * dy;
    const double dsb = 0.5 * dbeta * P.isb;
    const double dS = dud * P.sb + ud * dsb;
    const double dA = sg * eS * dS * kInvSqrtPi;
    const double dB = -B * (2.0 * S * dS + dsb * P.isb);
    const double M1 = ud * A + sg * B;
    const double dM1 = dud * A + ud * dA + sg * dB;
    const double de1 = 3.5 * dp + dk;
    const double de2 = 3.0 * dp + dk;
    const double drm = drho * M1 + P.rho * dM1;  // d(rho M1)
    const double rm = P.rho * M1;
    out[0] = drm;
    out[1] = drm * P.u + rm * du + (dp * A + P.p * dA) * dx;
    out[2] = drm * P.v + rm * dv + (dp * A + P.p * dA) * dy;
    out[3] = (dud * P.e1 + ud * de1) * A + ud * P.e1 * dA + sg * (de2 * B + P.e2 * dB);
}

__device__ __forceinline__ void flux_cons(const MathTables &T, const double U[4], double dx, double dy, double sg,
                                          double G[4])
{
    const PrimU P = prim_from_cons(U);
    const double ud = P.u * dx + P.v * dy;
    const double S = ud * P.sb;
    double A, eS;
    split_A(T, S, sg, A, eS);
    const double B = eS * kInv2SqrtPi * P.isb;
    const double M1 = fma(ud, A, sg * B);
    const double rm = P.rho * M1;
    const double pA = P.p * A;
    G[0] = rm;
    G[1] = fma(rm, P.u, pA * dx);
    G[2] = fma(rm, P.v, pA * dy);
    G[3] = fma(ud * P.e1, A, sg * P.e2 * B);
}

template <int TPP>
__device__ __forceinline__ double group_sum(double v)
{
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// q-derivatives (Eq. 10; with CORR, one Jacobi inner iteration of Eq. 16)
// ---------------------------------------------------------------------------
template <int TPP, bool CORR>
__global__ void __launch_bounds__(256) k_grad(Dev d, const double *__restrict__ q, const double *__restrict__ px,
                                              const double *__restrict__ py, double *__restrict__ qx,
                                              double *__restrict__ qy)
{
    if (halted(d.ctrl)) return;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = gt / TPP, sub = gt % TPP;
    const bool active = k < d.n;
    const int kk = active ? k : d.n - 1;
    const int ld = d.ld;
    double q0[4], px0[4], py0[4], sx[4], sy[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        q0[c] = q[c * ld + kk];
        if (CORR) {
            px0[c] = px[c * ld + kk];
            py0[c] = py[c * ld + kk];
        }
        sx[c] = 0.0;
        sy[c] = 0.0;
    }
    const int deg = d.deg[kk];
    const int base = d.slice_off[kk >> 5] + (kk & 31);
    for (int j = sub; j < deg; j += TPP) {
        const int e = base + 32 * j;
        const int i = d.nbr[e];
        const double wx = d.wgx[e], wy = d.wgy[e];
        double dx = 0.0, dy = 0.0;
        if (CORR) {
            dx = d.ndx[e];
            dy = d.ndy[e];
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
            double dq = q[c * ld + i] - q0[c];
            if (CORR) dq -= 0.5 * ((px[c * ld + i] - px0[c]) * dx + (py[c * ld + i] - py0[c]) * dy);
            sx[c] += wx * dq;
            sy[c] += wy * dq;
        }
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        sx[c] = group_sum<TPP>(sx[c]);
        sy[c] = group_sum<TPP>(sy[c]);
    }
    if (active && sub == 0) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            qx[c * ld + k] = sx[c];
            qy[c * ld + k] = sy[c];
        }
    }
}

// ---------------------------------------------------------------------------
// flux residual, time step, diagonal, norm partials
// ---------------------------------------------------------------------------
template <int TPP>
__global__ void __launch_bounds__(128) k_residual(Dev d, StateSet st, const double *__restrict__ gx,
                                                  const double *__restrict__ gy)
{
    __shared__ double red[32];
    __shared__ MathTables T;
    if (halted(d.ctrl)) return;
    load_math_tables(T);
    __syncthreads();
    const int n1 = ((const volatile Ctrl *)d.ctrl)->it + 1;
    const double cfl = (d.ramp > 0.0 && (double)n1 < d.ramp) ? d.cfl * ((double)n1 / d.ramp) : d.cfl;
    const double hc = n1 <= d.first_order ? 0.0 : 0.5;  // first-order start: q~ = q
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = gt / TPP, sub = gt % TPP;
    const bool active = k < d.n;
    const int kk = active ? k : d.n - 1;
    const int ld = d.ld;
    const int fl = d.flag[kk];
    const bool work = active && fl != kOuter;
    const bool wall = fl == kWall;
    const double *__restrict__ q = st.q;
    double R[4] = {0.0, 0.0, 0.0, 0.0};
    const double e1x = d.geo[G_E1X * ld + kk], e1y = d.geo[G_E1Y * ld + kk];
    const double e2x = d.geo[G_E2X * ld + kk], e2y = d.geo[G_E2Y * ld + kk];
    if (work) {
        double q0[4], gx0[4], gy0[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            q0[c] = q[c * ld + kk];
            gx0[c] = gx[c * ld + kk];
            gy0[c] = gy[c * ld + kk];
        }
        const int deg = d.deg[kk];
        const int base = d.slice_off[kk >> 5] + (kk & 31);
        for (int j = sub; j < deg; j += TPP) {
            const int e = base + 32 * j;
            const int mb = d.memb[e];
            if (!mb) continue;
            const int i = d.nbr[e];
            const double dx = d.ndx[e], dy = d.ndy[e];
            double qi[4], q0t[4];
#pragma unroll
            for (int c = 0; c < 4; c++) {
                qi[c] = q[c * ld + i] - hc * (dx * gx[c * ld + i] + dy * gy[c * ld + i]);
                q0t[c] = q0[c] - hc * (dx * gx0[c] + dy * gy0[c]);
            }
            const Prim Pi = q_to_prim(T, qi);
            const Prim P0 = q_to_prim(T, q0t);
            if (mb & 3) {
                const double sg = (mb & 1) ? 1.0 : -1.0;
                const double w = d.w1[e];
                double Gi[4], G0[4];
                if (wall) {
                    split_flux<2>(T, Pi, e1x, e1y, sg, Gi);
                    split_flux<2>(T, P0, e1x, e1y, sg, G0);
                } else {
                    split_flux<0>(T, Pi, 1.0, 0.0, sg, Gi);
                    split_flux<0>(T, P0, 1.0, 0.0, sg, G0);
                }
#pragma unroll
                for (int c = 0; c < 4; c++) R[c] = fma(w, Gi[c] - G0[c], R[c]);
            }
            if (mb & 12) {
                const double sg = (mb & 4) ? 1.0 : -1.0;
                const double w = d.w2[e];
                double Gi[4], G0[4];
                if (wall) {
                    split_flux<2>(T, Pi, e2x, e2y, sg, Gi);
                    split_flux<2>(T, P0, e2x, e2y, sg, G0);
                } else {
                    split_flux<1>(T, Pi, 0.0, 1.0, sg, Gi);
                    split_flux<1>(T, P0, 0.0, 1.0, sg, G0);
                }
#pragma unroll
                for (int c = 0; c < 4; c++) R[c] = fma(w, Gi[c] - G0[c], R[c]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 4; c++) R[c] = group_sum<TPP>(R[c]);
    double nrm = 0.0;
    if (work && sub == 0) {
#pragma unroll
        for (int c = 0; c < 4; c++) d.R[c * ld + k] = R[c];
        nrm = R[0] * R[0];
        // local time step (reading: CFL min_i|dr| / (|u| + a)) and the scalar
        // diagonal of Eq. 26 with the spectral radii of Eq. 34, kept at least
        // sum_s rho_s sum_i |w_i| so that it bounds the off-diagonal blocks
        const double *pr = st.prim;
        const double rho = pr[P_RHO * ld + k], u = pr[P_U * ld + k], v = pr[P_V * ld + k];
        const double p = pr[P_P * ld + k];
        const double a = sqrt(1.4 * p * pr[P_IRHO * ld + k]);
        const double dt = cfl * d.geo[G_DMIN * ld + k] / (sqrt(u * u + v * v) + a);
        (void)rho;
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
        d.D[k] = Dp > Ddom ? Dp : Ddom;
    }
    // block partial of sum R_rho^2 (fixed order: warp butterfly, then warp 0)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(kFull, nrm, o);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[wid] = nrm;
    __syncthreads();
    if (wid == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
        if (lane == 0) d.blk[blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// residual norm, history, stopping test (one block)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_norm(Dev d)
{
    __shared__ double red[32];
    if (halted(d.ctrl)) return;
    double t = 0.0;
    for (int b = threadIdx.x; b < d.n_blk; b += blockDim.x) t += d.blk[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[wid] = t;
    __syncthreads();
    if (wid == 0) {
        double s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (lane == 0) {
            Ctrl *c = d.ctrl;
            const double nrm = sqrt(s);
            const int n = c->it;
            if (n < c->hist_cap) c->hist[n] = nrm;
            if (!(c->hist0 > 0.0)) c->hist0 = nrm;
            c->it = n + 1;
            if (!isfinite(nrm)) {
                c->error = -4;  // LSKUM_ERR_DIVERGED
            } else if (c->target > 0.0 && nrm / c->hist0 <= c->target) {
                c->stop_after = 1;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// LU-SGS sweep, one colour level; one warp per point
// ---------------------------------------------------------------------------
// Points [lb, le) of the level (outer points excluded); [cb_lo, cb_hi) is the
// whole colour block: a neighbour i is "lower" (earlier in the sweep order)
// iff i < cb_lo and "upper" iff i >= cb_hi.
template <int JVP, bool FWD>
__global__ void __launch_bounds__(256) k_sweep(Dev d, StateSet st, int lb, int le, int cb_lo, int cb_hi)
{
    __shared__ MathTables T;
    if (halted(d.ctrl)) return;
    load_math_tables(T);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int k = lb + (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (k >= le) return;  // warp-uniform
    const int ld = d.ld;
    const double *__restrict__ dW = FWD ? d.dUs : d.dU;
    const double *__restrict__ pr = st.prim;
    const bool wall = d.flag[k] == kWall;
    const double e1x = d.geo[G_E1X * ld + k], e1y = d.geo[G_E1Y * ld + k];
    const double e2x = d.geo[G_E2X * ld + k], e2y = d.geo[G_E2Y * ld + k];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int deg = d.deg[k];
    const int base = d.slice_off[k >> 5] + (k & 31);
    for (int j = lane; j < deg; j += 32) {
        const int e = base + 32 * j;
        const int i = d.nbr[e];
        const int mb = d.memb[e];
        const bool side = FWD ? (i < cb_lo) : (i >= cb_hi);
        if (!side || !mb) continue;
        double dl[4];
#pragma unroll
        for (int c = 0; c < 4; c++) dl[c] = dW[c * ld + i];
        double J[4];
        if (JVP == 0) {
            const PrimU P = load_primu(pr, ld, i);
#pragma unroll
            for (int s = 0; s < 2; s++) {
                const int m = s == 0 ? (mb & 3) : (mb >> 2);
                if (!m) continue;
                const double sg = (m & 1) ? 1.0 : -1.0;
                const double w = s == 0 ? d.w1[e] : d.w2[e];
                const double ddx = s == 0 ? e1x : e2x, ddy = s == 0 ? e1y : e2y;
                double S, A, eS, B;
                if (!wall) {
                    // interior frame: d = (1,0) or (0,1), precomputed per point
                    const int f = s == 0 ? P_SX : P_SY;
                    S = pr[f * ld + i];
                    A = pr[(sg > 0.0 ? f + 1 : f + 2) * ld + i];
                    eS = pr[(f + 3) * ld + i];
                    B = pr[(f + 4) * ld + i];
                } else {
                    S = (P.u * ddx + P.v * ddy) * P.sb;
                    split_A(T, S, sg, A, eS);
                    B = eS * kInv2SqrtPi * P.isb;
                }
                jvp_exact(P, ddx, ddy, sg, S, A, eS, B, dl, J);
#pragma unroll
                for (int c = 0; c < 4; c++) acc[c] += w * J[c];
            }
        } else {
            double Ui[4], Up[4];
#pragma unroll
            for (int c = 0; c < 4; c++) {
                Ui[c] = st.U[c * ld + i];
                Up[c] = Ui[c] + dl[c];
            }
#pragma unroll
            for (int s = 0; s < 2; s++) {
                const int m = s == 0 ? (mb & 3) : (mb >> 2);
                if (!m) continue;
                const double sg = (m & 1) ? 1.0 : -1.0;
                const double w = s == 0 ? d.w1[e] : d.w2[e];
                const double ddx = s == 0 ? e1x : e2x, ddy = s == 0 ? e1y : e2y;
                double G1[4], G0[4];
                flux_cons(T, Up, ddx, ddy, sg, G1);
                flux_cons(T, Ui, ddx, ddy, sg, G0);
#pragma unroll
                for (int c = 0; c < 4; c++) acc[c] += w * (G1[c] - G0[c]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(kFull, acc[c], o);
    }
    if (lane == 0) {
        const double Dk = d.D[k];
        double w[4];
        if (FWD) {
#pragma unroll
            for (int c = 0; c < 4; c++) w[c] = -(d.R[c * ld + k] + acc[c]) / Dk;
        } else {
#pragma unroll
            for (int c = 0; c < 4; c++) w[c] = d.dUs[c * ld + k] - acc[c] / Dk;
        }
        if (wall) {
            const double nx = d.wnx[k], ny = d.wny[k];
            const double mn = w[1] * nx + w[2] * ny;
            w[1] -= mn * nx;
            w[2] -= mn * ny;
        }
        double *out = FWD ? d.dUs : d.dU;
#pragma unroll
        for (int c = 0; c < 4; c++) out[c * ld + k] = w[c];
    }
}

// ---------------------------------------------------------------------------
// state update (set cur -> set 1-cur) and per-point quantities of the new state
// ---------------------------------------------------------------------------
__global__ void k_begin(Ctrl *c)
{
    if (c->stop_after) c->stop = 1;
}

template <bool INC>
__global__ void __launch_bounds__(256) k_update(Dev d, int cur)
{
    __shared__ MathTables T;
    if (INC && halted(d.ctrl)) return;
    load_math_tables(T);
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    const int ld = d.ld;
    const StateSet src = d.set[cur];
    const StateSet dst = d.set[INC ? 1 - cur : cur];
    const int fl = d.flag[k];
    double U[4];
#pragma unroll
    for (int c = 0; c < 4; c++) U[c] = src.U[c * ld + k];
    if (INC && fl != kOuter) {
#pragma unroll
        for (int c = 0; c < 4; c++) U[c] += d.dU[c * ld + k];
    }
    if (fl == kWall) {
        const double nx = d.wnx[k], ny = d.wny[k];
        const double mn = U[1] * nx + U[2] * ny;
        U[1] -= mn * nx;
        U[2] -= mn * ny;
    }
    const PrimU P = prim_from_cons(U);
    const bool ok = P.rho > 0.0 && P.p > 0.0 && isfinite(P.rho) && isfinite(P.p) && isfinite(P.u) &&
                    isfinite(P.v);
    if (!ok) {
        atomicMin(&d.ctrl->bad_point, k);
        atomicExch(&d.ctrl->error, -3);  // LSKUM_ERR_NONPOSITIVE
        return;
    }
#pragma unroll
    for (int c = 0; c < 4; c++) dst.U[c * ld + k] = U[c];
    dst.q[0 * ld + k] = log(P.rho) + 2.5 * log(P.beta) - P.beta * P.q2;
    dst.q[1 * ld + k] = 2.0 * P.beta * P.u;
    dst.q[2 * ld + k] = 2.0 * P.beta * P.v;
    dst.q[3 * ld + k] = -2.0 * P.beta;
    double *pr = dst.prim;
    pr[P_RHO * ld + k] = P.rho;
    pr[P_IRHO * ld + k] = P.irho;
    pr[P_U * ld + k] = P.u;
    pr[P_V * ld + k] = P.v;
    pr[P_P * ld + k] = P.p;
    pr[P_BETA * ld + k] = P.beta;
    pr[P_SB * ld + k] = P.sb;
    pr[P_ISB * ld + k] = P.isb;
    pr[P_I2P * ld + k] = P.i2p;
    pr[P_Q2 * ld + k] = P.q2;
    pr[P_E1 * ld + k] = P.e1;
    pr[P_E2 * ld + k] = P.e2;
    const double sx = P.u * P.sb, sy = P.v * P.sb;
    double Ex, ex, Ey, ey;
    split_E(T, sx, Ex, ex);
    split_E(T, sy, Ey, ey);
    pr[P_SX * ld + k] = sx;
    pr[P_APX * ld + k] = sx >= 0.0 ? 1.0 - Ex : Ex;
    pr[P_AMX * ld + k] = sx >= 0.0 ? Ex : 1.0 - Ex;
    pr[P_EXPX * ld + k] = ex;
    pr[P_BX * ld + k] = ex * kInv2SqrtPi * P.isb;
    pr[P_SY * ld + k] = sy;
    pr[P_APY * ld + k] = sy >= 0.0 ? 1.0 - Ey : Ey;
    pr[P_AMY * ld + k] = sy >= 0.0 ? Ey : 1.0 - Ey;
    pr[P_EXPY * ld + k] = ey;
    pr[P_BY * ld + k] = ey * kInv2SqrtPi * P.isb;
}

__global__ void k_reset_ctrl(Ctrl *c)
{
    c->stop = 0;
    c->stop_after = 0;
    c->error = 0;
    c->bad_point = 0x7fffffff;
}

template <int TPP>
cudaError_t enqueue_grad(const Dev &d, int cur, cudaStream_t s, int *launches)
{
    const int gb = (d.n * TPP + 255) / 256;
    const StateSet st = d.set[cur];
    k_grad<TPP, false><<<gb, 256, 0, s>>>(d, st.q, nullptr, nullptr, d.qx[0], d.qy[0]);
    (*launches)++;
    for (int it = 1; it <= d.K; it++) {
        const int a = (it - 1) & 1, b = it & 1;
        k_grad<TPP, true><<<gb, 256, 0, s>>>(d, st.q, d.qx[a], d.qy[a], d.qx[b], d.qy[b]);
        (*launches)++;
    }
    return cudaGetLastError();
}

template <int TPP>
cudaError_t enqueue_res(const Dev &d, const Launch &L, int cur, cudaStream_t s, int *launches)
{
    const int fin = d.K & 1;
    const int rb = (d.n * TPP + L.res_block - 1) / L.res_block;
    k_residual<TPP><<<rb, L.res_block, 0, s>>>(d, d.set[cur], d.qx[fin], d.qy[fin]);
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

template <int JVP>
void enqueue_sweeps(const Dev &d, int cur, int n_levels, const int32_t *lvl_beg, const int32_t *lvl_act_end,
                    const int32_t *lvl_end, cudaStream_t s, int *launches, bool fwd, bool bwd)
{
    const StateSet st = d.set[cur];
    for (int l = 0; fwd && l < n_levels; l++) {
        const int np = lvl_act_end[l] - lvl_beg[l];
        if (np <= 0) continue;
        const int blocks = (np * 32 + 255) / 256;
        k_sweep<JVP, true><<<blocks, 256, 0, s>>>(d, st, lvl_beg[l], lvl_act_end[l], lvl_beg[l], lvl_end[l]);
        (*launches)++;
    }
    for (int l = n_levels - 1; bwd && l >= 0; l--) {
        const int np = lvl_act_end[l] - lvl_beg[l];
        if (np <= 0) continue;
        const int blocks = (np * 32 + 255) / 256;
        k_sweep<JVP, false><<<blocks, 256, 0, s>>>(d, st, lvl_beg[l], lvl_act_end[l], lvl_beg[l], lvl_end[l]);
        (*launches)++;
    }
}

cudaError_t enqueue_phase(const Dev &d, const Launch &L, int cur, int ph, int n_levels, const int32_t *lvl_beg,
                          const int32_t *lvl_act_end, const int32_t *lvl_end, cudaStream_t s, int *launches)
{
    switch (ph) {
    case 0:
        k_begin<<<1, 1, 0, s>>>(d.ctrl);
        (*launches)++;
        return enqueue_grad_res(d, L, cur, s, launches, true, false);
    case 1: return enqueue_grad_res(d, L, cur, s, launches, false, true);
    case 2:
        k_norm<<<1, 1024, 0, s>>>(d);
        (*launches)++;
        return cudaGetLastError();
    case 3:
    case 4:
        if (d.jvp == 0) enqueue_sweeps<0>(d, cur, n_levels, lvl_beg, lvl_act_end, lvl_end, s, launches, ph == 3, ph == 4);
        else enqueue_sweeps<1>(d, cur, n_levels, lvl_beg, lvl_act_end, lvl_end, s, launches, ph == 3, ph == 4);
        return cudaGetLastError();
    case 5:
        k_update<true><<<(d.n + 255) / 256, 256, 0, s>>>(d, cur);
        (*launches)++;
        return cudaGetLastError();
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int residual_blocks(const Dev &d, const Launch &L)
{
    return (d.n * L.tpp + L.res_block - 1) / L.res_block;
}

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
    return enqueue_phase(d, L, cur, phase, n_levels, lvl_beg, lvl_act_end, lvl_end, s, &launches);
}

cudaError_t launch_init_state(const Dev &d, int cur, cudaStream_t s)
{
    k_update<false><<<(d.n + 255) / 256, 256, 0, s>>>(d, cur);
    return cudaGetLastError();
}

cudaError_t launch_reset_ctrl(Ctrl *c, cudaStream_t s)
{
    k_reset_ctrl<<<1, 1, 0, s>>>(c);
    return cudaGetLastError();
}

}  // namespace lskum
