/*
 * Plain FP64 CPU oracle for one pseudo-time iteration of the implicit q-LSKUM
 * 2D Euler solver with the modified (AD) LU-SGS scheme of Verma, Mamidi and
 * Nemili, "GPU Accelerated Implicit Kinetic Meshfree Method based on Modified
 * LU-SGS" (2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * Everything is written the slow, obvious way: array-of-structures state
 * (U[4*p + k]), one point at a time, sums in neighbour order, libm elementary
 * functions, no fused multiply-add (built with -ffp-contract=off).
 *
 * Where the paper is silent the oracle takes these readings (each one is also
 * listed in the design notes):
 *   R1  gamma = 1.4 (the Gx listing of Appendix A hard-codes gamma-1 = 0.4);
 *       free stream rho = 1, p = 1/gamma (sound speed 1), u = M cos(aoa),
 *       v = M sin(aoa).
 *   R2  Kinetic split fluxes: half-range Psi-moments of the Maxwellian of Eq. 4
 *       (the paper cites KFVS but never prints them), in any unit direction d.
 *   R3  Split stencils (Eq. 13): N_d^+ = {Delta_d < 0}, N_d^- = {Delta_d > 0};
 *       a neighbour with Delta_d exactly 0 is in neither.
 *   R4  Wall points use the local frame (t, n), n the unit normal into the
 *       fluid and t = (n_y, -n_x); their residual is the sum of the t+, t- and
 *       n- split derivatives (molecules leaving the wall carry no separate
 *       term), and non-penetration is imposed on the increments and the state
 *       by removing the normal momentum (P(m) = m - (m.n) n).
 *   R5  q-derivative inner iterations (Eq. 16) are Jacobi sweeps from the
 *       first-order least-squares gradient; their count K is an option.
 *   R6  Local time step dt_0 = CFL min_i |r_i - r_0| / (|u_0| + a_0), shortened
 *       where needed so that D_0 >= sum_s rho_s sum_{i in s} |w_i| (w_i the LS
 *       weights of Eq. 11): with mixed-sign weights the scalar diagonal of
 *       Eq. 26 alone does not bound the off-diagonal blocks at large CFL.
 *       The time step does not enter the fixed point R = 0.
 *   R7  Eq. 34 read as rho(A+) = max(u_d + a, 0), rho(A-) = max(a - u_d, 0).
 *   R8  Sweep order: greedy colouring (Alg. 5) on the symmetrised neighbour
 *       graph, points stably sorted by colour; "i < 0" in Eq. 20-27 means
 *       "earlier in that order".  Outer (far-field) points are frozen at the
 *       free stream and skipped by the sweeps (their increments are 0).
 *   R9  Residual norm: sqrt of the sum of the squared density residual over
 *       wall and interior points; drop = norm_n / norm_1.
 *   R10 Cl, Cd: pressure integrated over the wall polygon (wall points in
 *       index order), each wall point carrying the sum of its two rotated half
 *       edges as n ds.
 *   R11 Start-up: the first `first_order` iterations (an option, 0 = none)
 *       use the first-order residual (q~ = q, no defect correction); the
 *       impulsive free-stream start otherwise drives the unlimited second-order
 *       reconstruction out of the Maxwellian range (q~_4 >= 0) at the
 *       leading edge of jittered clouds.
 *   R12 Kinetic far field (an option; the paper's sweeps visit outer points,
 *       Alg. 2 and 4, but it states no outer-boundary formula).  Outer points
 *       are then unknowns like the others, in the local frame (t, n), n the
 *       unit normal out of the domain and t = (n_y, -n_x).  Their residual is
 *       the sum of the t+, t- and n+ split derivatives over their (inside)
 *       neighbours, plus the n- derivative against ghost points that hold
 *       the free stream at the mirror images of the n+ neighbours across the
 *       tangent line: molecules entering the domain carry the free-stream
 *       Maxwellian.  Mirroring negates the n-derivative weights, so that term
 *       is LS_3(1) (G_n^-(U_inf) - G_n^-(U_0)) with LS_3(1) = -LS_2(1) and
 *       sum |w| equal to that of the n+ stencil; it is first order (the
 *       point's own conserved state, no defect correction).  On a 1D stencil
 *       it is the upwind difference against a free-stream ghost cell.  The
 *       sweeps, the update (no projection) and the norm then include outer
 *       points.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 1.4
#define GM1 0.4 /* gamma - 1 */

enum { PT_INTERIOR = 0, PT_WALL = 1, PT_OUTER = 2 };
enum { JVP_EXACT = 0, JVP_INCREMENT = 1 };

/* ------------------------------------------------------------------------- */
/* O1: primitive <-> conserved <-> q (Eq. 2, Eq. 14)                          */
/* ------------------------------------------------------------------------- */

void o_prim_to_cons(double rho, double u, double v, double p, double *U)
{
    U[0] = rho;
    U[1] = rho * u;
    U[2] = rho * v;
    U[3] = p / GM1 + 0.5 * rho * (u * u + v * v);
}

void o_cons_to_prim(const double *U, double *rho, double *u, double *v, double *p)
{
    *rho = U[0];
    *u = U[1] / U[0];
    *v = U[2] / U[0];
    *p = GM1 * (U[3] - 0.5 * U[0] * ((*u) * (*u) + (*v) * (*v)));
}

/* Eq. 14: q = [ln rho + ln(beta)/(gamma-1) - beta |u|^2, 2 beta u1, 2 beta u2, -2 beta] */
void o_prim_to_q(double rho, double u, double v, double p, double *q)
{
    double beta = rho / (2.0 * p);
    q[0] = log(rho) + log(beta) / GM1 - beta * (u * u + v * v);
    q[1] = 2.0 * beta * u;
    q[2] = 2.0 * beta * v;
    q[3] = -2.0 * beta;
}

/* Inverse of Eq. 14. */
void o_q_to_prim(const double *q, double *rho, double *u, double *v, double *p, double *beta)
{
    double b = -0.5 * q[3];
    *beta = b;
    *u = q[1] / (2.0 * b);
    *v = q[2] / (2.0 * b);
    *rho = exp(q[0] - log(b) / GM1 + b * ((*u) * (*u) + (*v) * (*v)));
    *p = (*rho) / (2.0 * b);
}

/* ------------------------------------------------------------------------- */
/* O2: Euler flux (Eq. 2) and kinetic split fluxes (reading R2)              */
/* ------------------------------------------------------------------------- */

/* Euler flux in unit direction d: G = [rho u_d, rho u u_d + p d, (rho e + p) u_d]. */
void o_euler_flux(double rho, double u, double v, double p, double dx, double dy, double *G)
{
    double ud = u * dx + v * dy;
    double rhoE = p / GM1 + 0.5 * rho * (u * u + v * v);
    G[0] = rho * ud;
    G[1] = rho * u * ud + p * dx;
    G[2] = rho * v * ud + p * dy;
    G[3] = (rhoE + p) * ud;
}

/*
 * Split flux G_d^sign: the Psi-moments of v_d F over the half range
 * sign * v_d > 0, F the Maxwellian of Eq. 4.  With beta = rho / 2p,
 * S = u_d sqrt(beta), A = (1 + sign erf S) / 2, B = exp(-S^2) / (2 sqrt(pi beta)):
 *   mass      rho (u_d A + sign B)
 *   momentum  rho u (u_d A + sign B) + p d A
 *   energy    u_d (gamma/(gamma-1) p + rho|u|^2/2) A
 *             + sign ((gamma+1)/(2(gamma-1)) p + rho|u|^2/2) B
 */
void o_split_flux(double rho, double u, double v, double p, double beta,
                  double dx, double dy, int sign, double *G)
{
    double sg = (double)sign;
    double ud = u * dx + v * dy;
    double S = ud * sqrt(beta);
    double A = 0.5 * (1.0 + sg * erf(S));
    double B = exp(-S * S) / (2.0 * sqrt(M_PI * beta));
    double M1 = ud * A + sg * B;
    double q2 = u * u + v * v;
    G[0] = rho * M1;
    G[1] = rho * u * M1 + p * dx * A;
    G[2] = rho * v * M1 + p * dy * A;
    G[3] = ud * (GAMMA / GM1 * p + 0.5 * rho * q2) * A
         + sg * ((GAMMA + 1.0) / (2.0 * GM1) * p + 0.5 * rho * q2) * B;
}

/* Split flux of a conserved state (used by the sweeps' Jacobian products). */
void o_split_flux_cons(const double *U, double dx, double dy, int sign, double *G)
{
    double rho, u, v, p;
    o_cons_to_prim(U, &rho, &u, &v, &p);
    o_split_flux(rho, u, v, p, rho / (2.0 * p), dx, dy, sign, G);
}

/* ------------------------------------------------------------------------- */
/* O8: split-flux Jacobian-vector products                                    */
/* ------------------------------------------------------------------------- */

/*
 * Exact product A_d^sign(U) dU by forward-mode differentiation of the chain
 * U -> (rho, u, v, p) -> (beta, S, A, B) -> G_d^sign (Sec. 3: one erf per
 * product).  Each primal quantity carries its tangent (prefix d).
 */
void o_split_jvp_exact(const double *U, const double *dUin, double dx, double dy, int sign, double *out)
{
    double sg = (double)sign;
    double rho = U[0], drho = dUin[0];
    double u = U[1] / rho, du = (dUin[1] - u * drho) / rho;
    double v = U[2] / rho, dv = (dUin[2] - v * drho) / rho;
    double q2 = u * u + v * v, dq2 = 2.0 * u * du + 2.0 * v * dv;
    double p = GM1 * (U[3] - 0.5 * rho * q2);
    double dp = GM1 * (dUin[3] - 0.5 * (drho * q2 + rho * dq2));
    double beta = rho / (2.0 * p);
    double dbeta = (drho - 2.0 * beta * dp) / (2.0 * p);
    double ud = u * dx + v * dy, dud = du * dx + dv * dy;
    double sb = sqrt(beta), dsb = dbeta / (2.0 * sb);
    double S = ud * sb, dS = dud * sb + ud * dsb;
    double eS = exp(-S * S);
    double A = 0.5 * (1.0 + sg * erf(S));
    double dA = sg * eS * dS / sqrt(M_PI);
    double B = eS / (2.0 * sqrt(M_PI) * sb);
    double dB = B * (-2.0 * S * dS) - B * dsb / sb;
    double M1 = ud * A + sg * B;
    double dM1 = dud * A + ud * dA + sg * dB;
    double E1 = GAMMA / GM1 * p + 0.5 * rho * q2;
    double dE1 = GAMMA / GM1 * dp + 0.5 * (drho * q2 + rho * dq2);
    double E2 = (GAMMA + 1.0) / (2.0 * GM1) * p + 0.5 * rho * q2;
    double dE2 = (GAMMA + 1.0) / (2.0 * GM1) * dp + 0.5 * (drho * q2 + rho * dq2);
    out[0] = drho * M1 + rho * dM1;
    out[1] = (drho * u + rho * du) * M1 + rho * u * dM1 + dp * dx * A + p * dx * dA;
    out[2] = (drho * v + rho * dv) * M1 + rho * v * dM1 + dp * dy * A + p * dy * dA;
    out[3] = (dud * E1 + ud * dE1) * A + ud * E1 * dA + sg * (dE2 * B + E2 * dB);
}

/* Eq. 28: A_d^sign dU ~ G_d^sign(U + dU) - G_d^sign(U). */
void o_split_jvp_increment(const double *U, const double *dUin, double dx, double dy, int sign, double *out)
{
    double Up[4], G1[4], G0[4];
    for (int k = 0; k < 4; k++) Up[k] = U[k] + dUin[k];
    o_split_flux_cons(Up, dx, dy, sign, G1);
    o_split_flux_cons(U, dx, dy, sign, G0);
    for (int k = 0; k < 4; k++) out[k] = G1[k] - G0[k];
}

/* ------------------------------------------------------------------------- */
/* Cloud, split stencils and frames                                           */
/* ------------------------------------------------------------------------- */

/* farfield: 0 = outer points frozen at the free stream (R8); 1 = the kinetic
 * far field (R12), with uinf the free-stream conserved state and (nx, ny) the
 * outward unit normals at outer points. */
typedef struct {
    int32_t n;
    const double *x, *y;
    const uint8_t *flag;
    const double *nx, *ny;
    const int32_t *off, *idx;
    int32_t farfield;
    double uinf[4];
} o_cloud;

/* Is point p an unknown of the iteration?  (Outer points only with R12.) */
static int is_active(const o_cloud *c, int p)
{
    return c->flag[p] != PT_OUTER || c->farfield == 1;
}

/* Stencil kind: 0 interior, 1 wall, 2 outer under the kinetic far field. */
static int kind_of(const o_cloud *c, int p)
{
    if (c->flag[p] == PT_WALL) return 1;
    if (c->flag[p] == PT_OUTER && c->farfield == 1) return 2;
    return 0;
}

/* Frame of point p: e1 = (1,0), e2 = (0,1) in the interior; (t, n) at the
 * wall (n into the fluid) and at kinetic outer points (n out of the domain). */
static void frame(const o_cloud *c, int p, double *e1x, double *e1y, double *e2x, double *e2y)
{
    if (kind_of(c, p) != 0) {
        *e1x = c->ny[p]; *e1y = -c->nx[p];
        *e2x = c->nx[p]; *e2y = c->ny[p];
    } else {
        *e1x = 1.0; *e1y = 0.0;
        *e2x = 0.0; *e2y = 1.0;
    }
}

/*
 * Split sub-stencils of a point, in a fixed order:
 *   interior: 0 = e1+ (a<0), 1 = e1- (a>0), 2 = e2+ (b<0), 3 = e2- (b>0)
 *   wall:     0 = t+  (a<0), 1 = t-  (a>0),                 3 = n-  (b>0)
 *   outer:    0 = t+  (a<0), 1 = t-  (a>0), 2 = n+  (b<0)   (3: the ghosts, R12)
 * a = Delta r . e1, b = Delta r . e2.  member() returns, for neighbour
 * offsets (a, b), the sub-stencils it joins (at most one per direction).
 */
static int members(int kind, double a, double b, int *s)
{
    int m = 0;
    if (a < 0.0) s[m++] = 0;
    else if (a > 0.0) s[m++] = 1;
    if (b < 0.0) { if (kind != 1) s[m++] = 2; }
    else if (b > 0.0) { if (kind != 2) s[m++] = 3; }
    return m;
}

/* Is sub-stencil s formed from the point's neighbours? */
static int real_sub(int kind, int s)
{
    return !((kind == 1 && s == 2) || (kind == 2 && s == 3));
}

static const int SUB_SIGN[4] = { +1, -1, +1, -1 };

/* The direction of sub-stencil s is e1 for s = 0, 1 and e2 for s = 2, 3;
 * for each member, d = offset along that direction, dp = offset along the
 * other one. */
static void sub_offsets(int s, double a, double b, double *d, double *dp)
{
    if (s < 2) { *d = a; *dp = b; }
    else { *d = b; *dp = a; }
}

/* ------------------------------------------------------------------------- */
/* a0: colouring (Alg. 5) and the canonical order (reading R8)               */
/* ------------------------------------------------------------------------- */

/*
 * Symmetrised adjacency: each point's own stencil in the given order,
 * followed by the points that list it but are not in its stencil, ascending.
 * Colours start at 1; out: colour[N], order[N] (point at each position),
 * rank[N] (position of each point).  Returns the number of colours, or -1.
 */
int o_color_order(int32_t n, const int32_t *off, const int32_t *idx,
                  int32_t *colour, int32_t *order, int32_t *rank)
{
    int64_t nnz = off[n];
    int32_t *cnt = calloc((size_t)n + 1, sizeof(int32_t));
    if (!cnt) return -1;
    /* reverse-only neighbours: for each edge p -> q with p not in stencil(q) */
    int32_t *roff = calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *ridx = malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    for (int32_t p = 0; p < n; p++)
        for (int32_t e = off[p]; e < off[p + 1]; e++) {
            int32_t q = idx[e], found = 0;
            for (int32_t f = off[q]; f < off[q + 1]; f++) if (idx[f] == p) { found = 1; break; }
            if (!found) roff[q + 1]++;
        }
    for (int32_t p = 0; p < n; p++) roff[p + 1] += roff[p];
    int32_t *fill = calloc((size_t)n, sizeof(int32_t));
    /* p ascending, so each list comes out ascending */
    for (int32_t p = 0; p < n; p++)
        for (int32_t e = off[p]; e < off[p + 1]; e++) {
            int32_t q = idx[e], found = 0;
            for (int32_t f = off[q]; f < off[q + 1]; f++) if (idx[f] == p) { found = 1; break; }
            if (!found) ridx[roff[q] + fill[q]++] = p;
        }
    for (int32_t p = 0; p < n; p++) colour[p] = 0;
    int ncol = 0;
    int32_t maxdeg = 0;
    for (int32_t p = 0; p < n; p++) {
        int32_t d = (off[p + 1] - off[p]) + (roff[p + 1] - roff[p]);
        if (d > maxdeg) maxdeg = d;
    }
    char *used = calloc((size_t)maxdeg + 2, 1);
#define SMALLEST_FREE(P, OUT)                                                  \
    do {                                                                       \
        memset(used, 0, (size_t)maxdeg + 2);                                   \
        for (int32_t f = off[P]; f < off[(P) + 1]; f++) {                      \
            int32_t cc = colour[idx[f]];                                       \
            if (cc <= maxdeg + 1) used[cc] = 1;                                \
        }                                                                      \
        for (int32_t f = roff[P]; f < roff[(P) + 1]; f++) {                    \
            int32_t cc = colour[ridx[f]];                                      \
            if (cc <= maxdeg + 1) used[cc] = 1;                                \
        }                                                                      \
        int32_t k = 1;                                                         \
        while (used[k]) k++;                                                   \
        (OUT) = k;                                                             \
    } while (0)
    if (n > 0) colour[0] = 1;
    for (int32_t i = 0; i < n; i++) {
        if (colour[i] == 0) SMALLEST_FREE(i, colour[i]);
        for (int32_t f = off[i]; f < off[i + 1]; f++) {
            int32_t p = idx[f];
            if (colour[p] == 0) SMALLEST_FREE(p, colour[p]);
        }
        for (int32_t f = roff[i]; f < roff[i + 1]; f++) {
            int32_t p = ridx[f];
            if (colour[p] == 0) SMALLEST_FREE(p, colour[p]);
        }
    }
#undef SMALLEST_FREE
    for (int32_t p = 0; p < n; p++) if (colour[p] > ncol) ncol = colour[p];
    /* stable sort by colour */
    int32_t pos = 0;
    for (int c = 1; c <= ncol; c++)
        for (int32_t p = 0; p < n; p++)
            if (colour[p] == c) { order[pos] = p; rank[p] = pos; pos++; }
    free(cnt); free(roff); free(ridx); free(fill); free(used);
    return ncol;
}

/* ------------------------------------------------------------------------- */
/* O5: q-derivatives by least squares with defect-correction inner iterations */
/* ------------------------------------------------------------------------- */

/* One pass of Eq. 16: least-squares gradients of q with
 * Delta q~_i = Delta q_i - (Delta x_i (px_i - px_0) + Delta y_i (py_i - py_0)) / 2
 * built from the previous iterate (px, py); with px = py = NULL the plain
 * first-order differences Delta q_i are used (Eq. 10).  q, px, py, qx, qy: [4N]. */
void o_q_gradient_pass(const o_cloud *c, const double *q, const double *px, const double *py,
                       double *qx, double *qy)
{
    for (int32_t p = 0; p < c->n; p++) {
        double sxx = 0.0, syy = 0.0, sxy = 0.0;
        double sx[4] = { 0, 0, 0, 0 }, sy[4] = { 0, 0, 0, 0 };
        for (int32_t e = c->off[p]; e < c->off[p + 1]; e++) {
            int32_t i = c->idx[e];
            double dx = c->x[i] - c->x[p];
            double dy = c->y[i] - c->y[p];
            sxx += dx * dx;
            syy += dy * dy;
            sxy += dx * dy;
            for (int k = 0; k < 4; k++) {
                double dq = q[4 * i + k] - q[4 * p + k];
                if (px) {
                    double corr = dx * (px[4 * i + k] - px[4 * p + k]) + dy * (py[4 * i + k] - py[4 * p + k]);
                    dq = dq - 0.5 * corr;
                }
                sx[k] += dx * dq;
                sy[k] += dy * dq;
            }
        }
        double det = sxx * syy - sxy * sxy;
        for (int k = 0; k < 4; k++) {
            qx[4 * p + k] = (syy * sx[k] - sxy * sy[k]) / det;
            qy[4 * p + k] = (sxx * sy[k] - sxy * sx[k]) / det;
        }
    }
}

/* First-order gradients followed by K Jacobi inner iterations (reading R5). */
void o_q_gradients(const o_cloud *c, const double *q, int K, double *qx, double *qy)
{
    int32_t n = c->n;
    double *px = malloc(sizeof(double) * 4 * (size_t)n);
    double *py = malloc(sizeof(double) * 4 * (size_t)n);
    o_q_gradient_pass(c, q, NULL, NULL, qx, qy);
    for (int it = 1; it <= K; it++) {
        memcpy(px, qx, sizeof(double) * 4 * (size_t)n);
        memcpy(py, qy, sizeof(double) * 4 * (size_t)n);
        o_q_gradient_pass(c, q, px, py, qx, qy);
    }
    free(px); free(py);
}

/* ------------------------------------------------------------------------- */
/* O6, O7: flux residual, local time step and scalar diagonal                 */
/* ------------------------------------------------------------------------- */

/*
 * For every wall and interior point:
 *   R_0 = sum over split sub-stencils s of the LS derivative (Eq. 11) of the
 *   split flux G_s evaluated at the modified q-variables of Eq. 15,
 *   Delta G_i = G_s(q~_i) - G_s(q~_0), q~ defined per neighbour pair;
 *   D_0 = 1/dt_0 - sum_s sign_s rho_s LS_s(1)  (Eq. 26 with Eq. 33-34).
 * Under the kinetic far field outer points add the ghost term of R12 as
 * sub-stencil 3; otherwise they get R = 0, D = 1.  R: [4N], D: [N].
 */
void o_residual(const o_cloud *c, const double *q, const double *qx, const double *qy,
                const double *U, double cfl, double *R, double *D)
{
    for (int32_t p = 0; p < c->n; p++) {
        if (!is_active(c, p)) {
            for (int k = 0; k < 4; k++) R[4 * p + k] = 0.0;
            D[p] = 1.0;
            continue;
        }
        int kind = kind_of(c, p);
        double e1x, e1y, e2x, e2y;
        frame(c, p, &e1x, &e1y, &e2x, &e2y);
        double sdd[4] = { 0 }, spp[4] = { 0 }, sdp[4] = { 0 }, sd1[4] = { 0 }, sp1[4] = { 0 };
        double sdG[4][4] = { { 0 } }, spG[4][4] = { { 0 } };
        double dmin = INFINITY;
        for (int32_t e = c->off[p]; e < c->off[p + 1]; e++) {
            int32_t i = c->idx[e];
            double dx = c->x[i] - c->x[p];
            double dy = c->y[i] - c->y[p];
            double dist = sqrt(dx * dx + dy * dy);
            if (dist < dmin) dmin = dist;
            double a = dx * e1x + dy * e1y;
            double b = dx * e2x + dy * e2y;
            int s[2];
            int m = members(kind, a, b, s);
            if (m == 0) continue;
            double qti[4], qt0[4];
            for (int k = 0; k < 4; k++) {
                qti[k] = q[4 * i + k] - 0.5 * (dx * qx[4 * i + k] + dy * qy[4 * i + k]);
                qt0[k] = q[4 * p + k] - 0.5 * (dx * qx[4 * p + k] + dy * qy[4 * p + k]);
            }
            double ri, ui, vi, pi, bi, r0, u0, v0, p0, b0;
            o_q_to_prim(qti, &ri, &ui, &vi, &pi, &bi);
            o_q_to_prim(qt0, &r0, &u0, &v0, &p0, &b0);
            for (int j = 0; j < m; j++) {
                int ss = s[j];
                double ddx = ss < 2 ? e1x : e2x, ddy = ss < 2 ? e1y : e2y;
                double Gi[4], G0[4];
                o_split_flux(ri, ui, vi, pi, bi, ddx, ddy, SUB_SIGN[ss], Gi);
                o_split_flux(r0, u0, v0, p0, b0, ddx, ddy, SUB_SIGN[ss], G0);
                double d, dp;
                sub_offsets(ss, a, b, &d, &dp);
                sdd[ss] += d * d;
                spp[ss] += dp * dp;
                sdp[ss] += d * dp;
                sd1[ss] += d;
                sp1[ss] += dp;
                for (int k = 0; k < 4; k++) {
                    double dG = Gi[k] - G0[k];
                    sdG[ss][k] += d * dG;
                    spG[ss][k] += dp * dG;
                }
            }
        }
        /* sum of |w_i| per sub-stencil, w_i the LS weight of Eq. 11 */
        double sabsw[4] = { 0, 0, 0, 0 };
        for (int32_t e = c->off[p]; e < c->off[p + 1]; e++) {
            int32_t i = c->idx[e];
            double dx = c->x[i] - c->x[p];
            double dy = c->y[i] - c->y[p];
            double a = dx * e1x + dy * e1y;
            double b = dx * e2x + dy * e2y;
            int s[2];
            int m = members(kind, a, b, s);
            for (int j = 0; j < m; j++) {
                int ss = s[j];
                double d, dp;
                sub_offsets(ss, a, b, &d, &dp);
                double det = sdd[ss] * spp[ss] - sdp[ss] * sdp[ss];
                sabsw[ss] += fabs((spp[ss] * d - sdp[ss] * dp) / det);
            }
        }
        if (kind == 2) sabsw[3] = sabsw[2]; /* the mirrored ghosts (R12) */
        double rho, u, v, pr;
        o_cons_to_prim(&U[4 * p], &rho, &u, &v, &pr);
        double snd = sqrt(GAMMA * pr / rho);
        double dt = cfl * dmin / (sqrt(u * u + v * v) + snd);
        double Dp = 1.0 / dt;
        double Ddom = 0.0;
        double Rp[4] = { 0, 0, 0, 0 };
        double ls1_2 = 0.0;
        for (int ss = 0; ss < 4; ss++) {
            if (kind == 1 && ss == 2) continue;
            double ls1;
            if (real_sub(kind, ss)) {
                double det = sdd[ss] * spp[ss] - sdp[ss] * sdp[ss];
                for (int k = 0; k < 4; k++)
                    Rp[k] += (spp[ss] * sdG[ss][k] - sdp[ss] * spG[ss][k]) / det;
                ls1 = (spp[ss] * sd1[ss] - sdp[ss] * sp1[ss]) / det;
                if (ss == 2) ls1_2 = ls1;
            } else {
                /* R12: LS_3(1) (G_n^-(U_inf) - G_n^-(U_0)), LS_3(1) = -LS_2(1) */
                ls1 = -ls1_2;
                double Gi[4], G0[4];
                o_split_flux_cons(c->uinf, e2x, e2y, -1, Gi);
                o_split_flux_cons(&U[4 * p], e2x, e2y, -1, G0);
                for (int k = 0; k < 4; k++) Rp[k] += ls1 * (Gi[k] - G0[k]);
            }
            double ddx = ss < 2 ? e1x : e2x, ddy = ss < 2 ? e1y : e2y;
            double ud = u * ddx + v * ddy;
            double rs;
            if (SUB_SIGN[ss] > 0) {
                rs = fmax(ud + snd, 0.0);
                Dp -= rs * ls1;
            } else {
                rs = fmax(snd - ud, 0.0);
                Dp += rs * ls1;
            }
            Ddom += rs * sabsw[ss];
        }
        /* reading R6: the local step shrinks where the split weights mix signs,
         * so that D_0 bounds sum_s rho_s sum_i |w_i| */
        if (Ddom > Dp) Dp = Ddom;
        for (int k = 0; k < 4; k++) R[4 * p + k] = Rp[k];
        D[p] = Dp;
    }
}

/* ------------------------------------------------------------------------- */
/* O8: LU-SGS forward and backward sweeps (Eq. 27, Anandhanarayanan diagonal) */
/* ------------------------------------------------------------------------- */

static void wall_project(const o_cloud *c, int p, double *w)
{
    double mn = w[1] * c->nx[p] + w[2] * c->ny[p];
    w[1] = w[1] - mn * c->nx[p];
    w[2] = w[2] - mn * c->ny[p];
}

/* Sum over sub-stencils of the LS x/y-derivative (Eq. 22-24) restricted to the
 * neighbours on one side of p in the order (lower: rank < rank[p]); the
 * geometric sums run over the whole sub-stencil. */
static void offdiag(const o_cloud *c, int p, const int32_t *rank, int lower,
                    const double *U, const double *dW, int jvp, double *out)
{
    int kind = kind_of(c, p);
    double e1x, e1y, e2x, e2y;
    frame(c, p, &e1x, &e1y, &e2x, &e2y);
    double sdd[4] = { 0 }, spp[4] = { 0 }, sdp[4] = { 0 };
    double sdJ[4][4] = { { 0 } }, spJ[4][4] = { { 0 } };
    for (int32_t e = c->off[p]; e < c->off[p + 1]; e++) {
        int32_t i = c->idx[e];
        double dx = c->x[i] - c->x[p];
        double dy = c->y[i] - c->y[p];
        double a = dx * e1x + dy * e1y;
        double b = dx * e2x + dy * e2y;
        int s[2];
        int m = members(kind, a, b, s);
        int side = lower ? (rank[i] < rank[p]) : (rank[i] > rank[p]);
        for (int j = 0; j < m; j++) {
            int ss = s[j];
            double d, dp;
            sub_offsets(ss, a, b, &d, &dp);
            sdd[ss] += d * d;
            spp[ss] += dp * dp;
            sdp[ss] += d * dp;
            if (!side) continue;
            double ddx = ss < 2 ? e1x : e2x, ddy = ss < 2 ? e1y : e2y;
            double J[4];
            if (jvp == JVP_EXACT) o_split_jvp_exact(&U[4 * i], &dW[4 * i], ddx, ddy, SUB_SIGN[ss], J);
            else o_split_jvp_increment(&U[4 * i], &dW[4 * i], ddx, ddy, SUB_SIGN[ss], J);
            for (int k = 0; k < 4; k++) {
                sdJ[ss][k] += d * J[k];
                spJ[ss][k] += dp * J[k];
            }
        }
    }
    for (int k = 0; k < 4; k++) out[k] = 0.0;
    for (int ss = 0; ss < 4; ss++) {
        if (!real_sub(kind, ss)) continue;
        double det = sdd[ss] * spp[ss] - sdp[ss] * sdp[ss];
        for (int k = 0; k < 4; k++)
            out[k] += (spp[ss] * sdJ[ss][k] - sdp[ss] * spJ[ss][k]) / det;
    }
}

/* Forward: dU*_0 = -(R_0 + L dU*)/D_0 over the order; backward, in reverse:
 * dU_0 = dU*_0 - (U dU)/D_0.  Wall increments are projected (reading R4).
 * dUs, dU: [4N] outputs (outer points 0 unless R12). */
void o_sweeps(const o_cloud *c, const int32_t *order, const int32_t *rank, const double *U,
              const double *R, const double *D, int jvp, double *dUs, double *dU)
{
    int32_t n = c->n;
    for (int64_t k = 0; k < 4 * (int64_t)n; k++) { dUs[k] = 0.0; dU[k] = 0.0; }
    for (int32_t pos = 0; pos < n; pos++) {
        int32_t p = order[pos];
        if (!is_active(c, p)) continue;
        double L[4];
        offdiag(c, p, rank, 1, U, dUs, jvp, L);
        double w[4];
        for (int k = 0; k < 4; k++) w[k] = -(R[4 * p + k] + L[k]) / D[p];
        if (c->flag[p] == PT_WALL) wall_project(c, p, w);
        for (int k = 0; k < 4; k++) dUs[4 * p + k] = w[k];
    }
    for (int32_t pos = n - 1; pos >= 0; pos--) {
        int32_t p = order[pos];
        if (!is_active(c, p)) continue;
        double Uc[4];
        offdiag(c, p, rank, 0, U, dU, jvp, Uc);
        double w[4];
        for (int k = 0; k < 4; k++) w[k] = dUs[4 * p + k] - Uc[k] / D[p];
        if (c->flag[p] == PT_WALL) wall_project(c, p, w);
        for (int k = 0; k < 4; k++) dU[4 * p + k] = w[k];
    }
}

/* ------------------------------------------------------------------------- */
/* O9, O10: state update, wall projection, q, residual norm                   */
/* ------------------------------------------------------------------------- */

/* Returns -1 when every updated state is physical, else the first bad point. */
int32_t o_update(const o_cloud *c, double *U, const double *dU, double *q)
{
    int32_t bad = -1;
    for (int32_t p = 0; p < c->n; p++) {
        if (is_active(c, p)) {
            for (int k = 0; k < 4; k++) U[4 * p + k] += dU[4 * p + k];
            if (c->flag[p] == PT_WALL) wall_project(c, p, &U[4 * p]);
        }
        double rho, u, v, pr;
        o_cons_to_prim(&U[4 * p], &rho, &u, &v, &pr);
        if (!(rho > 0.0) || !(pr > 0.0) || !isfinite(rho) || !isfinite(pr) || !isfinite(u) || !isfinite(v)) {
            if (bad < 0) bad = p;
            continue;
        }
        o_prim_to_q(rho, u, v, pr, &q[4 * p]);
    }
    return bad;
}

/* Over the points the iteration updates (R9; with R12 the outer points too). */
double o_residual_norm(const o_cloud *c, const double *R)
{
    double s = 0.0;
    for (int32_t p = 0; p < c->n; p++)
        if (is_active(c, p)) s += R[4 * p] * R[4 * p];
    return sqrt(s);
}

/* ------------------------------------------------------------------------- */
/* O11: lift and drag                                                         */
/* ------------------------------------------------------------------------- */

void o_forces(const o_cloud *c, const double *U, double mach, double aoa_deg, double *cl, double *cd)
{
    int32_t nw = 0;
    for (int32_t p = 0; p < c->n; p++) if (c->flag[p] == PT_WALL) nw++;
    *cl = 0.0; *cd = 0.0;
    if (nw < 3) return;
    int32_t *w = malloc(sizeof(int32_t) * (size_t)nw);
    nw = 0;
    for (int32_t p = 0; p < c->n; p++) if (c->flag[p] == PT_WALL) w[nw++] = p;
    double area2 = 0.0;
    for (int32_t k = 0; k < nw; k++) {
        int32_t a = w[k], b = w[(k + 1) % nw];
        area2 += c->x[a] * c->y[b] - c->x[b] * c->y[a];
    }
    double orient = area2 > 0.0 ? 1.0 : -1.0; /* +1: counter-clockwise */
    double pinf = 1.0 / GAMMA;
    double Fx = 0.0, Fy = 0.0;
    for (int32_t k = 0; k < nw; k++) {
        int32_t a = w[(k + nw - 1) % nw], m = w[k], b = w[(k + 1) % nw];
        double ex = 0.5 * (c->x[m] - c->x[a]) + 0.5 * (c->x[b] - c->x[m]);
        double ey = 0.5 * (c->y[m] - c->y[a]) + 0.5 * (c->y[b] - c->y[m]);
        double nxds = orient * ey, nyds = -orient * ex; /* into the fluid */
        double rho, u, v, pr;
        o_cons_to_prim(&U[4 * m], &rho, &u, &v, &pr);
        Fx -= (pr - pinf) * nxds;
        Fy -= (pr - pinf) * nyds;
    }
    double al = aoa_deg * M_PI / 180.0;
    double qinf = 0.5 * 1.0 * mach * mach;
    *cl = (Fy * cos(al) - Fx * sin(al)) / qinf;
    *cd = (Fx * cos(al) + Fy * sin(al)) / qinf;
    free(w);
}

/* ------------------------------------------------------------------------- */
/* Alg. 1: the implicit LSKUM loop                                            */
/* ------------------------------------------------------------------------- */

void o_freestream(double mach, double aoa_deg, double *Uinf)
{
    double al = aoa_deg * M_PI / 180.0;
    o_prim_to_cons(1.0, mach * cos(al), mach * sin(al), 1.0 / GAMMA, Uinf);
}

/* Free stream everywhere, then the wall projection (reading R4). */
void o_initial_state(const o_cloud *c, double mach, double aoa_deg, double *U)
{
    double Uinf[4];
    o_freestream(mach, aoa_deg, Uinf);
    for (int32_t p = 0; p < c->n; p++) {
        for (int k = 0; k < 4; k++) U[4 * p + k] = Uinf[k];
        if (c->flag[p] == PT_WALL) wall_project(c, p, &U[4 * p]);
    }
}

void o_q_from_state(const o_cloud *c, const double *U, double *q)
{
    for (int32_t p = 0; p < c->n; p++) {
        double rho, u, v, pr;
        o_cons_to_prim(&U[4 * p], &rho, &u, &v, &pr);
        o_prim_to_q(rho, u, v, pr, &q[4 * p]);
    }
}

/* CFL of iteration n (1-based): linear ramp over the first `ramp` iterations. */
double o_cfl_at(double cfl, double ramp, int32_t n)
{
    if (ramp > 0.0 && (double)n < ramp) return cfl * ((double)n / ramp);
    return cfl;
}

/*
 * The revised LU-SGS of Manish et al. (Sec. 3, "+AD" form): Jameson's
 * splitting A_d(+-) = (A_d +- rho(A_d) I)/2 with rho(A_d) = |u_d| + a turns
 * the block diagonal into the scalar
 *   D_0 = 1/dt + sum_s rho(A_dir(s)) |LS_s(1)| / 2
 * plus the term S_0 = -1/2 sum_s LS_s(1) A_dir(s)(U_0) dU_0, which is
 * evaluated with the previous iteration's increment (exact unsplit Jacobian
 * products, here the sum of the exact split ones: G = G+ + G-) and moved to
 * the right-hand side.  Sub-stencils s and frames as in o_residual (wall:
 * t+, t-, n-; kinetic outer: t+, t-, n+ and the ghosts of R12 with
 * LS_3(1) = -LS_2(1)).  With dUprev = NULL, S is not computed.
 */
void o_manish_terms(const o_cloud *c, const double *U, double cfl, const double *dUprev, double *D, double *S)
{
    for (int32_t p = 0; p < c->n; p++) {
        for (int k = 0; k < 4; k++) S[4 * p + k] = 0.0;
        if (!is_active(c, p)) {
            D[p] = 1.0;
            continue;
        }
        int kind = kind_of(c, p);
        double e1x, e1y, e2x, e2y;
        frame(c, p, &e1x, &e1y, &e2x, &e2y);
        double sdd[4] = { 0 }, spp[4] = { 0 }, sdp[4] = { 0 }, sd1[4] = { 0 }, sp1[4] = { 0 };
        double dmin = INFINITY;
        for (int32_t e = c->off[p]; e < c->off[p + 1]; e++) {
            int32_t i = c->idx[e];
            double dx = c->x[i] - c->x[p], dy = c->y[i] - c->y[p];
            double dist = sqrt(dx * dx + dy * dy);
            if (dist < dmin) dmin = dist;
            double a = dx * e1x + dy * e1y, b = dx * e2x + dy * e2y;
            int sub[2];
            int m = members(kind, a, b, sub);
            for (int j = 0; j < m; j++) {
                double d, dp;
                sub_offsets(sub[j], a, b, &d, &dp);
                sdd[sub[j]] += d * d;
                spp[sub[j]] += dp * dp;
                sdp[sub[j]] += d * dp;
                sd1[sub[j]] += d;
                sp1[sub[j]] += dp;
            }
        }
        double rho, u, v, pr;
        o_cons_to_prim(&U[4 * p], &rho, &u, &v, &pr);
        double snd = sqrt(GAMMA * pr / rho);
        double dt = cfl * dmin / (sqrt(u * u + v * v) + snd);
        double Dp = 1.0 / dt;
        double A1[4] = { 0 }, A2[4] = { 0 };
        if (dUprev) {
            double jp[4], jm[4];
            o_split_jvp_exact(&U[4 * p], &dUprev[4 * p], e1x, e1y, +1, jp);
            o_split_jvp_exact(&U[4 * p], &dUprev[4 * p], e1x, e1y, -1, jm);
            for (int k = 0; k < 4; k++) A1[k] = jp[k] + jm[k];
            o_split_jvp_exact(&U[4 * p], &dUprev[4 * p], e2x, e2y, +1, jp);
            o_split_jvp_exact(&U[4 * p], &dUprev[4 * p], e2x, e2y, -1, jm);
            for (int k = 0; k < 4; k++) A2[k] = jp[k] + jm[k];
        }
        double ls1_2 = 0.0;
        for (int ss = 0; ss < 4; ss++) {
            if (kind == 1 && ss == 2) continue;
            double ls1;
            if (real_sub(kind, ss)) {
                double det = sdd[ss] * spp[ss] - sdp[ss] * sdp[ss];
                ls1 = (spp[ss] * sd1[ss] - sdp[ss] * sp1[ss]) / det;
                if (ss == 2) ls1_2 = ls1;
            } else {
                ls1 = -ls1_2; /* the ghosts of R12 */
            }
            double ud = ss < 2 ? u * e1x + v * e1y : u * e2x + v * e2y;
            Dp += 0.5 * (fabs(ud) + snd) * fabs(ls1);
            for (int k = 0; k < 4; k++) S[4 * p + k] -= 0.5 * ls1 * (ss < 2 ? A1[k] : A2[k]);
        }
        D[p] = Dp;
    }
}

/*
 * Explicit q-LSKUM step (the paper's solver (e), Sec. 5: the same residual,
 * no implicit operator): forward Euler in pseudo-time with the local time
 * step of the implicit scheme, dt_0 = CFL min_i |r_i - r_0| / (|u_0| + a_0):
 * dU_0 = -dt_0 R_0 at wall and interior points, with the normal momentum
 * removed at wall points (reading R4, as for the implicit increments); outer
 * points keep dU = 0 unless R12.  D[p] receives 1/dt_0 (1 at frozen points).
 */
void o_explicit_step(const o_cloud *c, const double *U, double cfl, const double *R, double *D, double *dU)
{
    for (int32_t p = 0; p < c->n; p++) {
        for (int k = 0; k < 4; k++) dU[4 * p + k] = 0.0;
        if (!is_active(c, p)) {
            D[p] = 1.0;
            continue;
        }
        double dmin = INFINITY;
        for (int32_t e = c->off[p]; e < c->off[p + 1]; e++) {
            int32_t i = c->idx[e];
            double dx = c->x[i] - c->x[p], dy = c->y[i] - c->y[p];
            double dist = sqrt(dx * dx + dy * dy);
            if (dist < dmin) dmin = dist;
        }
        double rho, u, v, pr;
        o_cons_to_prim(&U[4 * p], &rho, &u, &v, &pr);
        double dt = cfl * dmin / (sqrt(u * u + v * v) + sqrt(GAMMA * pr / rho));
        D[p] = 1.0 / dt;
        for (int k = 0; k < 4; k++) dU[4 * p + k] = -dt * R[4 * p + k];
        if (c->flag[p] == PT_WALL) {
            double mn = dU[4 * p + 1] * c->nx[p] + dU[4 * p + 2] * c->ny[p];
            dU[4 * p + 1] -= mn * c->nx[p];
            dU[4 * p + 2] -= mn * c->ny[p];
        }
    }
}

/*
 * Run up to `iters` iterations from the state U (in/out, [4N]).  Iteration n
 * (counted from n0 + 1) computes q-derivatives, R(U^{n-1}) (first order while
 * n <= first_order) and its norm hist[n-1], sweeps, and
 * updates to U^n; it stops after iteration n when hist[n-1]/hist0 <= target
 * (hist0 = the first norm of this call unless *hist0 > 0 is passed in).
 * Returns 0, or -(1 + point) on a non-physical update.  *done = iterations run.
 * Work arrays (each [4N] unless noted) are supplied by the caller so that a
 * test can read the last iteration's intermediates:
 *   q, qx, qy, R, D[N], dUs, dU.
 */
int32_t o_run(const o_cloud *c, const int32_t *order, const int32_t *rank,
              double cfl, double ramp, int32_t K, int32_t jvp, int32_t first_order,
              int32_t iters, double target, int32_t n0,
              double *U, double *q, double *qx, double *qy, double *R, double *D,
              double *dUs, double *dU, double *hist, double *hist0, int32_t *done)
{
    *done = 0;
    double *zero = calloc(4 * (size_t)c->n, sizeof(double));
    o_q_from_state(c, U, q);
    for (int32_t it = 0; it < iters; it++) {
        int32_t n = n0 + it + 1;
        o_q_gradients(c, q, K, qx, qy);
        if (n <= first_order) o_residual(c, q, zero, zero, U, o_cfl_at(cfl, ramp, n), R, D);
        else o_residual(c, q, qx, qy, U, o_cfl_at(cfl, ramp, n), R, D);
        hist[it] = o_residual_norm(c, R);
        if (!(*hist0 > 0.0)) *hist0 = hist[it];
        o_sweeps(c, order, rank, U, R, D, jvp, dUs, dU);
        int32_t bad = o_update(c, U, dU, q);
        *done = it + 1;
        if (bad >= 0) {
            free(zero);
            return -(1 + bad);
        }
        if (hist[it] / *hist0 <= target) break;
    }
    free(zero);
    return 0;
}

/*
 * As o_run with the revised LU-SGS of Manish et al.: D from o_manish_terms
 * and the right-hand side -R + sigma S(dU of the previous iteration of this
 * call; zero at its first), sigma = +1 as the paper prints the sweeps, -1 as
 * the algebra of the split diagonal gives.  Both leave the fixed point R = 0
 * unchanged.  The history holds the norms of R.
 */
int32_t o_run_manish(const o_cloud *c, const int32_t *order, const int32_t *rank,
                     double cfl, double ramp, int32_t K, int32_t jvp, int32_t first_order, int32_t sigma,
                     int32_t iters, double target, int32_t n0,
                     double *U, double *q, double *qx, double *qy, double *R, double *D,
                     double *dUs, double *dU, double *hist, double *hist0, int32_t *done)
{
    *done = 0;
    size_t n4 = 4 * (size_t)c->n;
    double *zero = calloc(n4, sizeof(double));
    double *S = calloc(n4, sizeof(double));
    double *Reff = calloc(n4, sizeof(double));
    double *prev = calloc(n4, sizeof(double));
    o_q_from_state(c, U, q);
    int32_t status = 0;
    for (int32_t it = 0; it < iters; it++) {
        int32_t n = n0 + it + 1;
        double cfl_n = o_cfl_at(cfl, ramp, n);
        o_q_gradients(c, q, K, qx, qy);
        if (n <= first_order) o_residual(c, q, zero, zero, U, cfl_n, R, D);
        else o_residual(c, q, qx, qy, U, cfl_n, R, D);
        hist[it] = o_residual_norm(c, R);
        if (!(*hist0 > 0.0)) *hist0 = hist[it];
        o_manish_terms(c, U, cfl_n, prev, D, S);
        for (size_t k = 0; k < n4; k++) Reff[k] = R[k] - (double)sigma * S[k];
        o_sweeps(c, order, rank, U, Reff, D, jvp, dUs, dU);
        for (size_t k = 0; k < n4; k++) prev[k] = dU[k];
        int32_t bad = o_update(c, U, dU, q);
        *done = it + 1;
        if (bad >= 0) {
            status = -(1 + bad);
            break;
        }
        if (hist[it] / *hist0 <= target) break;
    }
    free(zero);
    free(S);
    free(Reff);
    free(prev);
    return status;
}

/* As o_run with the explicit step in place of the LU-SGS sweeps (dUs stays 0). */
int32_t o_run_explicit(const o_cloud *c, double cfl, double ramp, int32_t K, int32_t first_order,
                       int32_t iters, double target, int32_t n0,
                       double *U, double *q, double *qx, double *qy, double *R, double *D,
                       double *dU, double *hist, double *hist0, int32_t *done)
{
    *done = 0;
    double *zero = calloc(4 * (size_t)c->n, sizeof(double));
    o_q_from_state(c, U, q);
    for (int32_t it = 0; it < iters; it++) {
        int32_t n = n0 + it + 1;
        double cfl_n = o_cfl_at(cfl, ramp, n);
        o_q_gradients(c, q, K, qx, qy);
        if (n <= first_order) o_residual(c, q, zero, zero, U, cfl_n, R, D);
        else o_residual(c, q, qx, qy, U, cfl_n, R, D);
        hist[it] = o_residual_norm(c, R);
        if (!(*hist0 > 0.0)) *hist0 = hist[it];
        o_explicit_step(c, U, cfl_n, R, D, dU);
        int32_t bad = o_update(c, U, dU, q);
        *done = it + 1;
        if (bad >= 0) {
            free(zero);
            return -(1 + bad);
        }
        if (hist[it] / *hist0 <= target) break;
    }
    free(zero);
    return 0;
}
