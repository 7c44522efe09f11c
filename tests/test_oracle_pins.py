"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: kinetic
moment quadrature, the entropy function, finite differences, brute-force
linear algebra, closed forms and exact symmetries.  None needs a GPU.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2406_07441_gb300 import cloudgen as cg

GAMMA = 1.4
RNG = np.random.default_rng(7)


def _random_states(n, smax=3.0, rng=RNG):
    out = []
    for _ in range(n):
        rho = rng.uniform(0.3, 3.0)
        p = rng.uniform(0.2, 3.0)
        beta = rho / (2 * p)
        S = rng.uniform(-smax, smax)
        th = rng.uniform(0, 2 * math.pi)
        speed = abs(S) / math.sqrt(beta)
        out.append((rho, speed * math.cos(th), speed * math.sin(th), p))
    return out


# ---------------------------------------------------------------------------
# O1: q-variables are the entropy variables of the Euler equations (Eq. 14)
# ---------------------------------------------------------------------------

def test_q_roundtrip():
    for rho, u, v, p in _random_states(200):
        q = O.prim_to_q(rho, u, v, p)
        r2, u2, v2, p2, b2 = O.q_to_prim(q)
        assert abs(r2 - rho) <= 1e-14 * rho * 4
        assert abs(p2 - p) <= 1e-14 * p * 4
        assert abs(u2 - u) <= 1e-14 * (abs(u) + 1) * 4
        assert abs(v2 - v) <= 1e-14 * (abs(v) + 1) * 4
        assert abs(b2 - rho / (2 * p)) <= 1e-14 * b2 * 4
        U = O.prim_to_cons(rho, u, v, p)
        r3, u3, v3, p3 = O.cons_to_prim(U)
        assert np.allclose([r3, u3, v3, p3], [rho, u, v, p], rtol=1e-13, atol=1e-14)


def test_q_is_entropy_gradient():
    """q = d(eta)/dU with eta = -rho s / (gamma - 1), s = ln p - gamma ln rho
    (q_1 up to the constant (gamma + ln 2)/(gamma - 1))."""

    def eta(U):
        rho = U[0]
        p = (GAMMA - 1) * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / rho)
        return -rho * (math.log(p) - GAMMA * math.log(rho)) / (GAMMA - 1)

    for rho, u, v, p in _random_states(30, smax=1.5):
        U = O.prim_to_cons(rho, u, v, p)
        q = O.prim_to_q(rho, u, v, p)
        g = np.zeros(4)
        for k in range(4):
            h = 1e-5 * max(1.0, abs(U[k]))
            e = np.zeros(4)
            e[k] = h
            g[k] = (eta(U + e) - eta(U - e)) / (2 * h)
        assert np.allclose(q[1:], g[1:], rtol=1e-7, atol=1e-7)
        assert abs((g[0] - q[0]) - (GAMMA + math.log(2)) / (GAMMA - 1)) < 1e-6


# ---------------------------------------------------------------------------
# O2: split fluxes are half-range moments of the Maxwellian (Eq. 3-6)
# ---------------------------------------------------------------------------

def _gl(a, b, n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def _quadrature_flux(rho, u, v, p, d, sign):
    """Brute-force int v_d Psi F over sign*v_d > 0, F of Eq. 4 with the
    internal-energy variable integrated out (I0 = (2-gamma)/(gamma-1) p/rho)."""
    beta = rho / (2 * p)
    sig = 1 / math.sqrt(2 * beta)
    I0 = (2 - GAMMA) / (GAMMA - 1) * p / rho
    d = np.asarray(d, float)
    e = np.array([-d[1], d[0]])
    ud, ue = u * d[0] + v * d[1], u * e[0] + v * e[1]
    # half range in w = v.d, pieces of width ~ sigma for accuracy
    lo, hi = (0.0, max(ud, 0.0) + 14 * sig) if sign > 0 else (min(ud, 0.0) - 14 * sig, 0.0)
    edges = np.linspace(lo, hi, 41)
    ws, ww = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        x, w = _gl(a, b, 24)
        ws.append(x)
        ww.append(w)
    W, WW = np.concatenate(ws), np.concatenate(ww)
    edges = np.linspace(ue - 14 * sig, ue + 14 * sig, 41)
    es, ew = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        x, w = _gl(a, b, 24)
        es.append(x)
        ew.append(w)
    E, EW = np.concatenate(es), np.concatenate(ew)
    w_, e_ = np.meshgrid(W, E, indexing="ij")
    wt = np.outer(WW, EW)
    v1 = w_ * d[0] + e_ * e[0]
    v2 = w_ * d[1] + e_ * e[1]
    F = rho * beta / math.pi * np.exp(-beta * ((v1 - u) ** 2 + (v2 - v) ** 2))
    vd = w_
    psi = [np.ones_like(v1), v1, v2, I0 + 0.5 * (v1 ** 2 + v2 ** 2)]
    return np.array([np.sum(wt * vd * ps * F) for ps in psi])


@pytest.mark.parametrize("seed", range(6))
def test_split_flux_matches_kinetic_quadrature(seed):
    rng = np.random.default_rng(100 + seed)
    (rho, u, v, p), = _random_states(1, smax=2.5, rng=rng)
    th = rng.uniform(0, 2 * math.pi)
    d = (math.cos(th), math.sin(th))
    for sign in (+1, -1):
        G = O.split_flux(rho, u, v, p, d[0], d[1], sign)
        Q = _quadrature_flux(rho, u, v, p, d, sign)
        scale = np.max(np.abs(Q)) + np.max(np.abs(O.euler_flux(rho, u, v, p, d[0], d[1])))
        assert np.max(np.abs(G - Q)) <= 1e-10 * scale, (sign, G, Q)


def test_split_fluxes_sum_to_euler_flux_and_euler_matches_quadrature():
    for rho, u, v, p in _random_states(100):
        for d in ((1.0, 0.0), (0.0, 1.0), (0.6, 0.8)):
            Gp = O.split_flux(rho, u, v, p, d[0], d[1], +1)
            Gm = O.split_flux(rho, u, v, p, d[0], d[1], -1)
            E = O.euler_flux(rho, u, v, p, d[0], d[1])
            assert np.allclose(Gp + Gm, E, rtol=1e-14, atol=1e-14 * np.max(np.abs(E)) * 8)
    rho, u, v, p = 1.3, 0.4, -0.2, 0.9
    d = (0.6, 0.8)
    Q = _quadrature_flux(rho, u, v, p, d, +1) + _quadrature_flux(rho, u, v, p, d, -1)
    assert np.allclose(O.euler_flux(rho, u, v, p, *d), Q, rtol=1e-10, atol=1e-12)


def test_split_flux_limits():
    rho, p = 1.0, 1.0 / GAMMA
    beta = rho / (2 * p)
    u = 9.0 / math.sqrt(beta)  # S = 9: every molecule moves in +x
    Gm = O.split_flux(rho, u, 0.0, p, 1.0, 0.0, -1)
    Gp = O.split_flux(rho, u, 0.0, p, 1.0, 0.0, +1)
    E = O.euler_flux(rho, u, 0.0, p, 1.0, 0.0)
    assert np.max(np.abs(Gm)) < 1e-30
    assert np.allclose(Gp, E, rtol=1e-15)
    Gp2 = O.split_flux(rho, -u, 0.0, p, 1.0, 0.0, +1)
    assert np.max(np.abs(Gp2)) < 1e-30


# ---------------------------------------------------------------------------
# O8: Jacobian-vector products
# ---------------------------------------------------------------------------

def test_exact_jvp_matches_central_differences():
    rng = np.random.default_rng(11)
    for rho, u, v, p in _random_states(150, smax=5.0, rng=rng):
        U = O.prim_to_cons(rho, u, v, p)
        th = rng.uniform(0, 2 * math.pi)
        d = (math.cos(th), math.sin(th))
        dU = rng.normal(size=4) * (np.abs(U) + 0.1)
        for sign in (+1, -1):
            J = O.split_jvp(U, dU, d[0], d[1], sign, O.JVP_EXACT)
            h = 1e-4

            def G(t):
                return O.split_flux_cons(U + t * dU, d[0], d[1], sign)

            # fourth-order central difference
            fd = (-G(2 * h) + 8 * G(h) - 8 * G(-h) + G(-2 * h)) / (12 * h)
            scale = np.max(np.abs(fd)) + 1e-3 * np.max(np.abs(dU))
            assert np.max(np.abs(J - fd)) <= 1e-7 * scale, (J, fd)


def test_unsplit_jvp_from_split_pair_matches_listing_chain():
    """A_x dU = A_x^+ dU + A_x^- dU; the unsplit product follows the chain rule of
    the Gx routine of Appendix A (rho, u1, u2, p and their tangents)."""
    rng = np.random.default_rng(12)
    for rho, u, v, p in _random_states(40, rng=rng):
        U = O.prim_to_cons(rho, u, v, p)
        dU = rng.normal(size=4)
        Jp = O.split_jvp(U, dU, 1.0, 0.0, +1)
        Jm = O.split_jvp(U, dU, 1.0, 0.0, -1)
        r, rd = U[0], dU[0]
        u1, u1d = U[1] / r, (dU[1] - U[1] / r * rd) / r
        u2, u2d = U[2] / r, (dU[2] - U[2] / r * rd) / r
        pr = 0.4 * (U[3] - 0.5 * r * (u1 * u1 + u2 * u2))
        prd = 0.4 * (dU[3] - 0.5 * ((u1 * u1 + u2 * u2) * rd + r * (2 * u1 * u1d + 2 * u2 * u2d)))
        ref = np.array([u1 * rd + r * u1d, prd + u1 ** 2 * rd + 2 * r * u1 * u1d,
                        u2 * (u1 * rd + r * u1d) + r * u1 * u2d, u1 * (prd + dU[3]) + (pr + U[3]) * u1d])
        assert np.allclose(Jp + Jm, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_increment_jvp_is_exact_to_second_order():
    rng = np.random.default_rng(13)
    for rho, u, v, p in _random_states(20, rng=rng):
        U = O.prim_to_cons(rho, u, v, p)
        dU = rng.normal(size=4) * 0.1 * np.abs(U).max()
        errs = []
        for eps in (1e-2, 1e-3):
            a = O.split_jvp(U, eps * dU, 0.6, 0.8, +1, O.JVP_INCREMENT)
            b = O.split_jvp(U, eps * dU, 0.6, 0.8, +1, O.JVP_EXACT)
            errs.append(np.max(np.abs(a - b)))
        slope = math.log10(errs[0] / errs[1])
        assert 1.8 < slope < 2.2, (errs, slope)


# ---------------------------------------------------------------------------
# O4, O5: least-squares q-derivatives (Eq. 10, 16)
# ---------------------------------------------------------------------------

def test_ls_gradients_exact_for_linear_fields():
    c = cg.cartesian_box(12, 12, seed=3)
    o = O.Oracle(c)
    a = RNG.normal(size=4)
    b = RNG.normal(size=4)
    cc = RNG.normal(size=4)
    q = a[None, :] + np.outer(c.x, b) + np.outer(c.y, cc)
    for K in (0, 1, 3):
        qx, qy = o.q_gradients(q, K)
        assert np.allclose(qx, b[None, :], rtol=0, atol=1e-11)
        assert np.allclose(qy, cc[None, :], rtol=0, atol=1e-11)


def test_exact_gradient_of_a_quadratic_is_the_inner_iteration_fixed_point():
    """For quadratic q, Delta q_i - (Delta r . (grad q_i - grad q_0))/2 = Delta r . grad q_0
    exactly, so the exact gradient is a fixed point of Eq. 16; from the
    first-order start the Jacobi iterates approach it."""
    c = cg.cartesian_box(12, 12, seed=4)
    o = O.Oracle(c)
    H = RNG.normal(size=(4, 3))
    x, y = c.x, c.y
    q = np.stack([H[k, 0] * x * x + H[k, 1] * x * y + H[k, 2] * y * y for k in range(4)], 1)
    gx = np.stack([2 * H[k, 0] * x + H[k, 1] * y for k in range(4)], 1)
    gy = np.stack([H[k, 1] * x + 2 * H[k, 2] * y for k in range(4)], 1)
    qx, qy = o.q_gradient_pass(q, gx, gy)
    assert np.allclose(qx, gx, rtol=0, atol=1e-12) and np.allclose(qy, gy, rtol=0, atol=1e-12)
    errs = []
    for K in (0, 1, 2, 4, 8):
        qx, qy = o.q_gradients(q, K)
        errs.append(max(np.abs(qx - gx).max(), np.abs(qy - gy).max()))
    assert errs[0] > 1e-3
    assert all(e1 > e2 for e1, e2 in zip(errs[:-1], errs[1:])), errs
    # K passes equal K explicit single passes from the first-order start
    px, py = o.q_gradient_pass(q)
    for _ in range(3):
        px, py = o.q_gradient_pass(q, px, py)
    qx, qy = o.q_gradients(q, 3)
    assert np.array_equal(px, qx) and np.array_equal(py, qy)


# ---------------------------------------------------------------------------
# O6: residual
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["box", "ogrid"])
def test_free_stream_preserved_bitwise(which):
    # any uniform state, walls included (the residual only sees differences)
    c = cg.cartesian_box(9, 9) if which == "box" else cg.naca0012_block(40, 16)
    o = O.Oracle(c)
    Uinf = O.freestream(0.7, 3.0)
    U = np.tile(Uinf, (c.n, 1))
    q = o.q_from_state(U)
    qx, qy = o.q_gradients(q, 3)
    assert np.all(qx == 0.0) and np.all(qy == 0.0)
    R, D = o.residual(q, qx, qy, U, 100.0)
    assert np.all(R == 0.0)
    assert np.all(D[c.flag != cg.OUTER] > 0)
    dUs, dU = o.sweeps(U, R, D)
    assert np.all(dU == 0.0)


def _smooth_state(x, y, amp=0.05):
    rho = 1.0 + amp * np.sin(1.3 * x + 0.4) * np.cos(0.9 * y - 0.2)
    u = 0.6 + amp * np.cos(0.7 * x - 1.1 * y)
    v = 0.1 + amp * np.sin(0.8 * x + 0.5 * y)
    p = 1 / GAMMA + amp * np.cos(1.1 * x) * np.sin(0.6 * y + 0.3)
    return rho, u, v, p


def test_residual_mirror_symmetry():
    c = cg.cartesian_box(10, 9, seed=5)
    c2 = cg.Cloud(c.x, -c.y, c.flag, c.nx, -c.ny, c.nbr_off, c.nbr_idx, c.meta)
    rho, u, v, p = _smooth_state(c.x, c.y)
    U = np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)], 1)
    U2 = U * np.array([1, 1, -1, 1])
    out = []
    for cc, UU in ((c, U), (c2, U2)):
        o = O.Oracle(cc)
        q = o.q_from_state(UU)
        qx, qy = o.q_gradients(q, 3)
        out.append(o.residual(q, qx, qy, UU, 50.0))
    R1, D1 = out[0]
    R2, D2 = out[1]
    m = c.flag != cg.OUTER
    assert np.allclose(R2[m] * np.array([1, 1, -1, 1]), R1[m], rtol=1e-12, atol=1e-12 * np.abs(R1).max())
    assert np.allclose(D1[m], D2[m], rtol=1e-13)


def test_residual_converges_to_euler_divergence_second_order():
    """On regular Cartesian clouds R -> d(Gx)/dx + d(Gy)/dy at O(h^2) (the
    second-order claim of the defect-corrected scheme, Eq. 7-15).  (On jittered
    clouds the order approaches 2 only as the inner iterations converge.)"""
    errs = []
    hs = []
    for n in (17, 33):
        c = cg.cartesian_box(n, n, jitter=0.0, seed=9)
        o = O.Oracle(c)
        x, y = c.x * 2.0, c.y * 2.0  # domain [0,2]^2
        c2 = cg.Cloud(x, y, c.flag, c.nx, c.ny, c.nbr_off, c.nbr_idx, c.meta)
        o = O.Oracle(c2)
        rho, u, v, p = _smooth_state(x, y, amp=0.2)
        U = np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)], 1)
        q = o.q_from_state(U)
        qx, qy = o.q_gradients(q, 3)
        R, _ = o.residual(q, qx, qy, U, 100.0)
        # exact divergence of the Euler flux by central differences of the closed-form field
        h = 1e-5

        def flux(xx, yy, d):
            r, uu, vv, pp = _smooth_state(xx, yy, amp=0.2)
            E = pp / 0.4 + 0.5 * r * (uu * uu + vv * vv)
            un = uu * d[0] + vv * d[1]
            return np.stack([r * un, r * uu * un + pp * d[0], r * vv * un + pp * d[1], (E + pp) * un], 1)

        div = (flux(x + h, y, (1, 0)) - flux(x - h, y, (1, 0))) / (2 * h) \
            + (flux(x, y + h, (0, 1)) - flux(x, y - h, (0, 1))) / (2 * h)
        far = (x > 0.5) & (x < 1.5) & (y > 0.5) & (y < 1.5)
        errs.append(np.abs(R[far] - div[far]).max())
        hs.append(2.0 / (n - 1))
    order = math.log(errs[0] / errs[1]) / math.log(hs[0] / hs[1])
    assert order > 1.8, (errs, order)


# ---------------------------------------------------------------------------
# O8: sweeps equal the dense LU-SGS solve of Eq. 26-27 (brute force)
# ---------------------------------------------------------------------------

def _dense_lusgs(c, o, U, R, D, kinetic=False):
    n = c.n
    act = np.flatnonzero((c.flag != cg.OUTER) | kinetic)
    pos = {p: k for k, p in enumerate(act)}
    m = len(act)
    L = np.zeros((4 * m, 4 * m))
    Uu = np.zeros((4 * m, 4 * m))
    P = np.eye(4 * m)
    for p in act:
        r = c.nbr_idx[c.nbr_off[p]:c.nbr_off[p + 1]]
        dx = c.x[r] - c.x[p]
        dy = c.y[r] - c.y[p]
        wall = c.flag[p] == cg.WALL
        outer = c.flag[p] == cg.OUTER
        if wall or outer:
            e1 = (c.ny[p], -c.nx[p])
            e2 = (c.nx[p], c.ny[p])
        else:
            e1, e2 = (1.0, 0.0), (0.0, 1.0)
        if wall:
            nn = np.array([c.nx[p], c.ny[p]])
            k = pos[p]
            P[4 * k + 1:4 * k + 3, 4 * k + 1:4 * k + 3] = np.eye(2) - np.outer(nn, nn)
        a = dx * e1[0] + dy * e1[1]
        b = dx * e2[0] + dy * e2[1]
        subs = [(a < 0, a, b, e1, +1), (a > 0, a, b, e1, -1)]
        if not wall:
            subs.append((b < 0, b, a, e2, +1))
        if not outer:  # a kinetic outer point's n- side holds the constant free-stream ghosts
            subs.append((b > 0, b, a, e2, -1))
        for msk, dd, dp, e, sg in subs:
            sdd, spp, sdp = np.sum(dd[msk] ** 2), np.sum(dp[msk] ** 2), np.sum(dd[msk] * dp[msk])
            det = sdd * spp - sdp * sdp
            for i, di, pi in zip(r[msk], dd[msk], dp[msk]):
                w = (spp * di - sdp * pi) / det
                if c.flag[i] == cg.OUTER and not kinetic:
                    continue
                J = np.stack([O.split_jvp(U[i], np.eye(4)[k], e[0], e[1], sg) for k in range(4)], 1)
                tgt = L if o.rank[i] < o.rank[p] else Uu
                tgt[4 * pos[p]:4 * pos[p] + 4, 4 * pos[i]:4 * pos[i] + 4] += w * J
    Dinv = np.repeat(1.0 / D[act], 4)
    I = np.eye(4 * m)
    rhs = -(P @ (Dinv * R[act].ravel()))
    dus = np.linalg.solve(I + P @ (Dinv[:, None] * L), rhs)
    du = np.linalg.solve(I + P @ (Dinv[:, None] * Uu), P @ dus)
    out_s = np.zeros((n, 4))
    out = np.zeros((n, 4))
    out_s[act] = dus.reshape(m, 4)
    out[act] = du.reshape(m, 4)
    return out_s, out


@pytest.mark.parametrize("wall,ordering", [(False, 0), (True, 0), (True, 1), (True, 2)])
def test_sweeps_equal_dense_lusgs(wall, ordering):
    """Sequential sweeps in the order of Alg. 6 (colours), of Alg. 4 (wall
    points first, by colour) or of Alg. 2 (wall, interior, outer points in
    index order) equal the dense solve with L and U split by that order."""
    c = cg.cartesian_box(7, 7, seed=21, wall_bottom=wall)
    assert c.n == 49
    o = O.Oracle(c, ordering=ordering)
    if ordering >= 1:  # wall points lead the order, then interior, then outer
        f = c.flag[o.order]
        assert np.all(np.diff(np.where(f == cg.WALL, 0, np.where(f == cg.INTERIOR, 1, 2))) >= 0)
    if ordering == 2:  # each group in index order
        for g in (cg.WALL, cg.INTERIOR, cg.OUTER):
            assert np.all(np.diff(o.order[c.flag[o.order] == g]) > 0)
    rho, u, v, p = _smooth_state(c.x * 3, c.y * 3, amp=0.08)
    U = np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)], 1)
    if wall:
        wm = c.flag == cg.WALL
        U[wm, 2] = 0.0  # normal (y) momentum removed at the flat wall
    q = o.q_from_state(U)
    qx, qy = o.q_gradients(q, 3)
    R, D = o.residual(q, qx, qy, U, 5.0)
    dUs, dU = o.sweeps(U, R, D, O.JVP_EXACT)
    ds_ref, d_ref = _dense_lusgs(c, o, U, R, D)
    scale = np.abs(d_ref).max()
    assert scale > 1e-6
    assert np.allclose(dUs, ds_ref, rtol=0, atol=1e-12 * np.abs(ds_ref).max())
    assert np.allclose(dU, d_ref, rtol=0, atol=1e-12 * scale)


# ---------------------------------------------------------------------------
# Kinetic far field (outer points updated; ghosts hold the free stream)
# ---------------------------------------------------------------------------

def _kinetic_smooth_state(c, Uinf, amp=0.05):
    x, y = c.x, c.y
    rho = 1 + amp * np.sin(3 * x + 1) * np.cos(2 * y)
    u = Uinf[1] + amp * np.cos(2 * x - 3 * y)
    v = Uinf[2] + amp * np.sin(x + 2 * y)
    p = 1 / GAMMA + amp * np.cos(3 * x) * np.sin(2 * y + 0.3)
    return np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)], 1)


@pytest.mark.parametrize("which", ["box", "ogrid"])
def test_kinetic_far_field_preserves_the_free_stream_bitwise(which):
    c = cg.cartesian_box(9, 9, kinetic_outer=True) if which == "box" else cg.naca0012_block(40, 16, kinetic_outer=True)
    o = O.Oracle(c, farfield=O.FARFIELD_KINETIC, mach=1.2, aoa_deg=3.0)
    U = np.tile(O.freestream(1.2, 3.0), (c.n, 1))  # uniform, walls included (as above)
    q = o.q_from_state(U)
    qx, qy = o.q_gradients(q, 3)
    R, D = o.residual(q, qx, qy, U, 100.0)
    assert np.all(R == 0.0)
    assert np.all(D > 0) and np.all(D[c.flag == cg.OUTER] != 1.0)
    dUs, dU = o.sweeps(U, R, D)
    assert np.all(dU == 0.0)


def test_kinetic_ghost_term_is_the_mirrored_free_stream_stencil():
    """The far-field term equals an n-derivative over ghost points that carry
    the free stream at the mirror images of the point's inside (n+)
    neighbours: the difference of the residuals for two free streams A and B
    is, at an outer point, sum_g w_g (G_n^-(A) - G_n^-(B)) with w_g the
    least-squares n-derivative weights of the ghost set (solved here with
    numpy, from the coordinates), and exactly 0 at every other point."""
    c = cg.cartesian_box(9, 8, seed=11, kinetic_outer=True)
    A, B = (0.5, 10.0), (1.5, -20.0)
    Ua, Ub = O.freestream(*A), O.freestream(*B)
    U = _kinetic_smooth_state(c, Ua)
    out = []
    for m, al in (A, B):
        o = O.Oracle(c, farfield=O.FARFIELD_KINETIC, mach=m, aoa_deg=al)
        q = o.q_from_state(U)
        qx, qy = o.q_gradients(q, 3)
        out.append(o.residual(q, qx, qy, U, 10.0)[0])
    dR = out[0] - out[1]
    inner = c.flag != cg.OUTER
    assert np.all(dR[inner] == 0.0)
    checked = 0
    for p in np.flatnonzero(~inner):
        r = c.nbr_idx[c.nbr_off[p]:c.nbr_off[p + 1]]
        t = np.array([c.ny[p], -c.nx[p]])
        nn = np.array([c.nx[p], c.ny[p]])
        d = np.stack([c.x[r] - c.x[p], c.y[r] - c.y[p]], 1)
        inside = d @ nn < 0
        g = d[inside] - 2.0 * np.outer(d[inside] @ nn, nn)  # mirror images across the tangent line
        Xg = np.stack([g @ t, g @ nn], 1)
        W = np.linalg.solve(Xg.T @ Xg, Xg.T)  # rows: t- and n-derivative weights
        wn = W[1]
        expect = wn.sum() * (O.split_flux_cons(Ua, nn[0], nn[1], -1) - O.split_flux_cons(Ub, nn[0], nn[1], -1))
        assert np.allclose(dR[p], expect, rtol=1e-11, atol=1e-13 * np.abs(expect).max()), p
        assert wn.sum() > 0
        checked += 1
    assert checked == int((~inner).sum())


@pytest.mark.parametrize("wall", [False, True])
def test_kinetic_sweeps_equal_dense_lusgs(wall):
    """With the kinetic far field the outer points are unknowns of the dense
    system too; the sequential sweeps still equal its solve."""
    c = cg.cartesian_box(7, 7, seed=21, wall_bottom=wall, kinetic_outer=True)
    o = O.Oracle(c, farfield=O.FARFIELD_KINETIC, mach=0.8, aoa_deg=5.0)
    U = _kinetic_smooth_state(c, O.freestream(0.8, 5.0), amp=0.08)
    if wall:
        U[c.flag == cg.WALL, 2] = 0.0
    q = o.q_from_state(U)
    qx, qy = o.q_gradients(q, 3)
    R, D = o.residual(q, qx, qy, U, 5.0)
    dUs, dU = o.sweeps(U, R, D, O.JVP_EXACT)
    ds_ref, d_ref = _dense_lusgs(c, o, U, R, D, kinetic=True)
    scale = np.abs(d_ref).max()
    assert np.abs(dU[c.flag == cg.OUTER]).max() > 1e-3 * scale
    assert np.allclose(dUs, ds_ref, rtol=0, atol=1e-12 * np.abs(ds_ref).max())
    assert np.allclose(dU, d_ref, rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("mach,aoa", [(2.0, 10.0), (0.5, 10.0)])
@pytest.mark.parametrize("scheme", ["lusgs", "manish", "explicit"])
def test_kinetic_far_field_returns_to_the_free_stream(mach, aoa, scheme):
    """Without a body the free stream is the steady state: from a perturbed
    start (outer points included) every scheme drives the whole cloud back to
    it, through incoming (free-stream ghosts) and outgoing boundaries alike."""
    c = cg.cartesian_box(9, 9, seed=3, kinetic_outer=True)
    o = O.Oracle(c, farfield=O.FARFIELD_KINETIC, mach=mach, aoa_deg=aoa)
    Uinf = O.freestream(mach, aoa)
    U = _kinetic_smooth_state(c, Uinf)
    if scheme == "lusgs":
        r = o.run(U, 400, cfl=5.0, K=3)
    elif scheme == "manish":
        r = o.run_manish(U, 400, cfl=2.0, K=3)
    else:
        r = o.run_explicit(U, 3000, cfl=0.3, K=3)
    assert r["status"] == 0
    assert r["hist"][-1] < 1e-6 * r["hist"][0]
    assert np.abs(r["U"] - Uinf).max() < 1e-6


# ---------------------------------------------------------------------------
# a0: colouring (Alg. 5)
# ---------------------------------------------------------------------------

def _alg5(n, off, idx):
    own = [list(idx[off[p]:off[p + 1]]) for p in range(n)]
    sets = [set(r) for r in own]
    rev = [[] for _ in range(n)]
    for p in range(n):
        for q in own[p]:
            if p not in sets[q]:
                rev[q].append(p)
    adj = [own[p] + sorted(rev[p]) for p in range(n)]
    col = [0] * n
    col[0] = 1

    def smallest(p):
        used = {col[q] for q in adj[p]}
        k = 1
        while k in used:
            k += 1
        return k

    for i in range(n):
        if col[i] == 0:
            col[i] = smallest(i)
        for p in adj[i]:
            if col[p] == 0:
                col[p] = smallest(p)
    return np.array(col), adj


@pytest.mark.parametrize("which", ["box", "ogrid", "jit"])
def test_colouring_is_alg5_and_valid(which):
    if which == "box":
        c = cg.cartesian_box(9, 8)
    elif which == "ogrid":
        c = cg.naca0012_block(40, 16)
    else:
        c = cg.naca0012_jittered(40, 16, seed=5)
    o = O.Oracle(c)
    ref, adj = _alg5(c.n, c.nbr_off, c.nbr_idx)
    assert np.array_equal(o.colour, ref)
    for p in range(c.n):
        for q in adj[p]:
            assert o.colour[p] != o.colour[q]
    # canonical order: stable sort by colour
    assert np.array_equal(o.order, np.argsort(o.colour, kind="stable"))
    assert np.array_equal(o.rank[o.order], np.arange(c.n))


# ---------------------------------------------------------------------------
# O11: forces
# ---------------------------------------------------------------------------

def _circle_cloud(n=400, r=0.5):
    th = 2 * math.pi * np.arange(n) / n
    x = 0.5 + r * np.cos(th)
    y = r * np.sin(th)
    flag = np.full(n, cg.WALL, np.uint8)
    nx, ny = np.cos(th), np.sin(th)
    off = np.arange(n + 1, dtype=np.int32)
    idx = ((np.arange(n) + 1) % n).astype(np.int32)
    return cg.Cloud(x, y, flag, nx, ny, off, idx, {})


def test_forces_closed_forms():
    c = _circle_cloud()
    o = O.Oracle(c)
    mach = 0.5
    # uniform pressure: no force
    U = np.tile(O.prim_to_cons(1.0, 0.0, 0.0, 3.7), (c.n, 1))
    cl, cd = o.forces(U, mach, 0.0)
    assert abs(cl) < 1e-14 and abs(cd) < 1e-14
    # p = p_inf + A sin(theta) on a circle of radius r: F_y = -A pi r
    A, r = 0.01, 0.5
    th = 2 * math.pi * np.arange(c.n) / c.n
    U = np.stack([O.prim_to_cons(1.0, 0.0, 0.0, 1 / GAMMA + A * math.sin(t)) for t in th])
    cl, cd = o.forces(U, mach, 0.0)
    assert abs(cl - (-A * math.pi * r) / (0.5 * mach * mach)) < 1e-4 * abs(cl)
    assert abs(cd) < 1e-12
    # the same load seen at an angle of attack rotates into drag and lift
    al = 10.0
    cl2, cd2 = o.forces(U, mach, al)
    assert abs(cl2 - cl * math.cos(math.radians(al))) < 1e-12
    assert abs(cd2 - cl * math.sin(math.radians(al))) < 1e-12


def test_symmetric_aerofoil_symmetric_state_has_no_lift():
    c = cg.naca0012_block(40, 16)
    o = O.Oracle(c)
    U = o.initial_state(0.5, 0.0)
    n_i = 40
    # a pressure field symmetric about the chord line
    for p in range(c.n):
        j, i = divmod(p, n_i)
        r, u, v, pp = O.cons_to_prim(U[p])
        i_m = (n_i - i) % n_i
        pp = 1 / GAMMA + 0.01 * math.cos(2 * math.pi * min(i, i_m) / n_i)
        U[p] = O.prim_to_cons(r, u, v, pp)
    cl, cd = o.forces(U, 0.5, 0.0)
    assert abs(cl) < 1e-14


def _perturbed_state(o, c, mach=0.5, aoa=1.0, amp=0.02):
    U = o.initial_state(mach, aoa)
    rng = np.random.default_rng(17)
    act = c.flag != 2
    U[act, 0] *= 1 + amp * rng.uniform(-1, 1, act.sum())
    U[act, 3] *= 1 + amp * rng.uniform(-1, 1, act.sum())
    return U


def test_implicit_increment_tends_to_the_explicit_step_as_cfl_vanishes():
    """As the pseudo-time step shrinks, the LU-SGS system's diagonal 1/dt
    dominates and its increment tends to the forward Euler step -dt R: their
    difference is O(dt^2), so relative to dt R it halves with the CFL."""
    c = cg.naca0012_block(24, 10)
    o = O.Oracle(c)
    U = _perturbed_state(o, c)
    q = o.q_from_state(U)
    z = np.zeros((c.n, 4))
    errs = []
    for cfl in (2e-3, 1e-3, 5e-4):
        R, D = o.residual(q, z, z, U, cfl)
        _, dU = o.sweeps(U, R, D)
        dE, _ = o.explicit_step(U, R, cfl)
        errs.append(np.max(np.abs(dU - dE)) / np.max(np.abs(dE)))
    assert errs[0] < 1e-2
    for a, b in zip(errs, errs[1:]):
        assert 1.7 < a / b < 2.3, errs


def test_explicit_solver_is_forward_euler():
    """Two explicit steps at CFL c/2 and one at CFL c differ by O(dt^2)
    (first-order residual, so every step is U - dt R(U)): the difference
    quarters when the CFL halves; and the increment is -dt R with the
    normal momentum removed at wall points."""
    c = cg.naca0012_block(24, 10)
    o = O.Oracle(c)
    U = _perturbed_state(o, c)
    diffs = []
    for cfl in (0.02, 0.01, 0.005):
        one = o.run_explicit(U, 1, cfl=cfl, K=0, first_order=10)["U"]
        two = o.run_explicit(U, 2, cfl=cfl / 2, K=0, first_order=10)["U"]
        diffs.append(np.max(np.abs(one - two)))
    for a, b in zip(diffs, diffs[1:]):
        assert 3.4 < a / b < 4.6, diffs
    q = o.q_from_state(U)
    z = np.zeros((c.n, 4))
    R, _ = o.residual(q, z, z, U, 0.3)
    dE, D = o.explicit_step(U, R, 0.3)
    wall = c.flag == 1
    assert np.max(np.abs(dE[wall, 1] * c.nx[wall] + dE[wall, 2] * c.ny[wall])) < 1e-15
    inner = c.flag == 0
    assert np.allclose(dE[inner], -R[inner] / D[inner, None], rtol=0, atol=1e-15)
    assert np.all(dE[c.flag == 2] == 0.0)


def test_revised_lusgs_diagonal_and_lag_term_closed_forms():
    """Manish et al.'s diagonal on the regular 3x3 stencil of spacing h is
    1/dt + (|u| + a)/h + (|v| + a)/h (each split sub-stencil has LS(1) = -+1/h),
    and the lagged term S vanishes there (mirror sub-stencils: LS+(1) =
    -LS-(1)); S is zero for a zero increment and linear in it."""
    n = 9
    c = cg.cartesian_box(n, n, jitter=0.0, seed=3)
    o = O.Oracle(c)
    h = 1.0 / (n - 1)
    rng = np.random.default_rng(5)
    U = np.array([O.prim_to_cons(1.1, 0.3, -0.2, 0.8)] * c.n)
    centre = int(np.argmin((c.x - 0.5) ** 2 + (c.y - 0.5) ** 2))
    cfl = 3.0
    a = math.sqrt(1.4 * 0.8 / 1.1)
    dU = rng.normal(0, 1e-3, (c.n, 4))
    D, S = o.manish_terms(U, cfl, dU)
    dt = cfl * h / (math.hypot(0.3, 0.2) + a)
    assert abs(D[centre] - (1 / dt + (0.3 + a) / h + (0.2 + a) / h)) < 1e-12 * D[centre]
    assert np.max(np.abs(S[centre])) < 1e-15
    cj = cg.cartesian_box(n, n, jitter=0.25, seed=3)  # skewed stencils: S != 0
    oj = O.Oracle(cj)
    Uj = np.array([O.prim_to_cons(1.1, 0.3, -0.2, 0.8)] * cj.n)
    dUj = rng.normal(0, 1e-3, (cj.n, 4))
    _, Sj = oj.manish_terms(Uj, cfl, dUj)
    assert np.max(np.abs(Sj)) > 1e-4
    _, S0 = oj.manish_terms(Uj, cfl, np.zeros((cj.n, 4)))
    assert np.all(S0 == 0.0)
    _, S2 = oj.manish_terms(Uj, cfl, 2 * dUj)
    assert np.max(np.abs(S2 - 2 * Sj)) < 1e-12 * np.max(np.abs(Sj))


def test_revised_lusgs_keeps_the_fixed_point():
    """At a converged state (R ~ 0, dU ~ 0) the revised sweeps' increment
    vanishes too: the lagged term only changes the path."""
    c = cg.naca0012_block(40, 16)
    o = O.Oracle(c)
    r = o.run(o.initial_state(0.63, 2.0), 6000, cfl=100.0, K=2, first_order=50, target=1e-10)
    assert r["status"] == 0 and r["hist"][-1] / r["hist0"] <= 1e-10
    m = o.run_manish(r["U"], 3, cfl=3.0, K=2, n0=100, sigma=-1)
    assert m["status"] == 0
    assert np.max(np.abs(m["U"] - r["U"])) < 1e-9 * np.max(np.abs(r["U"]))
