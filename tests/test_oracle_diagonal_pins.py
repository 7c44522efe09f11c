"""Pins of the oracle's local time step and scalar LU-SGS diagonal (Eq. 26 with
Eq. 33-34, readings R6 and R7, the kinetic far field's ghost sub-stencil R12).

The oracle forms D_0 = 1/dt_0 - sum_s sigma_s rho_s LS_s(1) from its own
closed-form 2x2 least-squares sums and raises it to sum_s rho_s sum_i |w_i|
where the split weights mix signs.  These tests check that value against
two things the oracle does not use:

* a closed form on the regular 3x3 stencil of spacing h, where every split
  sub-stencil has three points, LS_+(1) = -1/h, LS_-(1) = +1/h and
  sum |w| = |LS(1)|, so the cap cannot bind:
  D = (|u| + a)/(CFL h) + (max(u + a, 0) + max(a - u, 0)
                           + max(v + a, 0) + max(a - v, 0)) / h;
* an independent restatement per point of every cloud kind (interior, wall
  points in their (t, n) frame with only the fluid-side n- sub-stencil,
  outer points under the kinetic far field with the n+ sub-stencil and the
  free-stream ghosts at the mirror images of its points): sub-stencil
  membership from the offsets, the least-squares weights of Eq. 11 solved by
  numpy's pseudo-inverse from the coordinates, the ghosts built as explicit
  mirrored points, and the local time step from the nearest neighbour.

States are drawn so that some points are supersonic in either direction
(rho_s clipped to 0) and, on skewed stencils at CFL 100, the cap binds at
many points.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2406_07441_gb300 import cloudgen as cg

GAMMA = 1.4


def _prim(U):
    rho = U[0]
    u, v = U[1] / rho, U[2] / rho
    p = (GAMMA - 1.0) * (U[3] - 0.5 * rho * (u * u + v * v))
    return rho, u, v, p


def _independent_diagonal(cloud, U, cfl, kinetic):
    """Per point: (D, cap binds?) from the paper's formula, computed without
    the oracle's least-squares sums."""
    n = cloud.n
    D = np.empty(n)
    capped = np.zeros(n, dtype=bool)
    for p in range(n):
        fl = cloud.flag[p]
        if fl == cg.OUTER and not kinetic:
            D[p] = 1.0  # frozen free stream: not an unknown
            continue
        if fl == cg.INTERIOR:
            e1, e2 = np.array([1.0, 0.0]), np.array([0.0, 1.0])
        else:  # wall: n into the fluid; kinetic outer: n out of the domain
            nrm = np.array([cloud.nx[p], cloud.ny[p]])
            e1, e2 = np.array([nrm[1], -nrm[0]]), nrm
        nb = cloud.nbr_idx[cloud.nbr_off[p]:cloud.nbr_off[p + 1]]
        off = np.stack([cloud.x[nb] - cloud.x[p], cloud.y[nb] - cloud.y[p]], axis=1)
        dmin = np.min(np.hypot(off[:, 0], off[:, 1]))
        a = off @ e1
        b = off @ e2
        # (offsets along the derivative direction, along the other one, sign, direction)
        subs = [(a[a < 0], b[a < 0], +1, e1), (a[a > 0], b[a > 0], -1, e1)]
        if fl != cg.WALL:
            subs.append((b[b < 0], a[b < 0], +1, e2))
        if fl != cg.OUTER:
            subs.append((b[b > 0], a[b > 0], -1, e2))
        else:
            # ghosts at the mirror images (a, -b) of the n+ points: an n- stencil
            subs.append((-b[b < 0], a[b < 0], -1, e2))
        rho, u, v, pr = _prim(U[p])
        snd = math.sqrt(GAMMA * pr / rho)
        lin = (math.hypot(u, v) + snd) / (cfl * dmin)
        dom = 0.0
        for d, dp, sign, e in subs:
            w = np.linalg.pinv(np.stack([d, dp], axis=1))[0]  # least-squares d/de weights
            ud = u * e[0] + v * e[1]
            rs = max(ud + snd, 0.0) if sign > 0 else max(snd - ud, 0.0)
            lin -= sign * rs * np.sum(w)
            dom += rs * np.sum(np.abs(w))
        D[p] = max(lin, dom)
        capped[p] = dom > lin
    return D, capped


def _random_states(n, rng, smax=1.8):
    rho = rng.uniform(0.7, 1.3, n)
    p = rng.uniform(0.5, 1.0, n)
    a = np.sqrt(GAMMA * p / rho)
    u = rng.uniform(-smax, smax, n) * a
    v = rng.uniform(-smax, smax, n) * a
    return np.array([O.prim_to_cons(*s) for s in zip(rho, u, v, p)])


def test_diagonal_closed_form_on_the_regular_stencil():
    n = 9
    c = cg.cartesian_box(n, n, jitter=0.0, seed=3)
    o = O.Oracle(c)
    h = 1.0 / (n - 1)
    centre = int(np.argmin((c.x - 0.5) ** 2 + (c.y - 0.5) ** 2))
    assert c.nbr_off[centre + 1] - c.nbr_off[centre] == 8
    # subsonic, supersonic in +x, in -x, in +y, in both: each max(., 0) branch
    for rho, u, v, p, cfl in ((1.1, 0.3, -0.2, 0.8, 3.0), (0.9, 1.6, 0.1, 0.7, 100.0),
                              (1.2, -1.5, 0.4, 0.6, 100.0), (1.0, 0.2, 1.4, 0.75, 10.0),
                              (1.0, -1.3, -1.3, 0.5, 100.0)):
        U = np.array([O.prim_to_cons(rho, u, v, p)] * c.n)
        _, D = o.residual(o.q_from_state(U), np.zeros((c.n, 4)), np.zeros((c.n, 4)), U, cfl)
        a = math.sqrt(GAMMA * p / rho)
        dt = cfl * h / (math.hypot(u, v) + a)
        ref = 1.0 / dt + (max(u + a, 0.0) + max(a - u, 0.0) + max(v + a, 0.0) + max(a - v, 0.0)) / h
        assert abs(D[centre] - ref) <= 1e-13 * ref, (D[centre], ref)


@pytest.mark.parametrize("which,kinetic,cfl", [
    ("box_jitter", False, 100.0), ("box_jitter", False, 0.5), ("box_wall", False, 100.0),
    ("box_kinetic", True, 100.0), ("box_kinetic", True, 0.5), ("jit_kinetic", True, 100.0),
    ("jit_kinetic", True, 0.5), ("ogrid", False, 100.0)])
def test_diagonal_against_an_independent_least_squares_restatement(which, kinetic, cfl):
    clouds = {
        "box_jitter": lambda: cg.cartesian_box(9, 8, jitter=0.3, seed=4),
        "box_wall": lambda: cg.cartesian_box(9, 8, jitter=0.3, seed=5, wall_bottom=True),
        "box_kinetic": lambda: cg.cartesian_box(9, 8, jitter=0.3, seed=6, kinetic_outer=True),
        "jit_kinetic": lambda: cg.naca0012_jittered(48, 20, seed=11, kinetic_outer=True),
        "ogrid": lambda: cg.naca0012_block(40, 16),
    }
    c = clouds[which]()
    rng = np.random.default_rng(17)
    U = _random_states(c.n, rng)
    kw = dict(farfield=O.FARFIELD_KINETIC, mach=0.6, aoa_deg=1.0) if kinetic else {}
    o = O.Oracle(c, **kw)
    z = np.zeros((c.n, 4))
    _, D = o.residual(o.q_from_state(U), z, z, U, cfl)
    ref, capped = _independent_diagonal(c, U, cfl, kinetic)
    rel = np.abs(D - ref) / np.abs(ref)
    assert rel.max() < 1e-12, (int(rel.argmax()), rel.max())
    active = (c.flag != cg.OUTER) | kinetic
    if cfl >= 100.0 and which != "ogrid":
        assert capped[active].mean() > 0.2  # the cap of R6 is exercised
    if cfl < 1.0:
        assert not capped.any()  # a small step dominates: the plain Eq. 26 value
    if which in ("box_wall", "jit_kinetic"):
        assert np.any(c.flag == cg.WALL)

