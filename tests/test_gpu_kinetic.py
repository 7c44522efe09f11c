"""The kinetic far field (outer points updated; the incoming half-flux from
free-stream ghosts) through the C-ABI against the FP64 CPU oracle.

Bars as in test_gpu_parity.py (same arithmetic, re-associated): per
iteration residual / increments normwise 1e-10, diagonal 1e-12 per entry,
state 1e-12 normwise; histories 1e-10 relative per entry.  Mixed precision:
the bars of test_gpu_mixed.py.
"""
import numpy as np
import pytest

import oracle as O
from paper_2406_07441_gb300 import cloudgen as cg
from tests.conftest import cached_cloud

pytestmark = pytest.mark.gpu

CLOUDS = {
    "ogrid40x16k": lambda: cg.naca0012_block(40, 16, kinetic_outer=True),
    "jit48x20k": lambda: cg.naca0012_jittered(48, 20, seed=11, kinetic_outer=True),
    "box9k": lambda: cg.cartesian_box(9, 9, seed=2, wall_bottom=True, kinetic_outer=True),
    "box9free": lambda: cg.cartesian_box(9, 9, seed=2, kinetic_outer=True),
    "naca160x64k": lambda: cg.naca0012_block(160, 64, kinetic_outer=True),
}


def _lk():
    from paper_2406_07441_gb300 import lskum
    return lskum


def nrel(a, b):
    s = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (s if s > 0 else 1.0))


def _pair(name, mach, aoa, **kw):
    lk = _lk()
    c = cached_cloud(name, CLOUDS[name])
    s = lk.Solver(c, mach, aoa, farfield=lk.FARFIELD_KINETIC, **kw)
    o = O.Oracle(c, ordering=kw.get("ordering", 0), farfield=O.FARFIELD_KINETIC, mach=mach, aoa_deg=aoa)
    return c, s, o


def test_kinetic_free_stream_is_exact():
    lk = _lk()
    c, s, o = _pair("box9free", 1.2, 3.0)
    U0 = s.field(lk.FIELD_U)
    assert s.run(2) == 2
    assert np.all(s.field(lk.FIELD_R) == 0.0)
    assert np.all(s.field(lk.FIELD_DU) == 0.0)
    assert np.array_equal(s.field(lk.FIELD_U), U0)
    assert np.all(s.field(lk.FIELD_D)[c.flag == cg.OUTER] > 1.0)


# (the coarse 48x20 jittered cloud leaves the Maxwellian range at its leading
# edge when second order starts at M 1.2 -- oracle and library alike -- so it
# runs the subsonic condition only)
@pytest.mark.parametrize("name,mach,aoa", [("ogrid40x16k", 1.2, 0.0), ("ogrid40x16k", 0.63, 2.0),
                                           ("jit48x20k", 0.63, 2.0), ("box9k", 1.2, 5.0), ("box9k", 0.63, 2.0)])
def test_kinetic_one_iteration_and_history(name, mach, aoa):
    lk = _lk()
    c, s, o = _pair(name, mach, aoa, inner_iters=2, first_order_iters=3)
    U0 = o.initial_state(mach, aoa)
    assert nrel(s.field(lk.FIELD_U), U0) < 1e-15
    r = o.run(U0, 1, cfl=100.0, K=2, first_order=3)
    assert s.run(1) == 1
    out = c.flag == cg.OUTER
    assert nrel(s.field(lk.FIELD_R), r["R"]) < 1e-10
    D = s.field(lk.FIELD_D)
    assert np.max(np.abs(D - r["D"]) / np.abs(r["D"])) < 1e-12
    assert nrel(s.field(lk.FIELD_DUS), r["dUs"]) < 1e-10
    assert nrel(s.field(lk.FIELD_DU), r["dU"]) < 1e-10
    assert nrel(s.field(lk.FIELD_U), r["U"]) < 1e-12
    c, s2, o = _pair(name, mach, aoa, inner_iters=2, first_order_iters=3)
    r2 = o.run(U0, 20, cfl=100.0, K=2, first_order=3)
    assert r2["status"] == 0 and s2.run(20) == 20
    assert np.abs(s2.field(lk.FIELD_U)[out] - U0[out]).max() > 0  # the outer points move
    h = s2.residuals()
    assert np.max(np.abs(h - r2["hist"]) / r2["hist"]) < 1e-10
    assert nrel(s2.field(lk.FIELD_U), r2["U"]) < 1e-9
    act = np.ones(c.n, bool)  # outer points are counted in the norms
    assert np.max(np.abs(s2.residuals4()[-1] - np.sqrt(np.sum(r2["R"][act] ** 2, axis=0)))
                  / np.sqrt(np.sum(r2["R"] ** 2, axis=0))) < 1e-10


@pytest.mark.parametrize("variant", ["manish", "explicit", "wall_first", "increment"])
def test_kinetic_with_each_option(variant):
    lk = _lk()
    name, mach, aoa, iters = "ogrid40x16k", 1.2, 0.0, 12
    kw = dict(inner_iters=2, first_order_iters=3)
    if variant == "explicit":  # (at M 1.2 the explicit start fails at the trailing edge, oracle and library alike)
        mach, aoa = 0.63, 2.0
    if variant == "manish":
        kw.update(lusgs=lk.LUSGS_MANISH, cfl=3.0)
    elif variant == "explicit":
        kw.update(scheme=lk.SCHEME_EXPLICIT, cfl=0.3)
    elif variant == "wall_first":
        kw.update(ordering=lk.ORDER_WALL_FIRST)
    else:
        kw.update(jvp=lk.JVP_INCREMENT)
    c, s, o = _pair(name, mach, aoa, **kw)
    U0 = o.initial_state(mach, aoa)
    cfl = kw.get("cfl", 100.0)
    if variant == "manish":
        r = o.run_manish(U0, iters, cfl=cfl, K=2, first_order=3, sigma=-1)
    elif variant == "explicit":
        r = o.run_explicit(U0, iters, cfl=cfl, K=2, first_order=3)
    else:
        r = o.run(U0, iters, cfl=cfl, K=2, first_order=3, jvp=kw.get("jvp", 0))
    assert r["status"] == 0 and s.run(iters) == iters
    h = s.residuals()
    assert np.max(np.abs(h - r["hist"]) / r["hist"]) < 1e-10
    assert nrel(s.field(lk.FIELD_DU), r["dU"]) < 1e-9
    assert nrel(s.field(lk.FIELD_U), r["U"]) < 1e-10


def test_kinetic_mixed_precision():
    lk = _lk()
    c, s, o = _pair("ogrid40x16k", 1.2, 0.0, inner_iters=2, first_order_iters=3, precision=1)
    U0 = o.initial_state(1.2, 0.0)
    r = o.run(U0, 1, cfl=100.0, K=2, first_order=3)
    assert s.run(1) == 1
    assert nrel(s.field(lk.FIELD_R), r["R"]) < 1e-10
    assert nrel(s.field(lk.FIELD_DUS), r["dUs"]) < 1e-5 and nrel(s.field(lk.FIELD_DU), r["dU"]) < 1e-5
    c, s2, o = _pair("ogrid40x16k", 1.2, 0.0, inner_iters=2, first_order_iters=3, precision=1)
    r2 = o.run(U0, 40, cfl=100.0, K=2, first_order=3)
    assert s2.run(40) == 40
    assert np.max(np.abs(s2.residuals() - r2["hist"]) / r2["hist"]) < 1e-4


def test_kinetic_batch_cases_equal_their_single_solves():
    """Each case's ghosts hold its own free stream."""
    lk = _lk()
    names = ["ogrid40x16k", "jit48x20k", "box9k"]
    clouds = [cached_cloud(n, CLOUDS[n]) for n in names]
    conds = [(1.2, 0.0), (0.63, 2.0), (1.5, -3.0)]
    kw = dict(inner_iters=2, first_order_iters=3, farfield=lk.FARFIELD_KINETIC)
    b = lk.Solver.batch(clouds, conds, **kw)
    assert b.run(8) == 8
    Ub = b.field(lk.FIELD_U)
    for cs, (c, (m, a)) in enumerate(zip(clouds, conds)):
        s = lk.Solver(c, m, a, **kw)
        assert s.run(8) == 8
        info = b.case_info(cs)
        sl = slice(info["first_point"], info["first_point"] + info["n_points"])
        assert np.array_equal(Ub[sl], s.field(lk.FIELD_U))
        assert np.array_equal(b.case_residuals(cs), s.residuals())


def test_kinetic_supersonic_naca0012_160x64():
    """M 1.2, AoA 0 (the paper's supersonic case) on the 10,240-point O-grid:
    300 iterations (50 first order, K = 2) against the oracle; Cl ~ 0 by
    symmetry."""
    lk = _lk()
    c, s, o = _pair("naca160x64k", 1.2, 0.0, inner_iters=2, first_order_iters=50)
    r = o.run(o.initial_state(1.2, 0.0), 300, cfl=100.0, K=2, first_order=50)
    assert r["status"] == 0 and s.run(300) == 300
    h = s.residuals()
    rel = np.abs(h - r["hist"]) / r["hist"]
    assert rel.max() < 1e-9, rel.max()
    assert nrel(s.field(lk.FIELD_U), r["U"]) < 1e-8
    cl, cd = s.forces()
    clo, cdo = o.forces(r["U"], 1.2, 0.0)
    print("M 1.2 kinetic far field, 300 iterations: history max rel", rel.max(), "Cl", cl, clo, "Cd", cd, cdo)
    assert abs(cd - cdo) < 1e-8 and abs(cl) < 1e-4


def _polygon_normals(c, flags):
    """Central-difference normals of the closed polygons of the given point
    types in index order (right-hand normal of a counter-clockwise polygon)."""
    nx, ny = np.zeros(c.n), np.zeros(c.n)
    for f in flags:
        v = np.flatnonzero(c.flag == f)
        x, y = c.x[v], c.y[v]
        orient = 1.0 if np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y) > 0 else -1.0
        tx, ty = np.roll(x, -1) - np.roll(x, 1), np.roll(y, -1) - np.roll(y, 1)
        ln = np.hypot(tx, ty)
        nx[v], ny[v] = orient * ty / ln, -orient * tx / ln
    return nx, ny


def test_normals_computed_by_the_library():
    """With nx = ny = NULL the library computes the normals from the wall
    polygon (and, under the kinetic far field, the outer polygon): the same
    solve, bit for bit, as with those normals computed here.  (The outer
    ring's polygon normals differ from the generator's radial ones by
    rounding, which can move a neighbour lying on a normal line into or out
    of a tangential sub-stencil, so the two are not compared.)"""
    lk = _lk()
    c = cached_cloud("ogrid40x16k", CLOUDS["ogrid40x16k"])
    bare = cg.Cloud(c.x, c.y, c.flag, None, None, c.nbr_off, c.nbr_idx, {})
    for flags, kw, cond in (((cg.WALL,), dict(), (0.63, 2.0)),
                            ((cg.WALL, cg.OUTER), dict(farfield=lk.FARFIELD_KINETIC), (1.2, 0.0))):
        nx, ny = _polygon_normals(c, flags)
        given = cg.Cloud(c.x, c.y, c.flag, nx, ny, c.nbr_off, c.nbr_idx, {})
        a = lk.Solver(given, *cond, inner_iters=2, first_order_iters=3, **kw)
        b = lk.Solver(bare, *cond, inner_iters=2, first_order_iters=3, **kw)
        assert a.run(10) == 10 and b.run(10) == 10
        assert np.array_equal(a.field(lk.FIELD_U), b.field(lk.FIELD_U))
        assert np.array_equal(a.residuals(), b.residuals())
    # the generator's wall normals are this formula
    nx, ny = _polygon_normals(c, (cg.WALL,))
    w = c.flag == cg.WALL
    assert np.array_equal(nx[w], c.nx[w]) and np.array_equal(ny[w], c.ny[w])
