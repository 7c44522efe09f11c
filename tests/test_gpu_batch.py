"""Batched solves: several (cloud, free stream) cases in one context.

The batch is the disjoint union of the cases' clouds; Alg. 5 colours each
component exactly as it would alone and every point's arithmetic is the same,
so each case must reproduce its own single-case solve (same launch shape:
all clouds here use the same threads-per-point choice), and a case that
reaches its drop target must stop while the others go on."""
import numpy as np
import pytest

import oracle as O
from paper_2406_07441_gb300 import cloudgen as cg
from tests.conftest import cached_cloud

pytestmark = pytest.mark.gpu

CASES = [("ogrid40x16", lambda: cg.naca0012_block(40, 16), (0.5, 0.0)),
         ("jit64x32", lambda: cg.naca0012_jittered(64, 32, seed=12), (0.8, 1.25)),
         ("ogrid48x20", lambda: cg.naca0012_block(48, 20), (0.63, 2.0))]


def _clouds():
    return [cached_cloud(n, b) for n, b, _ in CASES], [c for _, _, c in CASES]


def test_batch_cases_equal_their_single_solves():
    from paper_2406_07441_gb300 import lskum as lk
    clouds, conds = _clouds()
    kw = dict(first_order_iters=3, cfl=100.0, inner_iters=3)
    b = lk.Solver.batch(clouds, conds, **kw)
    assert b.run(8) == 8
    Ub = b.field(lk.FIELD_U)
    for cs, (c, (m, a)) in enumerate(zip(clouds, conds)):
        s = lk.Solver(c, m, a, **kw)
        assert s.run(8) == 8
        info = b.case_info(cs)
        sl = slice(info["first_point"], info["first_point"] + info["n_points"])
        assert info["n_points"] == c.n and info["iters"] == 8
        assert np.array_equal(Ub[sl], s.field(lk.FIELD_U))
        assert np.array_equal(b.case_residuals(cs), s.residuals())
        assert b.case_forces(cs) == s.forces()


def test_batch_case_matches_oracle():
    from paper_2406_07441_gb300 import lskum as lk
    clouds, conds = _clouds()
    b = lk.Solver.batch(clouds, conds, first_order_iters=3)
    assert b.run(5) == 5
    c, (m, a) = clouds[1], conds[1]
    o = O.Oracle(c)
    r = o.run(o.initial_state(m, a), 5, cfl=100.0, K=3, first_order=3)
    h = b.case_residuals(1)
    assert np.max(np.abs(h - r["hist"]) / r["hist"]) < 1e-10
    info = b.case_info(1)
    U = b.field(lk.FIELD_U)[info["first_point"]:info["first_point"] + c.n]
    assert np.max(np.abs(U - r["U"])) / np.max(np.abs(r["U"])) < 1e-11


def test_batch_cases_stop_independently():
    from paper_2406_07441_gb300 import lskum as lk
    clouds, conds = _clouds()
    kw = dict(first_order_iters=3)
    target = 0.5
    singles = []
    for c, (m, a) in zip(clouds, conds):
        s = lk.Solver(c, m, a, **kw)
        singles.append((s.run(60, target_drop=target), s))
    b = lk.Solver.batch(clouds, conds, **kw)
    done = b.run(60, target_drop=target)
    assert done == max(n for n, _ in singles)
    Ub = b.field(lk.FIELD_U)
    for cs, (n, s) in enumerate(singles):
        info = b.case_info(cs)
        assert info["iters"] == n and info["stopped"]
        sl = slice(info["first_point"], info["first_point"] + info["n_points"])
        assert np.array_equal(Ub[sl], s.field(lk.FIELD_U))


def test_autotune_restores_the_state():
    """The autotuner times real iterations under every launch shape and then
    restores state, counters and history: a solve that autotunes half way
    follows the plain solve (launch shapes change only the order of
    floating-point sums)."""
    from paper_2406_07441_gb300 import lskum as lk
    clouds, conds = _clouds()
    kw = dict(first_order_iters=3)
    b = lk.Solver.batch(clouds, conds, **kw)
    ref = lk.Solver.batch(clouds, conds, **kw)
    assert b.run(4) == 4 and ref.run(8) == 8
    U4 = b.field(lk.FIELD_U)
    h4 = [b.case_residuals(cs) for cs in range(len(clouds))]
    tpp, lanes, ms = b.autotune(3)
    print("autotune:", tpp, lanes, ms)
    assert tpp in (1, 2, 4, 8) and lanes in (2, 4, 8, 32) and ms > 0
    assert np.array_equal(b.field(lk.FIELD_U), U4)
    for cs in range(len(clouds)):
        assert np.array_equal(b.case_residuals(cs), h4[cs]) and b.case_info(cs)["iters"] == 4
    assert b.run(4) == 4
    for cs in range(len(clouds)):
        h, hr = b.case_residuals(cs), ref.case_residuals(cs)
        assert np.max(np.abs(h - hr) / hr) < 1e-10
    Ur = ref.field(lk.FIELD_U)
    assert np.max(np.abs(b.field(lk.FIELD_U) - Ur)) / np.max(np.abs(Ur)) < 1e-11


def _low_pressure_blob(c, U, fac=1e-2):
    """The free stream with the pressure of the interior points near
    (1.5, 0) cut by `fac`: a physical state whose update turns non-physical
    within a few iterations at CFL 100 (the oracle fails in iteration 4)."""
    V = U.copy()
    blob = (np.abs(c.x - 1.5) < 0.6) & (np.abs(c.y) < 0.6) & (c.flag == 0)
    ke = 0.5 * (V[:, 1] ** 2 + V[:, 2] ** 2) / V[:, 0]
    p = 0.4 * (V[:, 3] - ke)
    V[:, 3] = np.where(blob, p * fac, p) / 0.4 + ke
    return V


def test_failed_case_keeps_its_last_good_state_and_others_go_on():
    from paper_2406_07441_gb300 import lskum as lk
    clouds, conds = _clouds()
    kw = dict(first_order_iters=3)
    U0 = [O.Oracle(c).initial_state(m, a) for c, (m, a) in zip(clouds, conds)]
    U0[2] = _low_pressure_blob(clouds[2], U0[2])
    o = O.Oracle(clouds[2])
    r = o.run(U0[2], 8, cfl=100.0, K=3, first_order=3)
    assert r["status"] < 0 and r["done"] == 4  # fails in its 4th update
    singles = []
    for c, (m, a), U in zip(clouds, conds, U0):
        s = lk.Solver(c, m, a, **kw)
        s.set_conserved(U)
        try:
            s.run(8)
            err = 0
        except lk.LskumError as ex:
            err = ex.status
        singles.append((err, s.field(lk.FIELD_U), s.residuals()))
    assert [e for e, _, _ in singles] == [0, 0, lk.ERR_NONPOSITIVE]
    b = lk.Solver.batch(clouds, conds, **kw)
    b.set_conserved(np.concatenate(U0))
    assert b.run(8) == 8
    Ub = b.field(lk.FIELD_U)
    for cs, (err, U, h) in enumerate(singles):
        info = b.case_info(cs)
        sl = slice(info["first_point"], info["first_point"] + info["n_points"])
        assert info["status"] == err
        assert np.array_equal(Ub[sl], U)  # failed case: its last good state
        assert np.array_equal(b.case_residuals(cs), h)
        if err:
            assert info["stopped"] and info["iters"] == 4
            assert info["first_point"] <= info["bad_point"] < info["first_point"] + info["n_points"]
    # a failed case stays frozen in the next run; the others continue
    assert b.run(2) == 2
    assert b.case_info(2)["iters"] == 4 and b.case_info(0)["iters"] == 10
    assert np.array_equal(b.field(lk.FIELD_U)[b.case_info(2)["first_point"]:], singles[2][1])


@pytest.mark.parametrize("opts", [dict(precision=1), dict(lusgs=1, cfl=3.0), dict(ordering=1),
                                  dict(scheme=1, cfl=0.3), dict(precision=1, ordering=1, jvp=1)])
def test_batch_equals_single_solves_for_every_option(opts):
    """Every solver option keeps the batch property: each case of a batch is
    bit for bit its own single-case solve (same launch shape)."""
    from paper_2406_07441_gb300 import lskum as lk
    clouds, conds = _clouds()
    kw = dict(first_order_iters=3, inner_iters=2, **opts)
    b = lk.Solver.batch(clouds, conds, **kw)
    assert b.run(6) == 6
    Ub = b.field(lk.FIELD_U)
    for cs, (c, (m, a)) in enumerate(zip(clouds, conds)):
        s = lk.Solver(c, m, a, **kw)
        assert s.run(6) == 6
        info = b.case_info(cs)
        sl = slice(info["first_point"], info["first_point"] + info["n_points"])
        assert np.array_equal(Ub[sl], s.field(lk.FIELD_U)), (opts, cs)
        assert np.array_equal(b.case_residuals(cs), s.residuals())
