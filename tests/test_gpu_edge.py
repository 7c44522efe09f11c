"""Edge cases of the CUDA path: a cloud with no active point, zero-iteration
runs, a one-case batch, a 32-point cloud (one full ELL slice, no ragged
tail) and a 33-point one (a ragged tail of one point), each against the
oracle or against its definition."""
import numpy as np
import pytest

import oracle as O
from paper_2406_07441_gb300 import cloudgen as cg
from tests.conftest import cached_cloud

pytestmark = pytest.mark.gpu


def _lk():
    from paper_2406_07441_gb300 import lskum as lk
    return lk


def test_cloud_without_active_points_keeps_the_free_stream():
    lk = _lk()
    c = cg.cartesian_box(6, 6, seed=4)
    c.flag[:] = 2  # all outer: nothing is swept or updated
    s = lk.Solver(c, 0.5, 1.0)
    U0 = s.field(lk.FIELD_U)
    assert s.run(3) == 3
    assert np.array_equal(s.field(lk.FIELD_U), U0)
    assert np.all(s.residuals() == 0.0)


def test_zero_iterations_change_nothing():
    lk = _lk()
    c = cached_cloud("ogrid40x16", lambda: cg.naca0012_block(40, 16))
    s = lk.Solver(c, 0.63, 2.0)
    assert s.run(2) == 2
    U, h = s.field(lk.FIELD_U), s.residuals()
    assert s.run(0) == 0
    assert np.array_equal(s.field(lk.FIELD_U), U) and np.array_equal(s.residuals(), h)


def test_one_case_batch_equals_a_single_context():
    lk = _lk()
    c = cached_cloud("jit64x32", lambda: cg.naca0012_jittered(64, 32, seed=12))
    kw = dict(first_order_iters=3, inner_iters=2)
    b = lk.Solver.batch([c], [(0.7, 1.5)], **kw)
    s = lk.Solver(c, 0.7, 1.5, **kw)
    assert b.run(6) == 6 and s.run(6) == 6
    assert np.array_equal(b.field(lk.FIELD_U), s.field(lk.FIELD_U))
    assert np.array_equal(b.case_residuals(0), s.residuals())


@pytest.mark.parametrize("n,m,wall", [(8, 4, True), (11, 3, False)])
def test_full_and_ragged_slices_match_the_oracle(n, m, wall):
    """8x4 = 32 points with a flat wall (exactly one ELL slice) and 11x3 = 33
    points (a one-point ragged slice): one iteration, every field."""
    lk = _lk()
    c = cg.cartesian_box(n, m, seed=6, wall_bottom=wall)
    assert c.n in (32, 33)
    o = O.Oracle(c)
    U0 = o.initial_state(0.4, 3.0)
    r = o.run(U0, 1, cfl=20.0, K=2, first_order=0)
    s = lk.Solver(c, 0.4, 3.0, cfl=20.0, inner_iters=2)
    assert r["status"] == 0 and s.run(1) == 1
    for f, k in ((lk.FIELD_R, "R"), (lk.FIELD_DUS, "dUs"), (lk.FIELD_DU, "dU"), (lk.FIELD_U, "U")):
        got, ref = s.field(f), r[k]
        scale = max(np.max(np.abs(ref)), 1e-300)
        assert np.max(np.abs(got - ref)) / scale < 1e-10, k


def test_host_io_modes_give_the_same_bits():
    """Host arrays through the staging copies and, where the device reads and
    writes pageable host memory, straight through the reorder kernels: the
    same state, fields and history, bit for bit; a mode the device does not
    support is refused."""
    from paper_2406_07441_gb300 import cloudgen as cg
    from paper_2406_07441_gb300 import lskum as lk
    c = cg.naca0012_jittered(48, 20, seed=11)
    direct, supported = lk.Solver(c, 0.63, 2.0).host_io()
    assert direct == 0
    out = []
    for mode in ((0, 1) if supported else (0,)):
        s = lk.Solver(c, 0.63, 2.0, first_order_iters=3)
        s.set_host_io(mode)
        assert s.host_io() == (mode, supported)
        assert s.run(5) == 5
        U = s.field(lk.FIELD_U)
        s.set_conserved(U * 1.0)
        assert s.run(2) == 2
        out.append((s.field(lk.FIELD_U), s.field(lk.FIELD_QX), s.field(lk.FIELD_DU), s.get_state()[3], s.residuals()))
    for a, b in zip(out[0], out[-1]):
        assert np.array_equal(a, b)
    if not supported:
        with pytest.raises(lk.LskumError):
            lk.Solver(c, 0.63, 2.0).set_host_io(1)
