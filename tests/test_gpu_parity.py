"""CUDA path (through the C-ABI) against the FP64 CPU oracle, element by element.

Tolerances (derived from the arithmetic): the GPU evaluates the same
formulas with a different association of the same sums (per-slot LS weights
instead of the 2x2 solve of Eq. 11), fused multiply-adds, beta^(-5/2) instead
of exp(-ln(beta)/(gamma-1)) and CUDA's erf/exp/log (<= 2 ulp) instead of
glibc's.  Each evaluated quantity therefore differs by a few ulp of the terms
that form it.  A residual is a sum of differences of fluxes of size |G| times
weights of size 1/h, so its error is measured against max|R| over the cloud
(normwise), not per entry; the same for the increments.  Per iteration:
q-derivatives 1e-12, residual / increments / state 1e-10 (normwise),
diagonal 1e-12 (per entry, a sum of positive terms).  Histories and final
fields use the target tolerances of the plain FP64 path: 1e-10 relative per
history entry and 1e-9 normwise on the final state.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2406_07441_gb300 import cloudgen as cg
from tests.conftest import cached_cloud

pytestmark = pytest.mark.gpu


def _lskum():
    from paper_2406_07441_gb300 import lskum
    return lskum


def nrel(a, b):
    """normwise relative difference max|a - b| / max|b|"""
    s = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (s if s > 0 else 1.0))


CLOUDS = {
    "ogrid40x16": lambda: cg.naca0012_block(40, 16),
    "jit48x20": lambda: cg.naca0012_jittered(48, 20, seed=11),
    "jit64x32": lambda: cg.naca0012_jittered(64, 32, seed=12),
    "box9": lambda: cg.cartesian_box(9, 9, seed=2, wall_bottom=True),
    "naca160x64": lambda: cg.naca0012_block(160, 64),
}
COND = dict(mach=0.63, aoa_deg=2.0)


def _pair(name, jvp=0, K=3, cfl=100.0, **cond):
    cond = {**COND, **cond}
    c = cached_cloud(name, CLOUDS[name])
    s = _lskum().Solver(c, cond["mach"], cond["aoa_deg"], cfl=cfl, inner_iters=K, jvp=jvp)
    o = O.Oracle(c)
    return c, s, o, cond


@pytest.mark.parametrize("name", ["ogrid40x16", "jit48x20", "box9", "naca160x64"])
def test_colouring_and_sweep_order_match_oracle(name):
    c, s, o, _ = _pair(name)
    col, order, nc = s.order()
    assert nc == o.ncolours
    assert np.array_equal(col, o.colour)
    assert np.array_equal(order, o.order)


@pytest.mark.parametrize("name", ["ogrid40x16", "jit48x20", "box9", "naca160x64"])
@pytest.mark.parametrize("jvp", [0, 1])
def test_one_iteration_every_field(name, jvp):
    lk = _lskum()
    c, s, o, cond = _pair(name, jvp=jvp)
    U0 = o.initial_state(cond["mach"], cond["aoa_deg"])
    assert nrel(s.field(lk.FIELD_U), U0) < 1e-15
    r = o.run(U0, 1, cfl=100.0, K=3, jvp=jvp)
    assert r["status"] == 0
    assert s.run(1) == 1
    assert nrel(s.field(lk.FIELD_QX), r["qx"]) < 1e-12
    assert nrel(s.field(lk.FIELD_QY), r["qy"]) < 1e-12
    assert nrel(s.field(lk.FIELD_R), r["R"]) < 1e-10
    D = s.field(lk.FIELD_D)
    assert np.max(np.abs(D - r["D"]) / np.abs(r["D"])) < 1e-12
    assert nrel(s.field(lk.FIELD_DUS), r["dUs"]) < 1e-10
    assert nrel(s.field(lk.FIELD_DU), r["dU"]) < 1e-10
    assert nrel(s.field(lk.FIELD_U), r["U"]) < 1e-12
    assert nrel(s.field(lk.FIELD_Q), r["q"]) < 1e-12
    h = s.residuals()
    assert h.shape == (1,) and abs(h[0] - r["hist"][0]) <= 1e-12 * r["hist"][0]


def test_sweeps_from_the_same_residual_are_level_parallel_exact():
    """Sweep increments depend only on R, D and U: feeding the oracle the GPU's own
    R and D must reproduce the GPU's increments to rounding (checks the level
    schedule reproduces the sequential Gauss-Seidel order)."""
    lk = _lskum()
    c, s, o, cond = _pair("jit48x20")
    U0 = o.initial_state(cond["mach"], cond["aoa_deg"])
    s.run(1)
    R, D = s.field(lk.FIELD_R), s.field(lk.FIELD_D)
    dUs, dU = o.sweeps(U0, R, D, 0)
    assert nrel(s.field(lk.FIELD_DUS), dUs) < 1e-12
    assert nrel(s.field(lk.FIELD_DU), dU) < 1e-12


@pytest.mark.parametrize("shape", [None, (2, 32)])
@pytest.mark.parametrize("jvp,iters", [(0, 300), (1, 100)])
def test_history_and_final_fields_config1(jvp, iters, shape):
    """NACA 0012, 160x64 = 10,240 points, M = 0.63, AoA = 2 deg, CFL 100, in the
    context's default launch shape and in the packed sweeps at 2 threads per
    point."""
    lk = _lskum()
    c, s, o, cond = _pair("naca160x64", jvp=jvp)
    if shape is not None:
        s.set_launch_shape(*shape)
    r = _oracle_run(("naca160x64", jvp, iters), c, cond["mach"], cond["aoa_deg"], iters, cfl=100.0, K=3, jvp=jvp)
    assert r["status"] == 0 and r["done"] == iters
    assert s.run(iters) == iters
    h = s.residuals()
    rel = np.abs(h - r["hist"]) / r["hist"]
    assert rel.max() < 1e-10, (rel.argmax(), rel.max())
    assert nrel(s.field(lk.FIELD_U), r["U"]) < 1e-9
    cl, cd = s.forces()
    cl_o, cd_o = o.forces(r["U"], cond["mach"], cond["aoa_deg"])
    assert abs(cl - cl_o) < 1e-9 and abs(cd - cd_o) < 1e-9


def test_stops_at_the_same_iteration_as_the_oracle():
    c, s, o, cond = _pair("naca160x64")
    U0 = o.initial_state(cond["mach"], cond["aoa_deg"])
    r = o.run(U0, 100, cfl=100.0, K=3, target=0.4)
    assert r["status"] == 0
    done = s.run(100, target_drop=0.4)
    assert done == r["done"] < 100
    assert s.run(5) == 5  # a stopped run can be continued


@pytest.mark.parametrize("name,mach,aoa", [("jit64x32", 0.8, 1.25), ("naca160x64", 0.63, 2.0)])
def test_first_order_start_then_second_order(name, mach, aoa):
    """Iterations n <= first_order_iters use q~ = q; the switch happens at the same
    iteration on both sides."""
    lk = _lskum()
    c = cached_cloud(name, CLOUDS[name])
    s = lk.Solver(c, mach, aoa, first_order_iters=3)
    o = O.Oracle(c)
    r = o.run(o.initial_state(mach, aoa), 6, cfl=100.0, K=3, first_order=3)
    assert r["status"] == 0 and s.run(6) == 6
    h = s.residuals()
    assert np.max(np.abs(h - r["hist"]) / r["hist"]) < 1e-10
    assert nrel(s.field(lk.FIELD_U), r["U"]) < 1e-11
    assert nrel(s.field(lk.FIELD_R), r["R"]) < 1e-10


def test_checkpoint_resume_is_bitwise():
    lk = _lskum()
    c = cached_cloud("jit64x32", CLOUDS["jit64x32"])
    a = lk.Solver(c, 0.63, 2.0, first_order_iters=10)
    a.run(20)
    b = lk.Solver(c, 0.63, 2.0, first_order_iters=10)
    b.run(10)
    U10 = b.field(lk.FIELD_U)
    b2 = lk.Solver(c, 0.63, 2.0, first_order_iters=10)
    b2.run(10)
    b2.set_conserved(U10)
    b2.run(10)
    assert np.array_equal(a.field(lk.FIELD_U), b2.field(lk.FIELD_U))
    assert np.array_equal(a.residuals(), b2.residuals())


def test_enqueue_wait_equals_run():
    lk = _lskum()
    c = cached_cloud("ogrid40x16", CLOUDS["ogrid40x16"])
    a = lk.Solver(c, 0.63, 2.0)
    a.run(7)
    b = lk.Solver(c, 0.63, 2.0)
    b.enqueue(7)
    assert b.wait() == 7
    assert np.array_equal(a.field(lk.FIELD_U), b.field(lk.FIELD_U))


def test_set_state_round_trip_and_rejects_nonphysical():
    lk = _lskum()
    c = cached_cloud("ogrid40x16", CLOUDS["ogrid40x16"])
    s = lk.Solver(c, 0.5, 0.0)
    rho, u, v, p = s.get_state()
    assert np.allclose(rho, 1.0) and np.allclose(p[c.flag != cg.WALL], 1 / 1.4)
    bad = rho.copy()
    bad[7] = -1.0
    with pytest.raises(lk.LskumError) as ei:
        s.set_state(bad, u, v, p)
    assert ei.value.status == -3
    rho2, *_ = s.get_state()
    assert np.array_equal(rho2, rho)


_ORACLE_RUNS = {}


def _oracle_run(key, cloud, mach, aoa, iters, **kw):
    """One oracle run per (cloud, conditions), shared by the tests that need it."""
    if key not in _ORACLE_RUNS:
        o = O.Oracle(cloud)
        _ORACLE_RUNS[key] = o.run(o.initial_state(mach, aoa), iters, **kw)
    return _ORACLE_RUNS[key]


# Launch shapes (threads per point in the gradient and residual kernels, sweep
# lanes per point; 32 = the packed sweeps): the benchmark's autotuned choice on
# the 147,584- and 5,242,880-point clouds first (one thread per point, packed
# sweeps), the packed form at 2 and 4 threads per point (the autotuner's choice
# on other clouds and kernels), then the size-based default of a new context.
FULL_SIZE_SHAPES = [(1, 32), (2, 32), (4, 32), (1, 4)]


@pytest.mark.parametrize("jvp", [0, 1])
def test_config2_full_size(jvp):
    """Jittered 640x256 cloud, 10% removed: 147,584 points, M = 0.85, AoA = 1 deg,
    K = 2 (the benchmark's setting), each JVP mode: one first-order start-up
    iteration and two second-order ones, every field of the last against the
    oracle, in each launch shape of FULL_SIZE_SHAPES -- among them the packed
    sweeps at 1 thread per point that the benchmark times, at full size (all
    16 colour levels, framed-point warps spread over the grid, the interior
    groups of 20-slot lists)."""
    lk = _lskum()
    c = cached_cloud("jit640x256", lambda: cg.build_workload("naca0012_640x256_jit"))
    assert c.n == 147584
    r = _oracle_run(("jit640x256", jvp), c, 0.85, 1.0, 3, cfl=100.0, K=2, jvp=jvp, first_order=1)
    assert r["status"] == 0
    clo, cdo = O.Oracle(c).forces(r["U"], 0.85, 1.0)
    for tpp, lanes in FULL_SIZE_SHAPES:
        s = lk.Solver(c, 0.85, 1.0, inner_iters=2, jvp=jvp, first_order_iters=1)
        s.set_launch_shape(tpp, lanes)
        assert s.run(3) == 3
        shape = (tpp, lanes)
        assert nrel(s.field(lk.FIELD_QX), r["qx"]) < 1e-12, shape
        assert nrel(s.field(lk.FIELD_QY), r["qy"]) < 1e-12, shape
        assert nrel(s.field(lk.FIELD_R), r["R"]) < 1e-10, shape
        D = s.field(lk.FIELD_D)
        assert np.max(np.abs(D - r["D"]) / np.abs(r["D"])) < 1e-12, shape
        assert nrel(s.field(lk.FIELD_DUS), r["dUs"]) < 1e-10, shape
        assert nrel(s.field(lk.FIELD_DU), r["dU"]) < 1e-10, shape
        assert nrel(s.field(lk.FIELD_U), r["U"]) < 1e-12, shape
        assert nrel(s.field(lk.FIELD_Q), r["q"]) < 1e-12, shape
        h = s.residuals()
        assert np.max(np.abs(h - r["hist"]) / r["hist"]) < 1e-10, shape
        cl, cd = s.forces()
        assert abs(cl - clo) < 1e-11 and abs(cd - cdo) < 1e-11, shape
        del s


@pytest.mark.parametrize("tpp", [1, 2])
@pytest.mark.parametrize("jvp", [0, 1])
def test_packed_sweeps_history_41k_points(jvp, tpp):
    """The packed sweeps (1 or 2 threads per point in the gradient and
    residual kernels, the benchmark's shapes) on a jittered 336x136 cloud with
    10% removed (41,264 points, 14+ colour levels with many framed-point warps
    each): 40 iterations (20 first-order start-up, 20 second-order) against
    the oracle: history 1e-10 per entry, final state 1e-9, Cl / Cd 1e-9."""
    lk = _lskum()
    c = cached_cloud("jit336x136", lambda: cg.naca0012_jittered(336, 136, seed=cg.BASE_SEED + 21))
    assert c.n > 40000
    r = _oracle_run(("jit336x136", jvp), c, 0.8, 1.25, 40, cfl=100.0, K=2, jvp=jvp, first_order=20)
    assert r["status"] == 0 and r["done"] == 40
    s = lk.Solver(c, 0.8, 1.25, inner_iters=2, jvp=jvp, first_order_iters=20)
    s.set_launch_shape(tpp, 32)
    assert s.run(40) == 40
    h = s.residuals()
    rel = np.abs(h - r["hist"]) / r["hist"]
    assert rel.max() < 1e-10, (rel.argmax(), rel.max())
    assert nrel(s.field(lk.FIELD_U), r["U"]) < 1e-9
    cl, cd = s.forces()
    clo, cdo = O.Oracle(c).forces(r["U"], 0.8, 1.25)
    assert abs(cl - clo) < 1e-9 and abs(cd - cdo) < 1e-9


@pytest.mark.slow
@pytest.mark.skipif(os.environ.get("LSKUM_FULL_SIZE") != "1",
                    reason="5.24M-point cloud: about 5 minutes of host time; set LSKUM_FULL_SIZE=1")
def test_config3_full_size_fp64_and_mixed():
    """Jittered 2560x2048 cloud, nothing removed: 5,242,880 points, M = 0.8,
    AoA = 1.25 deg, exact JVPs: one first-order start-up iteration and one
    second-order one, plain FP64 and FP32 sweeps, every field of the last
    against the FP64 oracle."""
    lk = _lskum()
    c = cg.build_workload("naca0012_2560x2048_jit")
    assert c.n == 5242880
    o = O.Oracle(c)
    r = o.run(o.initial_state(0.8, 1.25), 2, cfl=100.0, K=3, first_order=1)
    assert r["status"] == 0
    for prec in (0, 1):
        s = lk.Solver(c, 0.8, 1.25, first_order_iters=1, precision=prec)
        assert s.run(2) == 2
        e = {k: nrel(s.field(f), r[v]) for k, f, v in (("R", lk.FIELD_R, "R"), ("dUs", lk.FIELD_DUS, "dUs"),
                                                        ("dU", lk.FIELD_DU, "dU"), ("U", lk.FIELD_U, "U"))}
        h = s.residuals()
        e["hist"] = float(np.max(np.abs(h - r["hist"]) / r["hist"]))
        rho, u, v, p = s.get_state()
        Uo = r["U"]
        rho_o = Uo[:, 0]
        p_o = 0.4 * (Uo[:, 3] - 0.5 * (Uo[:, 1] ** 2 + Uo[:, 2] ** 2) / rho_o)
        e["rho"] = float(np.max(np.abs(rho - rho_o)))
        e["p"] = float(np.max(np.abs(p - p_o)))
        cl, cd = s.forces()
        clo, cdo = o.forces(Uo, 0.8, 1.25)
        e["Cl"], e["Cd"] = abs(cl - clo), abs(cd - cdo)
        print("precision", prec, e)
        if prec == 0:
            assert e["R"] < 1e-10 and e["hist"] < 1e-10
            assert e["dUs"] < 1e-10 and e["dU"] < 1e-10 and e["U"] < 1e-12
        else:
            # the second residual is evaluated at the state the FP32 sweeps
            # produced (state error ~3e-8), so it inherits that error
            assert e["R"] < 1e-6 and e["hist"] < 1e-6
            assert e["dUs"] < 1e-5 and e["dU"] < 1e-5 and e["U"] < 1e-6
        del s


def test_device_pointer_variants_equal_the_host_ones():
    """lskum_get_field_dev / lskum_set_conserved_dev on torch CUDA tensors give
    bit for bit what the host calls give, FP64 and FP32-sweep contexts."""
    torch = pytest.importorskip("torch")
    lk = _lskum()
    c = cached_cloud("jit64x32", lambda: cg.naca0012_jittered(64, 32, seed=12))
    for prec in (0, 1):
        s = lk.Solver(c, 0.6, 1.5, first_order_iters=2, precision=prec)
        assert s.run(4) == 4
        st = torch.cuda.Stream()
        for f in range(8):
            shape = (c.n,) if f == lk.FIELD_D else (c.n, 4)
            t = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            s.field_dev(f, t.data_ptr(), st.cuda_stream)
            st.synchronize()
            assert np.array_equal(t.cpu().numpy(), s.field(f)), f
        U = s.field(lk.FIELD_U)
        s2 = lk.Solver(c, 0.6, 1.5, first_order_iters=2, precision=prec)
        s3 = lk.Solver(c, 0.6, 1.5, first_order_iters=2, precision=prec)
        s2.set_conserved(U)
        Ud = torch.from_numpy(U).cuda()
        torch.cuda.synchronize()
        s3.set_conserved_dev(Ud.data_ptr(), None)
        assert np.array_equal(s2.field(lk.FIELD_U), s3.field(lk.FIELD_U))
        assert s2.run(3) == 3 and s3.run(3) == 3
        assert np.array_equal(s2.field(lk.FIELD_U), s3.field(lk.FIELD_U))


@pytest.mark.parametrize("name", ["ogrid40x16", "jit64x32"])
def test_explicit_scheme_matches_oracle(name):
    """The explicit solver (forward Euler, the implicit scheme's local time
    step, no sweeps): one iteration's fields and a 40-iteration history."""
    lk = _lskum()
    c = cached_cloud(name, CLOUDS[name])
    o = O.Oracle(c)
    U0 = o.initial_state(0.5, 1.0)
    s = lk.Solver(c, 0.5, 1.0, cfl=0.3, inner_iters=2, first_order_iters=10, scheme=lk.SCHEME_EXPLICIT)
    r = o.run_explicit(U0, 1, cfl=0.3, K=2, first_order=10)
    assert s.run(1) == 1
    assert nrel(s.field(lk.FIELD_R), r["R"]) < 1e-10
    D = s.field(lk.FIELD_D)
    assert np.max(np.abs(D - r["D"]) / np.abs(r["D"])) < 1e-12
    assert nrel(s.field(lk.FIELD_DU), r["dU"]) < 1e-10
    assert nrel(s.field(lk.FIELD_U), r["U"]) < 1e-12
    s2 = lk.Solver(c, 0.5, 1.0, cfl=0.3, inner_iters=2, first_order_iters=10, scheme=lk.SCHEME_EXPLICIT)
    r2 = o.run_explicit(U0, 40, cfl=0.3, K=2, first_order=10)
    assert r2["status"] == 0 and s2.run(40) == 40
    h = s2.residuals()
    assert np.max(np.abs(h - r2["hist"]) / r2["hist"]) < 1e-10
    assert nrel(s2.field(lk.FIELD_U), r2["U"]) < 1e-9
    assert s2.info()["launches_per_iter"] < lk.Solver(c, 0.5, 1.0).info()["launches_per_iter"]


@pytest.mark.parametrize("name", ["ogrid40x16", "jit64x32"])
def test_revised_lusgs_matches_oracle(name):
    """The revised LU-SGS of Manish et al. (Jameson diagonal, lagged S term):
    fields of the first iteration (S = 0) and of the fifth (S from the fourth
    iteration's increment), and the history."""
    lk = _lskum()
    c = cached_cloud(name, CLOUDS[name])
    o = O.Oracle(c)
    U0 = o.initial_state(0.63, 2.0)
    for iters in (1, 5):
        s = lk.Solver(c, 0.63, 2.0, cfl=3.0, inner_iters=2, first_order_iters=2, lusgs=lk.LUSGS_MANISH)
        r = o.run_manish(U0, iters, cfl=3.0, K=2, first_order=2, sigma=-1)
        assert r["status"] == 0 and s.run(iters) == iters
        D = s.field(lk.FIELD_D)
        assert np.max(np.abs(D - r["D"]) / np.abs(r["D"])) < 1e-12
        assert nrel(s.field(lk.FIELD_R), r["R"]) < 1e-10
        assert nrel(s.field(lk.FIELD_DUS), r["dUs"]) < 1e-10
        assert nrel(s.field(lk.FIELD_DU), r["dU"]) < 1e-10
        assert nrel(s.field(lk.FIELD_U), r["U"]) < 1e-12
        h = s.residuals()
        assert np.max(np.abs(h - r["hist"]) / r["hist"]) < 1e-10


@pytest.mark.parametrize("name", ["ogrid40x16", "jit64x32"])
def test_wall_first_ordering_matches_oracle(name):
    """Alg. 4's order (wall points colour by colour, then interior points):
    the library's sweep order equals the oracle's, and an iteration's fields
    and a 20-iteration history match."""
    lk = _lskum()
    c = cached_cloud(name, CLOUDS[name])
    o = O.Oracle(c, ordering=1)
    s = lk.Solver(c, 0.63, 2.0, inner_iters=2, first_order_iters=3, ordering=lk.ORDER_WALL_FIRST)
    col, order, nc = s.order()
    assert nc == o.ncolours and np.array_equal(col, o.colour) and np.array_equal(order, o.order)
    r = o.run(o.initial_state(0.63, 2.0), 1, cfl=100.0, K=2, first_order=3)
    assert s.run(1) == 1
    assert nrel(s.field(lk.FIELD_DUS), r["dUs"]) < 1e-10
    assert nrel(s.field(lk.FIELD_DU), r["dU"]) < 1e-10
    assert nrel(s.field(lk.FIELD_U), r["U"]) < 1e-12
    s2 = lk.Solver(c, 0.63, 2.0, inner_iters=2, first_order_iters=3, ordering=lk.ORDER_WALL_FIRST)
    r2 = o.run(o.initial_state(0.63, 2.0), 20, cfl=100.0, K=2, first_order=3)
    assert s2.run(20) == 20
    h = s2.residuals()
    assert np.max(np.abs(h - r2["hist"]) / r2["hist"]) < 1e-10
    assert s2.info()["launches_per_iter"] >= lk.Solver(c, 0.63, 2.0, inner_iters=2).info()["launches_per_iter"]


def test_four_component_residual_history():
    """Column 0 of the four-component history is the density history bit for
    bit; the last row holds the norms of the oracle's last residual (wall and
    interior points) for all four components."""
    lk = _lskum()
    c = cached_cloud("jit64x32", CLOUDS["jit64x32"])
    o = O.Oracle(c)
    s = lk.Solver(c, 0.63, 2.0, first_order_iters=2)
    r = o.run(o.initial_state(0.63, 2.0), 6, cfl=100.0, K=3, first_order=2)
    assert s.run(6) == 6
    h4 = s.residuals4()
    assert h4.shape == (6, 4)
    assert np.array_equal(h4[:, 0], s.residuals())
    act = c.flag != 2
    ref = np.sqrt(np.sum(r["R"][act] ** 2, axis=0))
    assert np.max(np.abs(h4[-1] - ref) / ref) < 1e-10


@pytest.mark.parametrize("jvp", [0, 1])
def test_packed_sweeps_match_oracle(jvp):
    """The packed sweep form (sweep_lanes = 32: each point's axis Jacobian
    products formed once and gathered by interior points, four lanes per
    interior point; wall points one lane per slot in packed warps with
    segmented sums): one iteration's increments and a 30-iteration history
    against the oracle, FP64 and mixed precision."""
    lk = _lskum()
    c = cached_cloud("jit64x32", CLOUDS["jit64x32"])
    o = O.Oracle(c)
    U0 = o.initial_state(0.63, 2.0)
    r = o.run(U0, 1, cfl=100.0, K=3, jvp=jvp, first_order=10)
    s = lk.Solver(c, 0.63, 2.0, jvp=jvp, first_order_iters=10)
    s.set_launch_shape(2, 32)
    assert s.run(1) == 1
    assert nrel(s.field(lk.FIELD_DUS), r["dUs"]) < 1e-10
    assert nrel(s.field(lk.FIELD_DU), r["dU"]) < 1e-10
    assert nrel(s.field(lk.FIELD_U), r["U"]) < 1e-12
    r2 = o.run(U0, 30, cfl=100.0, K=3, jvp=jvp, first_order=10)
    assert r2["status"] == 0
    for precision, bar in ((0, 1e-10), (1, 1e-4)):
        s2 = lk.Solver(c, 0.63, 2.0, jvp=jvp, first_order_iters=10, precision=precision)
        s2.set_launch_shape(4, 32)
        assert s2.run(30) == 30
        h = s2.residuals()
        assert np.max(np.abs(h - r2["hist"]) / r2["hist"]) < bar
    # the launch count of the lanes-per-point form, plus (exact products) the
    # kernel forming the framed points' Jacobians before the forward sweep
    base = lk.Solver(c, 0.63, 2.0, jvp=jvp).info()["launches_per_iter"]
    assert s2.info()["launches_per_iter"] == base + (1 if jvp == 0 else 0)


def test_packed_sweeps_kinetic_and_batch():
    """Packed sweeps with the kinetic far field (outer points in the lists)
    and in a batch (frozen cases skip their points): equal to the
    lanes-per-point form to rounding and to single solves bit for bit."""
    lk = _lskum()
    c1 = cg.naca0012_block(40, 16, kinetic_outer=True)
    c2 = cg.naca0012_jittered(48, 20, seed=11, kinetic_outer=True)
    kw = dict(inner_iters=2, first_order_iters=3, farfield=lk.FARFIELD_KINETIC)
    a = lk.Solver(c1, 1.2, 0.0, **kw)
    b = lk.Solver(c1, 1.2, 0.0, **kw)
    a.set_launch_shape(2, 8)
    b.set_launch_shape(2, 32)
    assert a.run(10) == 10 and b.run(10) == 10
    assert nrel(b.field(lk.FIELD_U), a.field(lk.FIELD_U)) < 1e-12
    assert np.max(np.abs(b.residuals() - a.residuals()) / a.residuals()) < 1e-11
    conds = [(1.2, 0.0), (0.63, 2.0)]
    bt = lk.Solver.batch([c1, c2], conds, **kw)
    bt.set_launch_shape(2, 32)
    assert bt.run(6) == 6
    U = bt.field(lk.FIELD_U)
    for cs, (c, (m, al)) in enumerate(zip([c1, c2], conds)):
        s = lk.Solver(c, m, al, **kw)
        s.set_launch_shape(2, 32)
        assert s.run(6) == 6
        info = bt.case_info(cs)
        assert np.array_equal(U[info["first_point"]:info["first_point"] + c.n], s.field(lk.FIELD_U))


def test_packed_sweeps_wall_first_and_manish():
    """The packed form under the wall-first order (levels split by point
    type) and with the revised LU-SGS (its lagged term in the first lane of
    each point): increments against the oracle."""
    lk = _lskum()
    c = cached_cloud("ogrid40x16", CLOUDS["ogrid40x16"])
    o1 = O.Oracle(c, ordering=1)
    r = o1.run(o1.initial_state(0.63, 2.0), 4, cfl=100.0, K=2, first_order=2)
    s = lk.Solver(c, 0.63, 2.0, inner_iters=2, first_order_iters=2, ordering=lk.ORDER_WALL_FIRST)
    s.set_launch_shape(2, 32)
    assert s.run(4) == 4
    assert nrel(s.field(lk.FIELD_DUS), r["dUs"]) < 1e-10 and nrel(s.field(lk.FIELD_DU), r["dU"]) < 1e-10
    o = O.Oracle(c)
    r = o.run_manish(o.initial_state(0.63, 2.0), 5, cfl=3.0, K=2, first_order=2, sigma=-1)
    s = lk.Solver(c, 0.63, 2.0, cfl=3.0, inner_iters=2, first_order_iters=2, lusgs=lk.LUSGS_MANISH)
    s.set_launch_shape(2, 32)
    assert s.run(5) == 5
    assert nrel(s.field(lk.FIELD_DUS), r["dUs"]) < 1e-10 and nrel(s.field(lk.FIELD_DU), r["dU"]) < 1e-10
    h = s.residuals()
    assert np.max(np.abs(h - r["hist"]) / r["hist"]) < 1e-10


@pytest.mark.parametrize("name", ["ogrid40x16", "box9"])
def test_serial_order_matches_oracle(name):
    """The serial sweeps of Alg. 2 (wall, interior, outer points in index
    order), run level by level over their dependency graph: the same order as
    the oracle's sequential sweeps, one iteration's increments and a
    20-iteration history."""
    lk = _lskum()
    c = cached_cloud(name, CLOUDS[name])
    o = O.Oracle(c, ordering=2)
    s = lk.Solver(c, 0.63, 2.0, inner_iters=2, first_order_iters=3, ordering=lk.ORDER_SERIAL)
    col, order, nc = s.order()
    assert np.array_equal(order, o.order)
    U0 = o.initial_state(0.63, 2.0)
    r = o.run(U0, 1, cfl=100.0, K=2, first_order=3)
    assert s.run(1) == 1
    assert nrel(s.field(lk.FIELD_DUS), r["dUs"]) < 1e-10
    assert nrel(s.field(lk.FIELD_DU), r["dU"]) < 1e-10
    assert nrel(s.field(lk.FIELD_U), r["U"]) < 1e-12
    s.set_launch_shape(2, 32)
    r2 = o.run(r["U"], 19, cfl=100.0, K=2, first_order=3, n0=1, hist0=r["hist0"])
    assert r2["status"] == 0 and s.run(19) == 19
    h = s.residuals()
    ref = np.concatenate([r["hist"], r2["hist"]])
    assert np.max(np.abs(h - ref) / ref) < 1e-10
