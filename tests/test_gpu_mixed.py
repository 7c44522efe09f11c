"""Mixed precision (FP32 LU-SGS sweeps and Jacobian products; residual with
compensated sums, norm and update in FP64) against the FP64 oracle.

The residual, the diagonal and the norm are FP64 on both sides, so they keep
the FP64 bars of test_gpu_parity.py.  The increments carry FP32 rounding:
each Jacobian product and sum has a relative error of a few 2^-24 ~ 6e-8 of
the terms it adds, so dU* and dU are compared normwise at 1e-5 (about 100
units of FP32 rounding, room for the sums over up to 20 neighbours and the
division by D).  Over many iterations the FP32 increments only change the
path, not the fixed point R = 0; the history is compared at 1e-4 relative and
the measured errors are printed.
"""
import numpy as np
import pytest

import oracle as O
from paper_2406_07441_gb300 import cloudgen as cg
from tests.conftest import cached_cloud

pytestmark = pytest.mark.gpu


def nrel(a, b):
    s = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (s if s > 0 else 1.0))


@pytest.mark.parametrize("name", ["ogrid40x16", "jit64x32", "naca160x64"])
@pytest.mark.parametrize("jvp", [0, 1])
def test_mixed_one_iteration(name, jvp):
    from paper_2406_07441_gb300 import lskum as lk
    builders = {"ogrid40x16": lambda: cg.naca0012_block(40, 16),
                "jit64x32": lambda: cg.naca0012_jittered(64, 32, seed=12),
                "naca160x64": lambda: cg.naca0012_block(160, 64)}
    c = cached_cloud(name, builders[name])
    s = lk.Solver(c, 0.63, 2.0, jvp=jvp, precision=1)
    o = O.Oracle(c)
    r = o.run(o.initial_state(0.63, 2.0), 1, cfl=100.0, K=3, jvp=jvp)
    assert s.run(1) == 1
    e = {k: nrel(s.field(f), r[v]) for k, f, v in (("R", lk.FIELD_R, "R"), ("dUs", lk.FIELD_DUS, "dUs"),
                                                    ("dU", lk.FIELD_DU, "dU"), ("U", lk.FIELD_U, "U"))}
    D = s.field(lk.FIELD_D)
    e["D"] = float(np.max(np.abs(D - r["D"]) / np.abs(r["D"])))
    print(name, jvp, e)
    assert e["R"] < 1e-10 and e["D"] < 1e-12
    assert e["dUs"] < 1e-5 and e["dU"] < 1e-5
    assert e["U"] < 1e-6


def test_mixed_history_config1():
    from paper_2406_07441_gb300 import lskum as lk
    c = cached_cloud("naca160x64", lambda: cg.naca0012_block(160, 64))
    s = lk.Solver(c, 0.63, 2.0, precision=1)
    o = O.Oracle(c)
    iters = 100
    r = o.run(o.initial_state(0.63, 2.0), iters, cfl=100.0, K=3)
    assert s.run(iters) == iters
    h = s.residuals()
    rel = np.abs(h - r["hist"]) / r["hist"]
    eu = nrel(s.field(lk.FIELD_U), r["U"])
    cl, cd = s.forces()
    clo, cdo = o.forces(r["U"], 0.63, 2.0)
    print("mixed vs FP64 oracle, 100 iterations: history max rel", rel.max(), "state", eu,
          "Cl", abs(cl - clo), "Cd", abs(cd - cdo))
    assert rel.max() < 1e-4
    assert eu < 1e-5
