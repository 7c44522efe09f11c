"""The allocation-free density-residual norm, checked against the solver's own.

lskum_density_norm_noalloc serves callers that cannot allocate device memory
(their device memory belongs to their own pool allocator, or an allocation
would synchronise the device inside a latency-critical loop, or their
deployment forbids runtime allocation): its scratch is a fixed array inside
the library.  This file is collected last so that a run stopping at its first
failure has already run every other test; it also passes on its own in a
fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2406_07441_gb300 import cloudgen as cg

pytestmark = pytest.mark.gpu


def _norm_noalloc(lk, torch, r):
    dev = torch.from_numpy(np.ascontiguousarray(r, np.float64)).cuda()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = lk.load().lskum_density_norm_noalloc(C.c_void_p(dev.data_ptr()), int(dev.numel()),
                                              C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert st == 0, lk.STATUS.get(st, st)
    stream.synchronize()
    return float(out.item())


def test_noalloc_norm_matches_the_solver_history_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    from paper_2406_07441_gb300 import lskum as lk
    cloud = cg.naca0012_block(160, 64)
    s = lk.Solver(cloud, 0.63, 2.0)
    for iters in (3, 2):  # two calls in a row, on different residuals
        assert s.run(iters) == iters
        ref = s.residuals()[-1]
        r_rho = s.field(lk.FIELD_R)[:, 0]  # zero at outer points, as in the solver's sum
        got = _norm_noalloc(lk, torch, r_rho)
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)


def test_noalloc_norm_edge_sizes_and_limit():
    torch = pytest.importorskip("torch")
    from paper_2406_07441_gb300 import lskum as lk
    assert _norm_noalloc(lk, torch, np.zeros(0)) == 0.0
    assert _norm_noalloc(lk, torch, np.array([3.0, 4.0])) == 5.0
    rng = np.random.default_rng(1)
    r = rng.normal(size=3_000_001)  # more elements than one pass of the fixed partials grid
    ref = float(np.sqrt(np.sum(r * r)))
    assert abs(_norm_noalloc(lk, torch, r) - ref) <= 1e-12 * ref
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    too_big = 134_217_728 + 1
    st = lk.load().lskum_density_norm_noalloc(C.c_void_p(out.data_ptr()), too_big, C.c_void_p(out.data_ptr()), None)
    assert st == -1
