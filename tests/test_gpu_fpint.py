"""The kernels' integer-pipe FP64 arithmetic on the GB300 itself, through the
C-ABI self-test entry: the integer multiply equals the FP64 unit's multiply
(and the host's IEEE multiply) bit for bit, special cases included; the
fixed-point exp and erfcx equal the same header compiled for the host bit
for bit (whose integer steps the CPU tests check against exact emulations
and mpmath)."""
import shutil

import numpy as np
import pytest

from paper_2406_07441_gb300 import lskum

pytestmark = pytest.mark.gpu


def _bits_equal(x, y):
    bx, by = np.asarray(x).view(np.uint64), np.asarray(y).view(np.uint64)
    return (bx == by) | (np.isnan(x) & np.isnan(y))


def test_integer_multiply_equals_the_fp64_unit():
    rng = np.random.default_rng(31)
    n = 1 << 20
    ea = rng.integers(1023 - 600, 1023 + 600, n, dtype=np.uint64)
    eb = rng.integers(1023 - 600, 1023 + 600, n, dtype=np.uint64)
    a = ((rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)) | (ea << np.uint64(52))
         | rng.integers(0, 1 << 52, n, dtype=np.uint64)).view(np.float64)
    b = ((rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)) | (eb << np.uint64(52))
         | rng.integers(0, 1 << 52, n, dtype=np.uint64)).view(np.float64)
    # exact ties, binade carries, zeros, subnormals, infinities, NaN, range edges
    odd = ((rng.integers(0, 1 << 51, 4096, dtype=np.uint64) << np.uint64(1)) | np.uint64(1))
    ties = ((np.uint64(1023) << np.uint64(52)) | odd).view(np.float64)
    sp = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, np.ldexp(1.0, -1022),
                   np.finfo(np.float64).max, np.ldexp(1.0, 511), np.ldexp(1.5, -512), 2.0, 0.5])
    sa, sb = np.meshgrid(sp, sp)
    a = np.concatenate([a, ties, np.nextafter(np.ldexp(1.0, rng.integers(-30, 30, 4096)), 0.0), sa.ravel()])
    b = np.concatenate([b, np.full(4096, 1.5), np.nextafter(np.ldexp(1.0, rng.integers(-30, 30, 4096)), 0.0),
                        sb.ravel()])
    got = lskum.selftest_fpint(lskum.FPINT_MUL, a, b)
    unit = lskum.selftest_fpint(lskum.FPINT_MUL_FP64, a, b)
    with np.errstate(all="ignore"):
        host = a * b
    assert np.all(_bits_equal(unit, host))
    assert np.all(_bits_equal(got, unit))


def test_fixed_point_exp_and_erfcx_equal_the_host_build():
    from test_fixmath_cpu import build_host_fns, erfcx_args
    fns = build_host_fns()
    if fns is None:
        pytest.skip("no host C++ compiler")
    host_erfcx, host_exp, tmp = fns
    try:
        rng = np.random.default_rng(32)
        x = np.concatenate([rng.uniform(-707.9, 707.9, 200000), -rng.uniform(0, 81, 200000),
                            rng.normal(0, 1e-6, 10000), [0.0, -0.0, 5e-324, 1e-300, -707.99, 707.99]])
        assert np.array_equal(lskum.selftest_fpint(lskum.FPINT_EXP, x).view(np.uint64),
                              host_exp(x).view(np.uint64))
        # beyond |x| = 708 the library's exp (within an ulp of the host's)
        big = np.array([-745.0, -720.0, -708.5, 708.5, 709.7])
        e = lskum.selftest_fpint(lskum.FPINT_EXP, big)
        assert np.all(np.abs(e - np.exp(big)) <= np.spacing(np.exp(big)) * 1.0 + 5e-324)
        s = np.concatenate([erfcx_args(), rng.uniform(0, 12, 100000), -rng.uniform(0, 9, 1000)])
        ref = host_erfcx(np.minimum(np.abs(s), 9.0))
        assert np.array_equal(lskum.selftest_fpint(lskum.FPINT_ERFCX_HALF, s).view(np.uint64), ref.view(np.uint64))
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
