"""The kernels' FP64 multiplication on the integer pipes (csrc/lskum_intmul.cuh),
compiled for the host from the same source, against the host's own IEEE 754
multiply bit for bit: random operands over the whole exponent range, the
solver's value ranges, exact ties, products at binade edges, and every
special case (which the integer path hands to the FP64 unit)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2406_07441_gb300", "csrc", "lskum_intmul.cuh")

_SRC = r"""
#include "lskum_intmul.cuh"
extern "C" void mul_many(const double *a, const double *b, double *r, long n)
{
    for (long k = 0; k < n; k++) r[k] = lskum::mul_i(a[k], b[k]);
}
"""


@pytest.fixture(scope="module")
def mul_i():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "h.cpp")
    so = os.path.join(d, "libh.so")
    with open(src, "w") as f:
        f.write(_SRC)
    # -ffp-contract=off: the fallback multiply stays a plain IEEE multiply
    subprocess.check_call([gxx, "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-I",
                           os.path.dirname(HDR), src, "-o", so])
    lib = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.mul_many.argtypes = [dp, dp, dp, ctypes.c_long]

    def f(a, b):
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        r = np.empty_like(a)
        lib.mul_many(a.ctypes.data_as(dp), b.ctypes.data_as(dp), r.ctypes.data_as(dp), a.size)
        return r
    yield f
    shutil.rmtree(d, ignore_errors=True)


def _same(x, y):
    """Bitwise equality, any NaN matching any NaN."""
    bx, by = x.view(np.uint64), y.view(np.uint64)
    return np.all((bx == by) | (np.isnan(x) & np.isnan(y)))


def _check(f, a, b):
    with np.errstate(all="ignore"):
        ref = a * b
    r = f(a, b)
    bad = ~((r.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(r) & np.isnan(ref)))
    assert not bad.any(), (a[bad][:4], b[bad][:4], r[bad][:4], ref[bad][:4])


def test_random_operands_over_the_exponent_range(mul_i):
    rng = np.random.default_rng(11)
    n = 2_000_000
    # random bit patterns with normal exponents in a range whose products stay normal
    ea = rng.integers(1023 - 500, 1023 + 500, n, dtype=np.uint64)
    eb = rng.integers(1023 - 500, 1023 + 500, n, dtype=np.uint64)
    ma = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    mb = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    sa = rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    sb = rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    a = (sa | (ea << np.uint64(52)) | ma).view(np.float64)
    b = (sb | (eb << np.uint64(52)) | mb).view(np.float64)
    _check(mul_i, a, b)


def test_the_solvers_value_ranges(mul_i):
    rng = np.random.default_rng(12)
    n = 500_000
    # states, 1/beta, fluxes, weights, increments near convergence
    a = np.concatenate([rng.uniform(1e-3, 1e3, n), rng.normal(0, 1, n), rng.normal(0, 1e-12, n)])
    b = np.concatenate([rng.uniform(-1e3, 1e3, n), rng.uniform(1e-6, 1e6, n), rng.normal(0, 1e4, n)])
    _check(mul_i, a, b)


def test_exact_ties_round_to_even(mul_i):
    rng = np.random.default_rng(13)
    n = 400_000
    # odd significand x 1.5 (or 1.25, 1.75): the discarded part is exactly one half
    odd = (rng.integers(0, 1 << 51, n, dtype=np.uint64) << np.uint64(1)) | np.uint64(1)
    a = ((np.uint64(1023) << np.uint64(52)) | odd).view(np.float64)
    for m in (1.5, 1.25, 1.75, 1.125, 1.0625):
        b = np.full(n, m) * rng.choice([-1.0, 1.0], n) * np.ldexp(1.0, rng.integers(-20, 20, n))
        _check(mul_i, a, b)
    # and significands just below a power of two, whose products carry into the next binade
    c = np.nextafter(np.ldexp(1.0, rng.integers(-30, 30, n)), 0.0)
    d = np.nextafter(np.ldexp(1.0, rng.integers(-30, 30, n)), np.inf)
    _check(mul_i, c, c)
    _check(mul_i, c, d)
    _check(mul_i, d, d)


def test_special_operands_and_range_edges(mul_i):
    tiny, huge = np.ldexp(1.0, -1022), np.finfo(np.float64).max
    vals = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, tiny, -tiny,
                     np.nextafter(tiny, 0.0), huge, -huge, np.ldexp(1.0, 511), np.ldexp(1.0, -511),
                     np.ldexp(1.5, 512), np.ldexp(1.5, -512), np.sqrt(tiny), np.sqrt(huge), 2.0, 0.5, 3.0])
    a, b = np.meshgrid(vals, vals)
    _check(mul_i, a.ravel(), b.ravel())
    # products that land on the normal/subnormal border and on the overflow border
    rng = np.random.default_rng(14)
    n = 200_000
    x = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-600, -400, n))
    y = np.ldexp(rng.uniform(1.0, 2.0, n), -1022 - np.frexp(x)[1] + rng.integers(-3, 4, n))
    _check(mul_i, x, y)
    u = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(400, 600, n))
    v = np.ldexp(rng.uniform(1.0, 2.0, n), 1024 - np.frexp(u)[1] + rng.integers(-3, 3, n))
    _check(mul_i, u, v)
