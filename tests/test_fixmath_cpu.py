"""exp and erfcx on the integer pipes (csrc/lskum_fixmath.cuh): the header
compiled for the host with the generated tables gives bit for bit what exact
emulations of its integer steps give; erfcx is within the interpolant's own
error (6e-17) plus one rounding of erfcx(x)/2 by mpmath over the whole
clamped range [0, 9], interval edges and tiny arguments included (exp's
accuracy: test_fastmath_cpu)."""
import ctypes
import os
import shutil
import struct
import subprocess
import tempfile

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2406_07441_gb300", "csrc")

_SRC = r"""
#include <algorithm>
#include <cstdint>
using std::max;
#define __device__
#define __forceinline__ inline
#include "lskum_mathconst.h"
#include "lskum_fixmath.cuh"
extern "C" void exp_many(const double *x, double *r, long n)
{
    for (long k = 0; k < n; k++)
        r[k] = lskum::exp_fx<lskum::kExpShift>((const uint64_t *)lskum::kExpTableFx, lskum::kExpFxC, lskum::kExpFxL,
                                              x[k]);
}
extern "C" void erfcx_half_many(const double *x, double *r, long n)
{
    for (long k = 0; k < n; k++) {
        uint64_t b;
        memcpy(&b, &x[k], 8);
        const uint32_t ha = (uint32_t)(b >> 32), la = (uint32_t)b;
        const int iv = lskum::erfcx_interval((int)ha);
        r[k] = lskum::erfcx_half_fx<lskum::kErfcxDeg>(ha, la, iv, (const int64_t *)lskum::kErfcxFx[iv],
                                                      lskum::kErfcxFxShift[iv]);
    }
}
"""


def build_host_fns():
    """The header compiled for the host: (erfcx_half, exp) over float64
    arrays, and the temporary directory to remove; None without g++."""
    gxx = shutil.which("g++")
    if gxx is None:
        return None
    d = tempfile.mkdtemp()
    src, so = os.path.join(d, "h.cpp"), os.path.join(d, "libh.so")
    with open(src, "w") as f:
        f.write(_SRC)
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, src, "-o", so])
    lib = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.erfcx_half_many.argtypes = [dp, dp, ctypes.c_long]
    lib.exp_many.argtypes = [dp, dp, ctypes.c_long]

    def call(fn):
        def f(x):
            x = np.ascontiguousarray(x, dtype=np.float64)
            r = np.empty_like(x)
            fn(x.ctypes.data_as(dp), r.ctypes.data_as(dp), x.size)
            return r
        return f
    return call(lib.erfcx_half_many), call(lib.exp_many), d


@pytest.fixture(scope="module")
def host_fns():
    fns = build_host_fns()
    if fns is None:
        pytest.skip("no host C++ compiler")
    yield fns[:2]
    shutil.rmtree(fns[2], ignore_errors=True)


def erfcx_args():
    rng = np.random.default_rng(21)
    edges = []
    for e in range(-5, 4):  # the binade intervals' edges and their neighbours
        for m in range(16):
            a = 2.0 ** e * (1 + m / 16)
            edges += [a, np.nextafter(a, 0.0), np.nextafter(a, 10.0)]
    tiny = [0.0, 5e-324, 1e-300, 1e-20, 2.0 ** -17, 2.0 ** -6, np.nextafter(2.0 ** -5, 0.0)]
    return np.concatenate([rng.uniform(0.0, 9.0, 3000), np.exp(rng.uniform(np.log(1e-12), np.log(9.0), 2000)),
                           [x for x in edges if x <= 9.0], tiny, [9.0]])


def test_host_build_equals_the_exact_emulation(host_fns):
    from test_fastmath_cpu import erfcx_half_fx, exp_t
    x = erfcx_args()
    got = host_fns[0](x)
    ref = np.array([erfcx_half_fx(float(v)) for v in x])
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    rng = np.random.default_rng(22)
    y = np.concatenate([rng.uniform(-707.9, 707.9, 4000), -rng.uniform(0, 81, 4000), rng.normal(0, 1e-6, 500),
                        [0.0, -0.0, 5e-324, -5e-324, 1e-300, 707.99, -707.99, 1.0, -1.0]])
    got = host_fns[1](y)
    ref = np.array([exp_t(float(v)) for v in y])
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


def test_within_the_interpolant_error_and_one_rounding(host_fns):
    x = erfcx_args()
    got = host_fns[0](x)
    worst = 0.0
    with mp.workdps(40):
        for v, g in zip(x, got):
            ref = mp.exp(mp.mpf(float(v)) ** 2) * mp.erfc(mp.mpf(float(v))) / 2
            # error in units of the result's ulp
            worst = max(worst, float(abs(mp.mpf(float(g)) - ref) / mp.mpf(np.spacing(float(g)))))
    # 6e-17 relative (interpolant) is < 0.55 ulp; the final rounding adds 0.5
    assert worst <= 1.1, worst
