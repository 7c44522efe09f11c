"""The kernels' x/2 and 2x as integer steps of the exponent field (the FP64
multiplications by 1/2 and 2 of Eq. 14's inverse and of the Jacobian
tangents), emulated on the CPU bit for bit: the same bits as the FP64
multiplication for every normal input with a normal result, zeros and
non-finite values returned as they are."""
import numpy as np


def _step(x, up):
    """The device helper's rule: hi word +/- 2^20 when the exponent field
    is in [2, 0x7fe] (halving) or [1, 0x7fd] (doubling), else unchanged."""
    b = np.asarray(x, dtype=np.float64).view(np.uint64).copy()
    ex = (b >> np.uint64(52)) & np.uint64(0x7FF)
    if up:
        ok = (ex >= 1) & (ex <= 0x7FD)
        b[ok] += np.uint64(1 << 52)
    else:
        ok = (ex >= 2) & (ex <= 0x7FE)
        b[ok] -= np.uint64(1 << 52)
    return b.view(np.float64)


def _bits(a):
    return np.asarray(a, dtype=np.float64).view(np.uint64)


def test_steps_equal_the_multiplication_on_normals():
    rng = np.random.default_rng(7)
    # magnitudes across the whole normal range, both signs
    x = rng.choice([-1.0, 1.0], 200000) * np.ldexp(rng.uniform(1.0, 2.0, 200000), rng.integers(-1020, 1023, 200000))
    assert np.array_equal(_bits(_step(x, False)), _bits(x * 0.5))
    assert np.array_equal(_bits(_step(x, True)), _bits(x * 2.0))
    # the solver's own ranges: beta, 1/beta, rho |u|^2, increments near convergence
    y = np.concatenate([rng.uniform(1e-3, 1e3, 10000), -rng.uniform(1e-3, 1e3, 10000),
                        rng.uniform(1e-300, 1e-200, 1000), rng.normal(0, 1e-12, 1000)])
    assert np.array_equal(_bits(_step(y, False)), _bits(y * 0.5))
    assert np.array_equal(_bits(_step(y, True)), _bits(y * 2.0))


def test_zeros_and_non_finite_values_are_returned_unchanged():
    sp = np.array([0.0, -0.0, np.inf, -np.inf])
    for up, f in ((False, 0.5), (True, 2.0)):
        r = _step(sp, up)
        assert np.array_equal(_bits(r), _bits(sp))
        assert np.array_equal(_bits(r), _bits(sp * f))  # which is also the exact product
        n = _step(np.array([np.nan]), up)
        assert np.isnan(n[0])


def test_only_the_range_edges_differ_from_the_multiplication():
    """Halving of magnitudes below 2^-1021 (result subnormal), doubling of
    subnormal inputs and doubling above 2^1023 (result infinite) are left
    unscaled: the documented limits,
    far outside what a state, a q-derivative or an increment reaches."""
    tiny = np.array([np.ldexp(1.5, -1022), 5e-324, np.ldexp(1.0, -1021)])
    assert np.array_equal(_bits(_step(tiny[:2], False)), _bits(tiny[:2]))
    assert np.array_equal(_bits(_step(tiny[2:], False)), _bits(tiny[2:] * 0.5))
    # subnormal inputs (exponent field 0) are not doubled either
    sub = np.array([5e-324, np.ldexp(1.0, -1030), -np.ldexp(1.0, -1023)])
    assert np.array_equal(_bits(_step(sub, True)), _bits(sub))
    assert not np.any(_bits(sub * 2.0) == _bits(sub))
    huge = np.array([np.ldexp(1.5, 1023), np.ldexp(1.0, 1022)])
    with np.errstate(over="ignore"):
        assert _step(huge[:1], True)[0] == huge[0] and np.isinf(huge[0] * 2.0)
    assert np.array_equal(_bits(_step(huge[1:], True)), _bits(huge[1:] * 2.0))
