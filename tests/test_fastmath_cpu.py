"""The kernels' own exp and A = (1 + s erf S)/2, emulated on the CPU step by
step (the fixed-point integer steps of exp and of the erfcx polynomial
exactly, multiplications rounded once) with the constants of the generated
header, against mpmath at 60 digits."""
import functools
import os
import re
import struct

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2406_07441_gb300", "csrc", "lskum_mathconst.h")


def _consts():
    s = open(HDR).read()

    def scalar(name):
        return float.fromhex(re.search(name + r" = ([-0-9a-fx.p+]+);", s).group(1))

    def array(name):
        body = re.search(name + r"\[[^=]*\] = \{(.*?)\};", s, re.S).group(1)
        return [float.fromhex(t) for t in re.findall(r"-?0x[0-9a-f.]+p[-+]?\d+", body)]

    deg = int(re.search(r"kErfcxDeg = (\d+);", s).group(1))
    nI = int(re.search(r"kErfcxIntervals = (\d+);", s).group(1))
    body = re.search(r"kErfcxFx\[[^=]*\] = \{(.*?)\n\};", s, re.S).group(1)
    ecx = [[int(v) for v in re.findall(r"-?\d+(?=ll)", row)] for row in body.strip().split("\n")]
    assert len(ecx) == nI and all(len(r) == deg + 1 for r in ecx)
    esh = [int(v) for v in re.search(r"kErfcxFxShift\[[^=]*\] = \{(.*?)\};", s).group(1).split(",")]
    eshift = int(re.search(r"kErfcxShift = (\d+);", s).group(1))
    key0 = int(re.search(r"kErfcxKey0 = (0x[0-9a-f]+);", s).group(1), 16)
    n = int(re.search(r"kExpN = (\d+);", s).group(1))
    shift = int(re.search(r"kExpShift = (\d+);", s).group(1))
    cfx = int(re.search(r"kExpFxC = (\d+)ull;", s).group(1))
    lfx = int(re.search(r"kExpFxL = (\d+)ull;", s).group(1))
    tab = [int(v) for v in re.findall(r"(\d+)ull", re.search(r"kExpTableFx\[[^=]*\] = \{(.*?)\};", s, re.S).group(1))]
    assert len(tab) == n
    eshift = int(re.search(r"kErfcxShift = (\d+);", s).group(1))
    key0 = int(re.search(r"kErfcxKey0 = (0x[0-9a-f]+);", s).group(1), 16)
    return dict(cfx=cfx, lfx=lfx, n=n, shift=shift, tab=tab, ecx=ecx, esh=esh, deg=deg, eshift=eshift, key0=key0)

C = _consts()
# exact products and sums of doubles (rounded once by float()) need ~2 x 53
# bits plus the exponent spread; 300 bits, set locally so that no other test
# module's precision leaks in
PREC = 300


def fma(a, b, c):
    with mp.workprec(PREC):
        return float(mp.mpf(a) * mp.mpf(b) + mp.mpf(c))


def mul(a, b):
    with mp.workprec(PREC):
        return float(mp.mpf(a) * mp.mpf(b))


def hi_word(x):
    return struct.unpack(">i", struct.pack(">d", x)[:4])[0]


def lo_word(x):
    return struct.unpack(">i", struct.pack(">d", x)[4:])[0]


def from_words(h, l):
    return struct.unpack(">d", struct.pack(">ii", h, l))[0]


def exp_t(x):
    """exp(x) by the kernels' fixed-point integer steps, exactly."""
    M64 = 2 ** 64 - 1
    X = struct.unpack(">Q", struct.pack(">d", x))[0]
    hx, lx = X >> 32, X & 0xFFFFFFFF
    ex = (hx >> 20) & 0x7FF
    if (hx & 0x7FFFFFFF) >= 0x40862000:
        return float(mp.exp(mp.mpf(x)))  # the library's exp takes |x| >= 708
    M = (((hx & 0xFFFFF) | (0x100000 if ex else 0)) << 32) | lx
    P = M * C["cfx"]
    hi64, lo64 = P >> 64, P & M64
    sh = 1061 - ex
    if sh < 64:
        ka, fr = hi64 >> sh, ((hi64 << (64 - sh)) | (lo64 >> sh)) & M64
    else:
        ka, fr = 0, (hi64 >> (sh - 64) if sh < 128 else 0)
    neg = hx >> 31
    k = -ka - (fr != 0) if neg else ka
    f = (-fr) & M64 if neg else fr
    R = (f * C["lfx"]) >> 64
    R2 = (R * R) >> 64
    Rh, R2h = R >> 32, R2 >> 32
    Q = R + (R2 >> 13) + ((R2h * (Rh // 6)) >> 24) + ((R2h * (R2h // 24)) >> 36)
    E1 = 2 ** 63 + (Q >> 13)
    V = (E1 * C["tab"][k & (C["n"] - 1)]) >> 64
    c = V >> 63
    W = (V >> c) | (V & c)
    Mr = (W + 0x1FF + ((W >> 10) & 1)) >> 10
    m = (k >> C["shift"]) + c
    return float(Mr) * 2.0 ** (m - 52)


def fx_to_double(v, f):
    """v 2^-f (0 < v < 2^63) rounded to nearest even, as the kernels do it."""
    assert 0 < v < 2 ** 63
    lz = 64 - v.bit_length()
    w = v << (lz - 1)
    M = (w + 0x1FF + ((w >> 10) & 1)) >> 10
    return float(M) * 2.0 ** (10 - (lz - 1) - f)


def erfcx_half_fx(a):
    """erfcx(a)/2 by the kernels' integer steps (a >= 0 after the clamp)."""
    bits = struct.unpack(">Q", struct.pack(">d", a))[0]
    ha, la = bits >> 32, bits & 0xFFFFFFFF
    iv = max(0, (ha >> C["eshift"]) - C["key0"] + 1)
    assert 0 <= iv < len(C["ecx"])
    ex = ha >> 20
    M = (((ha & 0xFFFFF) | (0x100000 if ex else 0)) << 32) | la
    sh = 16 if iv > 0 else ex - 1006
    v = (M << sh) % 2 ** 64 if sh >= 0 else (M >> -sh if sh > -64 else 0)
    t = v ^ (1 << 63)
    t = t - 2 ** 64 if t >= 2 ** 63 else t  # t 2^63, signed
    c = C["ecx"][iv]
    p = c[C["deg"]]
    for j in range(C["deg"] - 1, -1, -1):
        p = ((p * t) >> 64) * 2 + c[j]  # floor of the high word, as the signed 128-bit product gives it
        assert -(2 ** 63) <= p < 2 ** 63
    return fx_to_double(p, 62 + C["esh"][iv])


def split_E(S):
    a = min(abs(S), 9.0)
    p = erfcx_half_fx(a)
    eS = exp_t(-mul(a, a))
    return mul(eS, p), eS


def ulp(x):
    return np.spacing(abs(x))


def _at_prec(test):
    """Run a test's mpmath references at PREC bits."""
    @functools.wraps(test)
    def run(*a, **k):
        with mp.workprec(PREC):
            return test(*a, **k)
    return run


@_at_prec
def test_exp_within_one_ulp():
    rng = np.random.default_rng(3)
    xs = np.concatenate([np.linspace(-700, 700, 401), rng.uniform(-5, 5, 600), rng.uniform(-1e-3, 1e-3, 50),
                         -rng.uniform(0, 81, 600), [0.0, -0.0, 5e-324, -1e-300, 1e-17, -1e-17]])
    worst, worst_small = 0.0, 0.0
    for x in xs:
        ref = mp.exp(mp.mpf(float(x)))
        got = exp_t(float(x))
        e = float(abs(mp.mpf(got) - ref)) / ulp(float(ref))
        worst = max(worst, e)
        if abs(x) <= 100:
            worst_small = max(worst_small, e)
    # one rounding plus the fixed-point steps (the constant N/ln2 adds |x| 2^-63)
    assert worst_small <= 0.52 and worst <= 1.0, (worst_small, worst)


@_at_prec
def test_split_A_absolute_and_tail_accuracy():
    rng = np.random.default_rng(4)
    Ss = np.concatenate([np.linspace(-9.5, 9.5, 381), rng.normal(0, 1.0, 400), [0.0, -0.0, 0.75, 1.75, 3.25, 5.5]])
    worst_abs = 0.0
    worst = {3.0: [0.0, 0.0], 9.0: [0.0, 0.0]}  # |S| bound -> [tail rel, exp(-S^2) rel]
    for S in Ss:
        S = float(S)
        E, eS = split_E(S)
        Ap = 1.0 - E if S >= 0 else E
        ref_p = (1 + mp.erf(mp.mpf(S))) / 2
        worst_abs = max(worst_abs, float(abs(mp.mpf(Ap) - ref_p)))
        tail = min(ref_p, 1 - ref_p)  # the side that equals E
        ref_e = mp.exp(-mp.mpf(S) ** 2)
        for bound, w in worst.items():
            if abs(S) <= bound:
                w[0] = max(w[0], float(abs(mp.mpf(E) - tail) / tail))
                w[1] = max(w[1], float(abs(mp.mpf(eS) - ref_e) / ref_e))
    assert worst_abs <= 2.5e-16, worst_abs
    # exp(-S^2) inherits the rounding of S^2: |S|^2 * 2^-53 relative
    assert worst[3.0][0] <= 1.5e-15 and worst[3.0][1] <= 1.5e-15, worst
    assert worst[9.0][0] <= 1.2e-14 and worst[9.0][1] <= 1.2e-14, worst
