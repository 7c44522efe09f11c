"""Generate lskum_mathconst.h: constants of the kernels' own FP64 exp and erfcx.

Run from the repository root:  python paper_2406_07441_gb300/csrc/gen_mathconst.py
(needs mpmath; the generated header is committed, so building does not).

exp (table-driven, after P. T. P. Tang, "Table-driven implementation of the
exponential function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989),
evaluated in 64-bit fixed point on the integer pipes (lskum_fixmath.cuh):
  x N/ln2 = k + f exactly to 2^-64 (the 53-bit significand times N/ln2 in
  units of 2^-50, a 116-bit integer product), k = N m + j, 0 <= f < 1,
  exp(x) = 2^m * 2^(j/N) * e^r with r = f ln2/N in [0, ln2/N), N = 4096,
  2^(j/N) tabulated in units of 2^-63 (rounded to nearest), e^r - 1 by its
  Taylor polynomial of degree 4 (truncation < 1.3e-21 on [0, ln2/N)).  The
  constant N/ln2 carries 63 bits, so the reduction is within |x| 2^-63 of
  exact: below 1e-17 relative for the |x| <= 81 the split fluxes need.

erfcx(x) = exp(x^2) erfc(x) for 0 <= x <= 9: the intervals are [0, 2^-5)
and, above it, sixteen per binade, [2^e (1 + m/16), 2^e (1 + (m+1)/16)) for
e = -5 .. 3 (132 in all, the last one [9, 9.5) holding only the clamp value
9): the interval of x is the high word of x shifted right by 16 (its
exponent and top four significand bits) minus that of 2^-5, plus one,
floored at 0 -- two integer instructions.  On each interval the Chebyshev
interpolant of degree 8 at Chebyshev points of the first kind, rewritten as
a polynomial in t = (x - c)/h (c, h the interval's centre and half width;
on the binade intervals t is 2u - 1 with u the significand bits below the
top four); the interpolants are within 6e-17 relative of erfcx in exact
arithmetic (checked at 200 points per interval with mpmath; the worst,
5.9e-17, on [8, 8.5], where E < 1e-28).  The kernels evaluate them by
Horner's rule in 64-bit fixed point on the integer pipes
(lskum_fixmath.cuh): coefficients of erfcx/2 in units of 2^-(62+s), the
scale s per interval the largest that keeps every Horner partial sum below
1.5 in magnitude on [-1, 1]; the generator runs those integer steps exactly
at the same 200 points and checks them against the exact-arithmetic
polynomial (within 2e-17 relative before the final rounding).  The kernels
use it as
  A = (1 + s erf S)/2 = 1 - E (s S >= 0)  or  E (s S < 0),
  E = exp(-S^2) erfcx(|S|) / 2,
which shares exp(-S^2) with the B term of the split flux and is accurate in
absolute terms for every S (the kernels clamp |S| to 9, where E < 1e-36).
"""
import os
import struct

import mpmath as mp

mp.mp.dps = 60
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "lskum_mathconst.h")

# Interval bounds: 0, then 2^e (1 + m/16) for e = -5 .. 3, m = 0 .. 15, up to
# the interval that holds 9 (the kernels' clamp of |S|).
LOW_EXP, MBITS = -5, 4


def _intervals():
    out = [(0.0, 2.0 ** LOW_EXP)]
    e = LOW_EXP
    while True:
        for m in range(2 ** MBITS):
            a = 2.0 ** e * (1 + m / 2 ** MBITS)
            b = 2.0 ** e * (1 + (m + 1) / 2 ** MBITS)
            out.append((a, b))
            if b > 9.0:
                return out
        e += 1


INTERVALS = _intervals()
DEGREE = 8
EXP_N = 4096
EXP_DEG = 4


def erfcx(x):
    return mp.exp(x * x) * mp.erfc(x)


def cheb_monomial(f, a, b, n):
    a, b = mp.mpf(a), mp.mpf(b)
    c, h = (a + b) / 2, (b - a) / 2
    N = n + 1
    xs = [mp.cos(mp.pi * (k + mp.mpf(1) / 2) / N) for k in range(N)]
    fs = [f(c + h * t) for t in xs]
    ck = [2 * mp.fsum(fs[k] * mp.cos(mp.pi * j * (k + mp.mpf(1) / 2) / N) for k in range(N)) / N
          for j in range(N)]
    ck[0] /= 2
    T = [[mp.mpf(1)], [mp.mpf(0), mp.mpf(1)]]
    for j in range(2, N):
        new = [mp.mpf(0)] * (j + 1)
        for i, v in enumerate(T[j - 1]):
            new[i + 1] += 2 * v
        for i, v in enumerate(T[j - 2]):
            new[i] -= v
        T.append(new)
    mono = [mp.mpf(0)] * N
    for j in range(N):
        for i, v in enumerate(T[j]):
            mono[i] += ck[j] * v
    return mono, c, h


def hexd(v):
    return float(v).hex()


def main(out=OUT):
    lines = [
        "// Generated by gen_mathconst.py (mpmath, 60 digits); do not edit.",
        "// Constants of the kernels' own FP64 exp and erfcx; see gen_mathconst.py for the methods.",
        "#pragma once",
        "",
        "namespace lskum {",
        "",
        f"constexpr int kExpN = {EXP_N};  // table size N (a power of two)",
        f"constexpr int kExpShift = {EXP_N.bit_length() - 1};  // log2 N",
    ]
    # N/ln2 in units of 2^-50 (63 bits) and ln2/N in units of 2^-76 (64 bits)
    cfx = int(mp.nint(EXP_N / mp.log(2) * mp.mpf(2) ** 50))
    lfx = int(mp.nint(mp.log(2) / EXP_N * mp.mpf(2) ** 76))
    assert 2 ** 62 <= cfx < 2 ** 63 and 2 ** 63 <= lfx < 2 ** 64
    lines += [
        f"constexpr int kExpDeg = {EXP_DEG};  // degree of the polynomial for e^r - 1",
        f"constexpr unsigned long long kExpFxC = {cfx}ull;  // N/ln2 in units of 2^-50",
        f"constexpr unsigned long long kExpFxL = {lfx}ull;  // ln2/N in units of 2^-76",
        f"// 2^(j/N), j = 0..N-1, in units of 2^-63 (rounded to nearest)",
        f"__device__ unsigned long long kExpTableFx[{EXP_N}] = {{",
    ]
    for j in range(0, EXP_N, 4):
        lines.append("    " + ", ".join(str(int(mp.nint(mp.power(2, mp.mpf(k) / EXP_N) * mp.mpf(2) ** 63))) + "ull"
                                        for k in range(j, j + 4)) + ",")
    lines.append("};")
    # the polynomial's truncation on 0 <= r < ln2/N
    rmax = mp.log(2) / EXP_N
    trunc = abs(mp.exp(rmax) - (1 + rmax + rmax ** 2 / 2 + rmax ** 3 / 6 + rmax ** 4 / 24)) / mp.exp(rmax)
    assert EXP_DEG == 4 and trunc < 1.3e-21, trunc
    nI = len(INTERVALS)
    key0 = (int.from_bytes(struct.pack(">d", 2.0 ** LOW_EXP), "big") >> 32) >> (20 - MBITS)
    # the index function reproduces the table's intervals
    for k, (a, b) in enumerate(INTERVALS):
        for x in (a, (a + b) / 2, b * (1 - 2 ** -52)):
            ha = int.from_bytes(struct.pack(">d", x), "big") >> 32
            assert max(0, (ha >> (20 - MBITS)) - key0 + 1) == k or x == 0.0 and k == 0, (k, x)
    lines.append(f"constexpr int kErfcxDeg = {DEGREE};")
    lines.append(f"constexpr int kErfcxIntervals = {nI};")
    lines.append(f"constexpr int kErfcxShift = {20 - MBITS};  // high word >> shift: exponent and top {MBITS} bits")
    lines.append(f"constexpr int kErfcxKey0 = 0x{key0:x};  // that key of 2^{LOW_EXP}")
    lines.append("// interval of x in [0, 9.5): [0, 2^" + str(LOW_EXP) + f") is 0, then {2 ** MBITS} per binade")
    lines.append("__device__ __forceinline__ int erfcx_interval(int ha)  // ha: high word of x >= 0")
    lines.append("{")
    lines.append("    return max(0, (ha >> kErfcxShift) - kErfcxKey0 + 1);")
    lines.append("}")
    coef_rows, shifts = [], []
    for a, b in INTERVALS:
        mono, c, h = cheb_monomial(erfcx, a, b, DEGREE)
        half = [m / 2 for m in mono]  # E = exp(-S^2) * (erfcx/2)
        # the scale: every Horner partial sum below 1.5 x 2^-s on [-1, 1]
        bound = mp.mpf(0)
        for k in range(401):
            t = mp.mpf(-1) + mp.mpf(2) * k / 400
            p = mp.mpf(0)
            for m in reversed(half):
                p = p * t + m
                bound = max(bound, abs(p))
        sft = int(mp.floor(mp.log(mp.mpf(1.5) / bound, 2)))
        assert 0 <= sft <= 8, sft
        fx = [int(mp.nint(m * mp.mpf(2) ** (62 + sft))) for m in half]
        assert all(abs(v) < 2 ** 63 for v in fx)
        for k in range(200):
            x = mp.mpf(a) + (mp.mpf(b) - a) * k / 199
            t = (x - c) / h
            p = mp.mpf(0)
            for m in reversed(mono):
                p = p * t + m
            # the interpolant in exact arithmetic
            assert abs(p / erfcx(x) - 1) < 6e-17, (a, b, x)
            # the kernels' integer steps, exactly (t in 2^-63 units, floor of
            # the high word of each 128-bit product, shifted left by one)
            tq = int(mp.floor(t * 2 ** 63))
            q = fx[DEGREE]
            for j in range(DEGREE - 1, -1, -1):
                q = ((q * tq) >> 64) * 2 + fx[j]
                assert abs(q) < 2 ** 63
            assert abs(mp.mpf(q) / mp.mpf(2) ** (62 + sft) / (p / 2) - 1) < 2e-17, (a, b, x)
        coef_rows.append([str(v) + "ll" if v >= -(2 ** 63) + 1 else None for v in fx])
        shifts.append(str(sft))
    # global (not constant) memory: blocks copy the tables with coalesced loads
    lines.append(f"// erfcx/2 on each interval as a polynomial in t, coefficients of t^0 .. t^{DEGREE}")
    lines.append(f"// in units of 2^-(62 + kErfcxFxShift[interval])")
    lines.append(f"__device__ int kErfcxFxShift[{nI}] = {{" + ", ".join(shifts) + "};")
    lines.append(f"__device__ long long kErfcxFx[{nI}][{DEGREE + 1}] = {{")
    for row in coef_rows:
        lines.append("    {" + ", ".join(row) + "},")
    lines.append("};")
    lines += ["", "}  // namespace lskum", ""]
    with open(out, "w") as f:
        f.write("\n".join(lines))
    print(out)


if __name__ == "__main__":
    main()
