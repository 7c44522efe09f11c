// exp and erfcx on the integer pipes, in 64-bit fixed point.
//
// The split fluxes need, per residual slot, six exponentials (one per
// inverse of Eq. 14, one per split flux) and four erfcx evaluations.  In
// FP64 that is 7 and 9 FP64 instructions each, and every one holds GB300's
// FP64 unit for 64 cycles per warp.  Here both run on the integer pipes,
// with 32x32->64-bit multiply-adds, funnel shifts and adds; the only FP64
// values are the argument and the result:
//
// exp (Tang's table-driven method in fixed point): the 53-bit significand of
// x times N/ln2 (63 bits) is an exact 116-bit integer, which one variable
// shift splits into k and the fraction f (64 bits) of x N/ln2; with
// k = N m + j, exp(x) = 2^m 2^(j/N) e^r, r = f ln2/N < ln2/N, the table
// entry in units of 2^-63 and e^r by its quartic in units of 2^-76.  The
// steps truncate by a few units of 2^-62 relative; the constant's rounding
// adds |x| 2^-63 relative.  One rounding to the nearest double at the end.
//
// erfcx (Horner's rule in fixed point):
// - the interval of x = |S| is [2^e (1 + m/16), 2^e (1 + (m+1)/16)) (or
//   [0, 2^-5)); there t = (x - c)/h = 2u - 1 with u the significand bits
//   below the top four, so t * 2^63 is those 48 bits shifted left by 16 with
//   the top bit flipped: exact, two or three integer instructions (on
//   [0, 2^-5): t = 64 x - 1, the significand shifted by the exponent);
// - Horner's rule p <- p t + c_j with p and c_j in fixed point (2^(62+s)
//   units, s per interval so that every partial sum stays below 2 in
//   magnitude) and t in 2^63 units: each step is the high word of a signed
//   64x64-bit product, one shift and one add.  Each step truncates by at
//   most 2 units of 2^-(62+s), so the value is within ~2^-57 relative of the
//   polynomial in exact arithmetic, far below FP64's own Horner rounding;
// - the positive result is rounded once to the nearest double.
//
// Host and device compile the same code; the CPU tests check both against
// mpmath and against exact emulations of the same integer steps.
#pragma once
#include <cmath>
#include <cstdint>

#include "lskum_intmul.cuh"

namespace lskum {

// High 64 bits of the signed 128-bit product a b.
LSKUM_HD int64_t mulhi_s64(int64_t a, int64_t b)
{
#ifdef __CUDA_ARCH__
    return __mul64hi((long long)a, (long long)b);
#else
    return (int64_t)(((__int128)a * b) >> 64);
#endif
}

LSKUM_HD int clz64(uint64_t v)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

// v 2^-f for 0 < v < 2^63, rounded to the nearest double (ties to even);
// the result must be a normal number (the callers' values are within a few
// binades of 1).
LSKUM_HD double fx_to_double(uint64_t v, int f)
{
    const int lz = clz64(v);                  // >= 1
    const uint64_t w = v << (lz - 1);         // in [2^62, 2^63)
    // 53-bit significand: bits 62..10; bit 9 rounds, bits 8..0 are sticky
    const uint64_t M = (w + 0x1ffu + ((w >> 10) & 1u)) >> 10;  // in [2^52, 2^53]
    // v 2^-f = M 2^(10 - (lz - 1) - f), i.e. the binade 2^(63 - lz - f);
    // the exponent field is written one less, and the hidden bit of M adds
    // the one back (a rounding carry into 2^53 moves to the next binade)
    const uint32_t E = (uint32_t)(1023 + 63 - lz - f - 1) << 20;
    return f64_from_bits(((uint64_t)E << 32) + M);
}

LSKUM_HD uint64_t umulhi64(uint64_t a, uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// The library's own exp, for arguments outside exp_fx's range.
#ifdef __CUDA_ARCH__
__device__ __noinline__ double exp_outside(double x) { return exp(x); }
#else
inline double exp_outside(double x) { return std::exp(x); }
#endif

// exp(x) to the nearest double within 0.51 ulp for |x| <= 100 (the split
// fluxes' range), within 1 ulp up to |x| = 708; larger |x|, infinities and
// NaN go to the library's exp.  tab: 2^(j/N) in units of 2^-63; C: N/ln2
// in units of 2^-50; L: ln2/N in units of 2^-76 (N = 2^NB).
template <int NB>
LSKUM_HD double exp_fx(const uint64_t *tab, uint64_t C, uint64_t L, double x)
{
    const uint64_t X = f64_bits(x);
    const uint32_t hx = (uint32_t)(X >> 32), lx = (uint32_t)X;
    const uint32_t ex = (hx >> 20) & 0x7ffu;
    if ((hx & 0x7fffffffu) >= 0x40862000u) return exp_outside(x);  // |x| >= 708
    // P = M C (M the significand, 53 bits; C 63 bits) as hi64 2^64 + lo64
    const uint32_t m1 = (hx & 0x000fffffu) | (ex ? 0x00100000u : 0u), m0 = lx;
    const uint32_t c1 = (uint32_t)(C >> 32), c0 = (uint32_t)C;
    const uint64_t p00 = (uint64_t)m0 * c0, p01 = (uint64_t)m0 * c1, p10 = (uint64_t)m1 * c0;
    const uint64_t mid = (p00 >> 32) + (uint32_t)p01 + (uint32_t)p10;  // < 3 2^32
    const uint64_t hi64 = (uint64_t)m1 * c1 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
    const uint64_t lo64 = (mid << 32) | (uint32_t)p00;
    // |x| N/ln2 = P 2^(ex - 1125): integer part ka, fraction fr (2^-64 units)
    const int sh = 1061 - (int)ex;  // >= 29 below 708
    uint64_t ka, fr;
    if (sh < 64) {
        ka = hi64 >> sh;
        fr = (hi64 << (64 - sh)) | (lo64 >> sh);
    } else {
        ka = 0;
        fr = sh < 128 ? hi64 >> (sh - 64) : 0;
    }
    // x < 0: x N/ln2 = -(ka + fr) = k + f with k = -ka - (fr != 0), f = -fr mod 2^64
    const bool neg = hx >> 31;
    const int32_t k = neg ? -(int32_t)ka - (fr != 0) : (int32_t)ka;
    const uint64_t f = neg ? (uint64_t)0 - fr : fr;
    // r 2^76 = f L 2^-64; e^r - 1 = r + r^2/2 + r^3/6 + r^4/24 in 2^-76 units
    const uint64_t R = umulhi64(f, L);             // < 2^63.5
    const uint64_t R2 = umulhi64(R, R);            // r^2 2^88
    const uint32_t Rh = (uint32_t)(R >> 32);       // r 2^44
    const uint32_t R2h = (uint32_t)(R2 >> 32);     // r^2 2^56
    const uint64_t T3 = ((uint64_t)R2h * (Rh / 6u)) >> 24;   // r^3/6 2^76
    const uint64_t T4 = ((uint64_t)R2h * (R2h / 24u)) >> 36; // r^4/24 2^76
    const uint64_t Q = R + (R2 >> 13) + T3 + T4;
    const uint64_t E1 = 0x8000000000000000ull + (Q >> 13);  // e^r 2^63
    const uint64_t V = umulhi64(E1, tab[k & ((1 << NB) - 1)]);  // 2^(j/N) e^r 2^62
    // 2^(j/N) e^r < 2, but the table's rounding can carry V to 2^63 when r
    // is within 1e-19 of ln2/N and j = N - 1: normalise into [2^62, 2^63),
    // the shifted-out bit kept sticky
    const uint32_t c = (uint32_t)(V >> 63);
    const uint64_t W = (V >> c) | (V & c);
    // W 2^(m + c - 62) to the nearest double: bits 62..10 kept
    const uint64_t M = (W + 0x1ffu + ((W >> 10) & 1u)) >> 10;
    const int m = (k >> NB) + (int)c;  // floor(k / N), plus the carry
    const uint32_t E = (uint32_t)(1023 + m - 1) << 20;  // the hidden bit adds the last one
    return f64_from_bits(((uint64_t)E << 32) + M);
}

// erfcx(x)/2 for 0 <= x <= 9 (x = |S| after the clamp), given the high and
// low words of x, its interval iv, that interval's fixed-point coefficients
// c[0..deg] and its scale s (coefficients in units of 2^-(62+s)).
template <int DEG>
LSKUM_HD double erfcx_half_fx(uint32_t ha, uint32_t la, int iv, const int64_t *c, int s)
{
    // u 2^64 (t = 2u - 1): the significand shifted left by 16, modulo 2^64,
    // on the binade intervals; x 2^69 on [0, 2^-5), the significand shifted
    // by the exponent (x < 2^-5: at most 11 places left)
    const uint32_t ex = ha >> 20;                                   // x >= 0
    const uint64_t M = ((uint64_t)((ha & 0x000fffffu) | (ex ? 0x00100000u : 0u)) << 32) | la;
    const int sh = iv > 0 ? 16 : (int)ex - 1006;
    const uint64_t v = sh >= 0 ? M << sh : (sh > -64 ? M >> -sh : 0);
    const int64_t t = (int64_t)(v ^ 0x8000000000000000ull);       // t 2^63
    int64_t p = c[DEG];
#pragma unroll
    for (int j = DEG - 1; j >= 0; j--) p = (int64_t)((uint64_t)mulhi_s64(p, t) << 1) + c[j];
    return fx_to_double((uint64_t)p, 62 + s);
}

}  // namespace lskum
