// erfcx on the integer pipes: Horner's rule in 64-bit fixed point.
//
// The split fluxes need erfcx(|S|)/2 four times per residual slot, a degree-8
// polynomial per interval (lskum_mathconst.h).  In FP64 that is nine FP64
// instructions (the argument map and eight fused multiply-adds), and each
// holds GB300's FP64 unit for 64 cycles per warp.  Here the argument map is
// read off the bits of |S| and the polynomial is evaluated with 64x64-bit
// integer products, so the FP64 unit is not used at all:
//
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
// Host and device compile the same code; the CPU tests check it against
// mpmath and against an exact emulation of the same integer steps.
#pragma once
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
