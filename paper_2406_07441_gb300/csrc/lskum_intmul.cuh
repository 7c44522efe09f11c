// IEEE 754 binary64 multiplication on the integer pipes, correctly rounded
// (round to nearest, ties to even): the same bits as the FP64 multiply.
//
// GB300 issues FP64 at 1/64 of the FP32 rate (two DFMA per SM and clock), so
// a warp's FP64 instruction holds its sub-partition's FP64 unit for 64
// cycles while the integer pipes, which issue a warp instruction every one
// or two cycles, stand idle in an FP64-bound kernel.  mul_i moves a
// multiplication onto those pipes: the 106-bit product of the two 53-bit
// significands from four 32x32->64-bit integer multiply-adds, then
// normalisation, rounding and packing: about fifty integer instructions in
// all (ncu), some thirty of them on the ALU pipe, which issues one every two
// cycles per sub-partition -- as fast as the FP64 unit's 64 cycles, and it
// runs beside it.
//
// Method: the textbook binary multiplication of IEEE 754-2008 sec. 4.3 and
// 5.4.1 (exact significand product, one normalising shift, round to nearest
// even with a guard bit and a sticky bit).  Operands or results outside the
// normal range -- zeros, subnormals, infinities, NaNs, overflow, underflow --
// take the FP64 multiply itself, so every input gives the FP64 multiply's
// result.  Host and device compile the same code (the CPU tests check it
// against the host's own IEEE multiply).
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define LSKUM_HD __host__ __device__ __forceinline__
#else
#define LSKUM_HD inline
#endif

namespace lskum {

LSKUM_HD uint64_t f64_bits(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    std::memcpy(&u, &x, sizeof u);
    return u;
#endif
}

LSKUM_HD double f64_from_bits(uint64_t u)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    std::memcpy(&x, &u, sizeof x);
    return x;
#endif
}

// The FP64 unit's product, for the operands the integer path leaves to it.
#ifdef __CUDA_ARCH__
__device__ __noinline__ double mul_fp64_unit(double a, double b) { return a * b; }
#else
inline double mul_fp64_unit(double a, double b) { return a * b; }
#endif

// High word of (hi:lo) << n and low word of (hi:lo) >> n, 0 <= n < 32 (one
// funnel shift each on the device).
LSKUM_HD uint32_t funnel_l(uint32_t lo, uint32_t hi, uint32_t n)
{
#ifdef __CUDA_ARCH__
    return __funnelshift_l(lo, hi, n);
#else
    return (uint32_t)((((uint64_t)hi << 32) | lo) << n >> 32);
#endif
}
LSKUM_HD uint32_t funnel_r(uint32_t lo, uint32_t hi, uint32_t n)
{
#ifdef __CUDA_ARCH__
    return __funnelshift_r(lo, hi, n);
#else
    return (uint32_t)((((uint64_t)hi << 32) | lo) >> n);
#endif
}

// a * b, rounded to nearest even, on the integer pipes.  Everything is kept
// in 32-bit words: the exponent fields stay in place in the high word (bits
// 20..30), so the result's high word is one three-input add.
LSKUM_HD double mul_i(double a, double b)
{
    const uint64_t A = f64_bits(a), B = f64_bits(b);
    const uint32_t ah = (uint32_t)(A >> 32), al = (uint32_t)A;
    const uint32_t bh = (uint32_t)(B >> 32), bl = (uint32_t)B;
    // significands with the hidden bit, as (21-bit high, 32-bit low) halves
    const uint32_t ma = (ah & 0x000fffffu) | 0x00100000u, mb = (bh & 0x000fffffu) | 0x00100000u;
    // P = (ma 2^32 + al)(mb 2^32 + bl), 2^104 <= P < 2^106, as H 2^64 + mid 2^32 + lo
    const uint64_t p00 = (uint64_t)al * bl;
    const uint64_t p01 = (uint64_t)al * mb + (uint32_t)(p00 >> 32);  // < 2^53 + 2^32
    const uint64_t p10 = (uint64_t)ma * bl + (uint32_t)p01;          // < 2^53 + 2^32
    const uint32_t c = (uint32_t)(p01 >> 32) + (uint32_t)(p10 >> 32);  // < 2^22
    const uint64_t H = (uint64_t)ma * mb + c;                          // < 2^42
    const uint32_t hh = (uint32_t)(H >> 32), hl = (uint32_t)H, mid = (uint32_t)p10, lo = (uint32_t)p00;
    // X = floor(P / 2^42) = (xh, xl) in [2^62, 2^64)
    const uint32_t xh = funnel_l(hl, hh, 22), xl = funnel_l(mid, hl, 22);
    const uint32_t st = ((mid & 0x3ffu) | lo) != 0u;  // the 42 bits below X
    const uint32_t s = xh >> 31;  // 1 when the significand product is >= 2
    // normalise to [2^62, 2^63): shift right by s, the shifted-out bit and
    // the sticky bit into bit 0
    const uint32_t nh = xh >> s;
    const uint32_t nl = funnel_r(xl, xh, s) | (xl & s) | st;
    // 53-bit significand: bits 62..10; bit 9 rounds, bits 8..0 are sticky.
    // Adding 0x1ff plus the kept lsb carries into bit 10 exactly when the
    // discarded part is above half, or half with an odd lsb (ties to even).
    const uint64_t N = (((uint64_t)nh << 32) | nl) + (0x1ffu + ((nl >> 10) & 1u));
    const uint32_t Mh = (uint32_t)(N >> 42), Ml = funnel_r((uint32_t)N, (uint32_t)(N >> 32), 10);
    // biased exponent e = ea + eb - 1023 + s, kept as (e - 1) << 20 (mod 2^32):
    // the hidden bit of M (Mh >= 2^20) adds the last 1, and a rounding carry
    // into 2^53 moves to the next binade by itself
    const uint32_t xa = ah & 0x7ff00000u, xb = bh & 0x7ff00000u;
    const uint32_t E = xa + xb + (s << 20) - (1024u << 20);
    const bool normal_in = (xa - 0x00100000u < 0x7fe00000u) && (xb - 0x00100000u < 0x7fe00000u);
    const bool normal_out = E < (2045u << 20);  // 1 <= e <= 2045: finite after the carry
    if (!(normal_in && normal_out)) return mul_fp64_unit(a, b);
    const uint32_t rh = ((ah ^ bh) & 0x80000000u) + E + Mh;
    return f64_from_bits(((uint64_t)rh << 32) | Ml);
}

// FP32 keeps its own multiply (its pipe is not the scarce one); the overload
// lets code templated on the precision call mul_i for both.
LSKUM_HD float mul_i(float a, float b) { return a * b; }

}  // namespace lskum
