// FP64 elementary functions of the split fluxes, shaped for GB300's scarce
// FP64 issue rate (1/64 of FP32): everything that can run on the integer
// pipes (range-reduction index, exponent scaling, interval selection, sign
// tests, the multiplications: mul_i, the erfcx polynomial in fixed point:
// lskum_fixmath.cuh) does, and exp(-S^2) is shared between the two places a
// split flux needs it.  Constants: lskum_mathconst.h (gen_mathconst.py
// documents the methods and their accuracy).  The tables are read per thread at diverging
// indices, which would serialise constant-cache reads, so they live in
// memory: the kernels that evaluate them at every point (the residual and
// the update) stage a copy in shared memory; the sweeps, which
// need them only at wall and outer points, read one global copy (g_math).
#pragma once
#include "lskum_fixmath.cuh"
#include "lskum_intmul.cuh"
#include "lskum_mathconst.h"

namespace lskum {

struct MathTables {
    double exp2j[kExpN];                           // 2^(j/N)
    long long ecx[kErfcxIntervals][kErfcxDeg + 1]; // erfcx/2 per interval, fixed-point Horner coefficients
    int esh[kErfcxIntervals];                      // their scales: units of 2^-(62 + esh)
};

// Copy the tables into shared memory (all threads of the block; then sync).
__device__ __forceinline__ void load_math_tables(MathTables &T)
{
    for (int i = threadIdx.x; i < kExpN; i += blockDim.x) T.exp2j[i] = kExpTable[i];
    for (int i = threadIdx.x; i < kErfcxIntervals * (kErfcxDeg + 1); i += blockDim.x)
        T.ecx[i / (kErfcxDeg + 1)][i % (kErfcxDeg + 1)] = kErfcxFx[i / (kErfcxDeg + 1)][i % (kErfcxDeg + 1)];
    for (int i = threadIdx.x; i < kErfcxIntervals; i += blockDim.x) T.esh[i] = kErfcxFxShift[i];
}

// exp(x) for |x| <= 700 (Tang's table-driven method, N = 4096 table entries,
// e^r - 1 of degree 3): 8 FP64 instructions.
__device__ __forceinline__ double exp_t(const MathTables &T, double x)
{
    const double big = 0x1.8p52;                            // rounds x*N/ln2 into the low word
    const double t = fma(x, kExpInvLn2N, big);
    const int k = __double2loint(t);                        // round(x * N / ln2)
    const double kd = t - big;
    double r = fma(kd, -kExpLn2NHi, x);
    r = fma(kd, -kExpLn2NLo, r);                            // |r| <= ln2/(2N)
    static_assert(kExpDeg == 3, "exp_t evaluates a cubic");
    const double h = fma(r, 1.0 / 6.0, 0.5);
    const double p = fma(mul_i(r, r), h, r);                // e^r - 1
    const double e = T.exp2j[k & (kExpN - 1)];
    const double res = fma(e, p, e);                        // 2^(j/N) e^r
    return __hiloint2double(__double2hiint(res) + ((k >> kExpShift) << 20), __double2loint(res));
}

// E = exp(-S^2) erfcx(|S|)/2 and eS = exp(-S^2); then (1 + erf S)/2 is 1 - E
// for S >= 0 and E for S < 0, and (1 - erf S)/2 the other one.  |S| is
// clamped to 9 (E < 1e-36 there), which also keeps exp's argument in range;
// the absolute value, the clamp and the interval come from the high word on
// the integer pipe (positive doubles order like their high words).  A NaN S
// is clamped too and gives finite E and eS, but S is NaN only when u_d or
// beta is, and both enter every split flux directly, so a NaN state still
// yields NaN fluxes; the update's positivity and finiteness check reports it.
__device__ __forceinline__ void split_E(const MathTables &T, double S, double &E, double &eS)
{
    constexpr int kNineHi = 0x40220000;  // high word of 9.0 (low word 0)
    const int hs = __double2hiint(S) & 0x7fffffff;
    const bool clamp = hs >= kNineHi;
    const int ha = clamp ? kNineHi : hs, la = clamp ? 0 : __double2loint(S);
    const double a = __hiloint2double(ha, la);
    const int iv = erfcx_interval(ha);
    const double p = erfcx_half_fx<kErfcxDeg>((uint32_t)ha, (uint32_t)la, iv, (const int64_t *)T.ecx[iv], T.esh[iv]);
    eS = exp_t(T, -mul_i(a, a));
    E = mul_i(eS, p);
}

// A = (1 + sg erf S)/2 (sg = +1 if pos, else -1) and eS = exp(-S^2).
__device__ __forceinline__ void split_A(const MathTables &T, double S, bool pos, double &A, double &eS)
{
    double E;
    split_E(T, S, E, eS);
    A = ((__double2hiint(S) >= 0) == pos) ? 1.0 - E : E;
}

}  // namespace lskum
