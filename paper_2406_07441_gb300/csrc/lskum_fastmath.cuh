// FP64 elementary functions of the split fluxes, shaped for GB300's scarce
// FP64 issue rate (1/64 of FP32): everything that can run on the integer
// pipes (range-reduction index, exponent scaling, interval selection, sign
// tests, exp and the erfcx polynomial in fixed point: lskum_fixmath.cuh)
// does, and exp(-S^2) is shared between the two places a split flux needs
// it.  Constants: lskum_mathconst.h (gen_mathconst.py documents the methods
// and their accuracy).  The tables are read per thread at diverging
// indices, which would serialise constant-cache reads, so they live in
// memory: the kernels that evaluate them at every point (the residual and
// the update) stage a copy in shared memory; the sweeps, which need them
// only at wall and outer points, read one global copy (g_math).
#pragma once
#include "lskum_fixmath.cuh"
#include "lskum_intmul.cuh"
#include "lskum_mathconst.h"

namespace lskum {

struct MathTables {
    unsigned long long exp2j[kExpN];               // 2^(j/N) in units of 2^-63
    long long ecx[kErfcxIntervals][kErfcxDeg + 1]; // erfcx/2 per interval, fixed-point Horner coefficients
    int esh[kErfcxIntervals];                      // their scales: units of 2^-(62 + esh)
};

// Copy the tables into shared memory (all threads of the block; then sync).
__device__ __forceinline__ void load_math_tables(MathTables &T)
{
    for (int i = threadIdx.x; i < kExpN; i += blockDim.x) T.exp2j[i] = kExpTableFx[i];
    for (int i = threadIdx.x; i < kErfcxIntervals * (kErfcxDeg + 1); i += blockDim.x)
        T.ecx[i / (kErfcxDeg + 1)][i % (kErfcxDeg + 1)] = kErfcxFx[i / (kErfcxDeg + 1)][i % (kErfcxDeg + 1)];
    for (int i = threadIdx.x; i < kErfcxIntervals; i += blockDim.x) T.esh[i] = kErfcxFxShift[i];
}

// exp(x) in fixed point on the integer pipes (lskum_fixmath.cuh): within
// 0.51 ulp for |x| <= 100, 1 ulp up to 708, the library's exp beyond.  A
// real call, not inlined: each of its call sites in the residual's slot
// loop would otherwise carry ~80 instructions into a loop that already
// strains the instruction cache (measured 2% faster out of line; erfcx and
// split_E out of line measured slower).
__device__ __noinline__ double exp_t(const MathTables &T, double x)
{
    return exp_fx<kExpShift>((const uint64_t *)T.exp2j, kExpFxC, kExpFxL, x);
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
    // the two multiplications stay on the FP64 unit (short latency on the
    // path to A; measured faster than the integer multiply here)
    eS = exp_t(T, -(a * a));
    E = eS * p;
}

// A = (1 + sg erf S)/2 (sg = +1 if pos, else -1) and eS = exp(-S^2).
__device__ __forceinline__ void split_A(const MathTables &T, double S, bool pos, double &A, double &eS)
{
    double E;
    split_E(T, S, E, eS);
    A = ((__double2hiint(S) >= 0) == pos) ? 1.0 - E : E;
}

}  // namespace lskum
