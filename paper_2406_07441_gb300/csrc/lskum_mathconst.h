// Generated by gen_mathconst.py (mpmath, 60 digits); do not edit.
// Constants of the kernels' own FP64 exp and erfcx; see gen_mathconst.py for the methods.
#pragma once

namespace lskum {

constexpr double kExpInvLn2_64 = 0x1.71547652b82fep+6;  // 64 / ln 2
constexpr double kExpLn2_64Hi = 0x1.62e42fe000000p-7;  // ln2/64, 29 significant bits
constexpr double kExpLn2_64Lo = 0x1.f473de6af278fp-36;  // ln2/64 - kExpLn2_64Hi
// 2^(j/64), j = 0..63, correctly rounded
__constant__ double kExpTable[64] = {
    0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0, 0x1.0874518759bc8p+0,
    0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0, 0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0,
    0x1.172b83c7d517bp+0, 0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0,
    0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0, 0x1.2d285a6e4030bp+0,
    0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0, 0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0,
    0x1.3dea64c123422p+0, 0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0,
    0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0, 0x1.56f4736b527dap+0,
    0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0, 0x1.6247eb03a5585p+0, 0x1.6623882552225p+0,
    0x1.6a09e667f3bcdp+0, 0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0,
    0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0, 0x1.868d99b4492edp+0,
    0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0, 0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0,
    0x1.9c49182a3f090p+0, 0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0,
    0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0, 0x1.bcc1e904bc1d2p+0,
    0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0, 0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0,
    0x1.d5818dcfba487p+0, 0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0,
    0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0, 0x1.fa7c1819e90d8p+0,
};
constexpr int kErfcxDeg = 13;
constexpr int kErfcxIntervals = 10;
// high words of the interior interval bounds 0.5, 1.0, 1.5, 2.25, 3.0, 4.0, 5.0, 6.0, 7.5; then scale 1/h and offset -c/h of t = (x - c)/h per interval
__device__ __forceinline__ int erfcx_interval(int ha)  // ha: high word of x >= 0
{
    return (ha >= 0x3fe00000) + (ha >= 0x3ff00000) + (ha >= 0x3ff80000) + (ha >= 0x40020000) + (ha >= 0x40080000) + (ha >= 0x40100000) + (ha >= 0x40140000) + (ha >= 0x40180000) + (ha >= 0x401e0000);
}
__constant__ double kErfcxScale[10] = {0x1.0000000000000p+2, 0x1.0000000000000p+2, 0x1.0000000000000p+2, 0x1.5555555555555p+1, 0x1.5555555555555p+1, 0x1.0000000000000p+1, 0x1.0000000000000p+1, 0x1.0000000000000p+1, 0x1.5555555555555p+0, 0x1.5555555555555p+0};
__constant__ double kErfcxOffset[10] = {-0x1.0000000000000p+0, -0x1.8000000000000p+1, -0x1.4000000000000p+2, -0x1.4000000000000p+2, -0x1.c000000000000p+2, -0x1.c000000000000p+2, -0x1.2000000000000p+3, -0x1.6000000000000p+3, -0x1.2000000000000p+3, -0x1.6000000000000p+3};
// erfcx/2 on each interval as a polynomial in t, coefficients of t^0 .. t^13
__constant__ double kErfcxHalf[10][14] = {
    {0x1.8a6adcda2ea92p-2, -0x1.7c857b9b3c191p-4, 0x1.2b497df35f8cfp-6, -0x1.97997ad330318p-9, 0x1.f0ac9d324abd6p-12, -0x1.146985bdac45dp-14, 0x1.1d0c2795710c2p-17, -0x1.132db78cf552ep-20, 0x1.f54d3f56d40bap-24, -0x1.b181df76bf71cp-27, 0x1.658e4ec31edf1p-30, -0x1.1aab1e21ecc3bp-33, 0x1.ba2e44941ccd1p-37, -0x1.4371ff52e055fp-40},
    {0x1.038d54ea3d834p-2, -0x1.78cdd551ee51ap-5, 0x1.d90093ae108b0p-8, -0x1.09e77d40e0214p-10, 0x1.1192f5bd775ccp-13, -0x1.054d68296477dp-16, 0x1.d43a7c4dbe650p-20, -0x1.8c97dd32ae0e1p-23, 0x1.3f81a9597de0ap-26, -0x1.ec0d1ccb09b6fp-30, 0x1.6b80da7254f0fp-33, -0x1.02a2c5796f3cap-36, 0x1.6be408e744acbp-40, -0x1.e34f70587b39ap-44},
    {0x1.78a692138767ap-3, -0x1.abaacdbfa8b07p-6, 0x1.b56f45eef7e3fp-9, -0x1.9b635ac624ac6p-12, 0x1.68a25a664836fp-15, -0x1.299636d6c9209p-18, 0x1.d1b69597f0c3dp-22, -0x1.5b8bc9419d840p-25, 0x1.f0fe8a88d3cd7p-29, -0x1.55c08c80d2503p-32, 0x1.c55c924775cc5p-36, -0x1.22f10017ec710p-39, 0x1.71368494f04cfp-43, -0x1.bde45264f2361p-47},
    {0x1.13e5743b60481p-3, -0x1.6a8c2095f9678p-6, 0x1.bbbcdecac77dcp-9, -0x1.ff44800b6bb0ep-12, 0x1.1770a1387a55bp-14, -0x1.238aaeeff0ef9p-17, 0x1.23addb3a12f79p-20, -0x1.18e8a07eba6efp-23, 0x1.054059cefc55dp-26, -0x1.d682dcf30e74bp-30, 0x1.9af4a1c5406c6p-33, -0x1.5d3b0fd15c227p-36, 0x1.2b78f446ee404p-39, -0x1.e2dd46e69319ep-43},
    {0x1.9d7738e1f4db7p-4, -0x1.a4ad387d18a36p-7, 0x1.985ce31879abep-10, -0x1.7c27aaae14f17p-13, 0x1.54c5cde0c42dbp-16, -0x1.271fb78890faap-19, 0x1.ef3c4f7e3a39ep-23, -0x1.937ffc5efe7c9p-26, 0x1.3fe3e305e5001p-29, -0x1.ee631de19f54ep-33, 0x1.74d3ca511dc82p-36, -0x1.12edb53981337p-39, 0x1.97bdca17eee26p-43, -0x1.2001ce79d92f7p-46},
    {0x1.3e0a99a0ee914p-4, -0x1.5285d2eb1ef74p-7, 0x1.5d581133377e1p-10, -0x1.5e5d7e98990adp-13, 0x1.5632136dcfdf2p-16, -0x1.460abd6b5aac9p-19, 0x1.2f839defbf63dp-22, -0x1.146bc3b72634ap-25, 0x1.ed2b25c545409p-29, -0x1.af5dd63878f3cp-32, 0x1.721b31a16be1fp-35, -0x1.381bbf4ef7a2ep-38, 0x1.0c53817265dbep-41, -0x1.b52b88aa6a398p-45},
    {0x1.f5b2a049cf4c6p-5, -0x1.aa3eb6a946f7ep-8, 0x1.62c12cb5f7555p-11, -0x1.218ed930b239ap-14, 0x1.d00785f2fe34fp-18, -0x1.6d54b133e1dafp-21, 0x1.1ad6a31498c35p-24, -0x1.aef8ea2825beap-28, 0x1.43551f4037b8bp-31, -0x1.de0985254e968p-35, 0x1.5c4a449ee453dp-38, -0x1.f4c4d68de7790p-42, 0x1.6cee7cc8c027ep-45, -0x1.fee5cbcae7c93p-49},
    {0x1.9d8a8f2284f2cp-5, -0x1.238ca71b93fc3p-8, 0x1.95252b932efdcp-12, -0x1.15976ddda3c9dp-15, 0x1.774f4826df938p-19, -0x1.f4e46d17a1e30p-23, 0x1.4a17e192d447ap-26, -0x1.add7ac91b071bp-30, 0x1.149ce494d441ap-33, -0x1.60002e1ef0109p-37, 0x1.baf6971d5b9c3p-41, -0x1.13ce55f015bd9p-44, 0x1.5ae57d91ad3bfp-48, -0x1.a7111368968b7p-52},
    {0x1.52b80d463c470p-5, -0x1.26cfae569219ep-8, 0x1.fc0d925cb9bd1p-12, -0x1.b1824073cd015p-15, 0x1.6e66b15c39900p-18, -0x1.32d4007c83afcp-21, 0x1.fd44931e8bec1p-25, -0x1.a2efa7e968f20p-28, 0x1.55aef0217abedp-31, -0x1.14598d251aeaep-34, 0x1.bb2aa06cc5859p-38, -0x1.60ad29029c8e7p-41, 0x1.2010958d391b0p-44, -0x1.c33613da16dbep-48},
    {0x1.1618fbc75f8a0p-5, -0x1.8ec506eb645fap-9, 0x1.1bedf98ef6527p-12, -0x1.9196f54750860p-16, 0x1.1a1ee1759f40ep-19, -0x1.89ce516e5c4d4p-23, 0x1.1118e35c230b5p-26, -0x1.78668f170f874p-30, 0x1.01cae5867ee54p-33, -0x1.5efb042e31e5ap-37, 0x1.dae5ddbbbf417p-41, -0x1.3f7b094fefbe1p-44, 0x1.b5e7d16dee5dep-48, -0x1.2329273438940p-51},
};

}  // namespace lskum
