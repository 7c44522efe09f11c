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
constexpr int kErfcxDeg = 17;
// interval bounds (upper limits of intervals 0..3), scale 1/h and offset -c/h of t = (x - c)/h
constexpr double kErfcxBreak[4] = {0.75, 1.75, 3.25, 5.5};
__constant__ double kErfcxScale[5] = {0x1.5555555555555p+1, 0x1.0000000000000p+1, 0x1.5555555555555p+0, 0x1.c71c71c71c71cp-1, 0x1.2492492492492p-1};
__constant__ double kErfcxOffset[5] = {-0x1.0000000000000p+0, -0x1.4000000000000p+1, -0x1.aaaaaaaaaaaabp+1, -0x1.f1c71c71c71c7p+1, -0x1.0924924924925p+2};
// erfcx/2 on each interval as a polynomial in t, coefficients of t^0 .. t^17
__constant__ double kErfcxHalf[5][18] = {
    {0x1.5f28ade3ca4acp-2, -0x1.d78a9b6c39906p-4, 0x1.066ec7e9d3637p-5, -0x1.fe7cd332f7cdep-8, 0x1.bee62667c60e7p-10, -0x1.66e2f5701f58ep-12, 0x1.0be20ec8b9b7cp-14, -0x1.7751fff41c288p-17, 0x1.f12d9161ee160p-20, -0x1.392c4dd75f27cp-22, 0x1.78ff0130aa716p-25, -0x1.b35a1d1954186p-28, 0x1.e3e1bec1de83bp-31, -0x1.03882591f1b41p-33, 0x1.0cd8534ccb692p-36, -0x1.0e93032db208bp-39, 0x1.19dd42653c398p-42, -0x1.0b387d9f2e217p-45},
    {0x1.78a692138767ap-3, -0x1.abaacdbfa8b07p-5, 0x1.b56f45eef7e54p-7, -0x1.9b635ac624ad3p-9, 0x1.68a25a6642604p-11, -0x1.299636d6c5c2cp-13, 0x1.d1b695aa2f084p-16, -0x1.5b8bc94c18337p-18, 0x1.f0fe701071532p-21, -0x1.55c07d51f080fp-23, 0x1.c570150580da3p-26, -0x1.22fc2f897d7a9p-28, 0x1.6a1f9e61f1ef2p-31, -0x1.b5c38e603ea19p-34, 0x1.00a5432e17734p-36, -0x1.265fe133263efp-39, 0x1.66df2b2c822bap-42, -0x1.87225d22d7ebfp-45},
    {0x1.afbb3f3b7343bp-4, -0x1.c8ca43e8282c8p-6, 0x1.cba83bc9e010bp-8, -0x1.ba746c7f90a7cp-10, 0x1.9940762e167d8p-12, -0x1.6d14f0daa3008p-14, 0x1.3b0d0864add93p-16, -0x1.07ac34bfe02d7p-18, 0x1.acf4e1e2d9e4ep-21, -0x1.53c35ef3c9288p-23, 0x1.0679c8912b6e2p-25, -0x1.8c1a9842f362ap-28, 0x1.245f0d1048559p-30, -0x1.a676f1d32e312p-33, 0x1.28d3a71ea5e37p-35, -0x1.9c996d1cc3ca3p-38, 0x1.4118e5a4fd282p-40, -0x1.ac9aeff844472p-43},
    {0x1.01afcc22e71b8p-4, -0x1.f974dd6f23b4ep-7, 0x1.e523040980d6ep-9, -0x1.c83e185fa67b3p-11, 0x1.a4df48f2ba79ep-13, -0x1.7d3233c30b1dfp-15, 0x1.5349b8aba65f0p-17, -0x1.28ff334c60491p-19, 0x1.ffba53c69719cp-22, -0x1.b229c2763c53bp-24, 0x1.6af9bd1d12acbp-26, -0x1.2b33815a69a04p-28, 0x1.e6d82a5ae9965p-31, -0x1.86aca3db6bc32p-33, 0x1.315d1493f99f2p-35, -0x1.de45ba75a199ep-38, 0x1.b949f34ad5869p-40, -0x1.501da4dfdabd1p-42},
    {0x1.3bcc59a28358cp-5, -0x1.2b5da7e32c4a6p-7, 0x1.194c1fd21c328p-9, -0x1.060e8d0d95955p-11, 0x1.e42fa0c62d4d4p-14, -0x1.bba6bffaf74d3p-16, 0x1.9345123121a2ep-18, -0x1.6bb4f625c8088p-20, 0x1.4586359aad2a5p-22, -0x1.212ce5b7061dcp-24, 0x1.fe005be4b3783p-27, -0x1.be85503060b2fp-29, 0x1.8490ae85b5704p-31, -0x1.4f78b8e5e652cp-33, 0x1.19d757a7efc39p-35, -0x1.e070bcc5ebd00p-38, 0x1.fa65a456aa635p-40, -0x1.a8c30a795c542p-42},
};

}  // namespace lskum
