// e^x in FP64 by Tang's table-driven method (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989), with 32 table entries:
//   x = N ln2/32 + r,  N = round(32 x / ln2),  |r| <= ln2/64,
//   e^x = 2^m 2^(j/32) e^r  with N = 32 m + j, 0 <= j < 32,
// the reduction by ln2/32 = L1 + L2 (L1 of 36 bits, so that N L1 is exact),
// e^r by its Taylor polynomial of degree 6 (the first omitted term, r^7/7!, is
// below 2^-58 for |r| <= ln2/64) and 2^m placed in the exponent field of the
// table entry.  Eleven FP64 operations; within 2 ulp of e^x for x in
// [-700, 700] (tests/test_gpu_math.py checks it against the library's exp).
// The constants come from csrc/gen_exp_tab.py.
#pragma once

#include <cuda_runtime.h>

#include "pab_bits.cuh"

namespace pab {
namespace {

__constant__ double kExp2Tab[32] = {
    0x1.0000000000000p+0, 0x1.059b0d3158574p+0, 0x1.0b5586cf9890fp+0, 0x1.11301d0125b51p+0,
    0x1.172b83c7d517bp+0, 0x1.1d4873168b9aap+0, 0x1.2387a6e756238p+0, 0x1.29e9df51fdee1p+0,
    0x1.306fe0a31b715p+0, 0x1.371a7373aa9cbp+0, 0x1.3dea64c123422p+0, 0x1.44e086061892dp+0,
    0x1.4bfdad5362a27p+0, 0x1.5342b569d4f82p+0, 0x1.5ab07dd485429p+0, 0x1.6247eb03a5585p+0,
    0x1.6a09e667f3bcdp+0, 0x1.71f75e8ec5f74p+0, 0x1.7a11473eb0187p+0, 0x1.82589994cce13p+0,
    0x1.8ace5422aa0dbp+0, 0x1.93737b0cdc5e5p+0, 0x1.9c49182a3f090p+0, 0x1.a5503b23e255dp+0,
    0x1.ae89f995ad3adp+0, 0x1.b7f76f2fb5e47p+0, 0x1.c199bdd85529cp+0, 0x1.cb720dcef9069p+0,
    0x1.d5818dcfba487p+0, 0x1.dfc97337b9b5fp+0, 0x1.ea4afa2a490dap+0, 0x1.f50765b6e4540p+0,
};

__device__ __forceinline__ double exp_tab(double x)
{
    constexpr double kInvL = 0x1.71547652b82fep+5;  // 32/ln2
    constexpr double kL1 = 0x1.62e42fefa0000p-6;    // ln2/32, the leading 36 bits
    constexpr double kL2 = 0x1.cf79abc9e3b3ap-45;   // ln2/32 - L1
    constexpr double kShift = 0x1.8p52;             // adding it rounds to an integer
    const double t = fma(x, kInvL, kShift);
    const int N = (int)(uint32_t)ubits(t);           // the integer in the low bits
    const double n = t - kShift;
    double r = fma(-n, kL1, x);
    r = fma(-n, kL2, r);
    double p = 1.0 / 720.0;
    p = fma(p, r, 1.0 / 120.0);
    p = fma(p, r, 1.0 / 24.0);
    p = fma(p, r, 1.0 / 6.0);
    p = fma(p, r, 0.5);
    p = fma(p, r, 1.0);
    p = fma(p, r, 1.0);
    const double T = from_bits(ubits(kExp2Tab[N & 31]) + ((uint64_t)(int64_t)(N >> 5) << 52));
    return T * p;
}

}  // namespace
}  // namespace pab
