// Products of doubles formed on the integer pipe.
//
// GB300 issues 2 FP64 operations per clock and SM but 64 32-bit integer
// multiplies, so a pass that streams doubles from HBM and multiplies each a few
// times is bound by the FP64 pipe long before the memory.  Here the 53-bit
// significands are multiplied as integers: each significand, shifted to the top
// of 64 bits, splits into 32-bit halves, and the top 64 bits of the 128-bit
// product are the high half-product plus the high words of the two cross
// products (the dropped low words and the low half-product make it at most 2
// units short in its last bit, less than 2^-8 of the result's ulp).  The result
// is then rounded to 53 bits, to nearest, with the exponent added as an integer.
// So it is the correctly rounded product except where the exact one lies within
// 2^-8 ulp of a tie, and then 1 ulp from it at most.  A zero operand gives a
// signed zero.  Subnormal, infinite and NaN operands and results outside the
// normal range clear the caller's flag instead: the caller then forms that
// group of values again with FP64 instructions.  (A select between the two
// forms would not do: the compiler evaluates both sides of a select, and the
// FP64 side would run for every value.)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pab {
namespace {

// The significand of a double as A = A1 2^32 + A0 in [2^63, 2^64), its biased exponent and
// its sign bit (in bit 31).
struct Sig {
    uint32_t a1, a0, sign;
    int e;
};

__device__ __forceinline__ Sig split_sig(double x)
{
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    Sig s;
    s.e = (int)((hi >> 20) & 0x7ffu);
    s.sign = hi & 0x80000000u;
    s.a1 = __funnelshift_l(lo, (hi & 0xfffffu) | 0x100000u, 11);
    s.a0 = lo << 11;
    return s;
}

// floor(A B / 2^64) less 0, 1 or 2, for A, B in [2^63, 2^64): the result lies in [2^62, 2^64)
__device__ __forceinline__ uint64_t mulhi_sig(uint32_t a1, uint32_t a0, uint32_t b1, uint32_t b0)
{
    return (uint64_t)a1 * b1 + __umulhi(a1, b0) + __umulhi(a0, b1);
}

// The double nearest (P / 2^64) 2^k for P in [2^62, 2^64), with the sign bit given in bit 31 of
// sign; false where its biased exponent leaves [1, 2046] (a subnormal, zero or infinite result).
__device__ __forceinline__ bool pack_sig(uint64_t P, int k, uint32_t sign, double &out)
{
    const int top = (int)(P >> 63);
    const int E = k + 1021 + top;
    // 54 bits, then halved with the round bit added: the significand in [2^52, 2^53]
    const uint64_t m = ((P >> (9 + top)) + 1u) >> 1;
    // the hidden bit adds one to the exponent field (and a rounding carry to 2^53 one more)
    const uint64_t bits = ((uint64_t)(uint32_t)(E - 1) << 52) + m + ((uint64_t)sign << 32);
    out = __longlong_as_double((long long)bits);
    return (unsigned)(E - 1) < 2046u;
}

// A factor used for many products: its split, and whether it is a normal number.
struct IntFactor {
    Sig s;
    bool normal;
};

__device__ __forceinline__ IntFactor int_factor(double x)
{
    IntFactor f;
    f.s = split_sig(x);
    f.normal = (unsigned)(f.s.e - 1) < 2046u;
    return f;
}

__device__ __forceinline__ bool is_zero_sig(double x)
{
    return ((__double2hiint(x) & 0x7fffffff) | __double2loint(x)) == 0;
}

// x f, within 1 ulp of the FP64 product (and equal to it but near ties); ok cleared where x is
// subnormal, infinite or NaN, f is not a normal number or the product leaves the normal range.
__device__ __forceinline__ double mul_int(double x, const IntFactor &f, bool &ok)
{
    const Sig a = split_sig(x);
    double r;
    const bool in_range = pack_sig(mulhi_sig(a.a1, a.a0, f.s.a1, f.s.a0), a.e + f.s.e - 2044,
                                   a.sign ^ f.s.sign, r);
    if (is_zero_sig(x)) {
        r = __longlong_as_double((long long)((uint64_t)(a.sign ^ f.s.sign) << 32));
        ok = ok && f.normal;
    } else {
        ok = ok && in_range && f.normal && (unsigned)(a.e - 1) < 2046u;
    }
    return r;
}

// x y with both operands split here; a zero operand (the other a normal number or zero) gives a
// signed zero; ok cleared where an operand is subnormal, infinite or NaN or the product leaves
// the normal range.
__device__ __forceinline__ double mul2_int(double x, double y, bool &ok)
{
    const Sig a = split_sig(x), b = split_sig(y);
    double r;
    const bool in_range = pack_sig(mulhi_sig(a.a1, a.a0, b.a1, b.a0), a.e + b.e - 2044,
                                   a.sign ^ b.sign, r);
    const bool na = (unsigned)(a.e - 1) < 2046u, nb = (unsigned)(b.e - 1) < 2046u;
    const bool za = is_zero_sig(x), zb = is_zero_sig(y);
    if (za || zb) {
        r = __longlong_as_double((long long)((uint64_t)(a.sign ^ b.sign) << 32));
        ok = ok && (za || na) && (zb || nb);
    } else {
        ok = ok && in_range && na && nb;
    }
    return r;
}

// x^3 from the significand's square kept to 64 bits and then times the significand once more,
// rounded once: within 1 ulp of the exact cube (and equal to its rounding but near ties); ok
// cleared where x is subnormal, infinite or NaN or the cube leaves the normal range.
__device__ __forceinline__ double cube_int(double x, bool &ok)
{
    const Sig a = split_sig(x);
    uint64_t P2 = (uint64_t)a.a1 * a.a1 + 2ull * __umulhi(a.a1, a.a0);
    const int t2 = (int)(P2 >> 63);
    P2 <<= 1 - t2;  // in [2^63, 2^64): x^2 = (P2 / 2^64) 2^(2e - 2045 + t2)
    double r;
    const bool in_range = pack_sig(mulhi_sig((uint32_t)(P2 >> 32), (uint32_t)P2, a.a1, a.a0),
                                   3 * a.e - 3067 + t2, a.sign, r);
    if (is_zero_sig(x))
        r = x;
    else
        ok = ok && in_range && (unsigned)(a.e - 1) < 2046u;
    return r;
}

// 1/x for a normal x, on the integer pipe but for one FP32 approximate reciprocal: y0, the
// special-function unit's 1/f of the significand's top 24 bits f (within 2^-22 of 1/m, m the
// significand), taken exactly as Y = y0 2^30; then e = 1 - m y0 exactly as an integer,
// E = e 2^82 = 2^82 - X Y for the integer significand X, which fits in 64 bits while |e| < 2^-19;
// and 1/m = y0 / (1 - e) = y0 (1 + e + e^2) to within e^3 (2^-66), the e^2 term from the top
// half of E.  Rounded once: within 1 ulp of 1/x (the correct rounding but near ties); ok cleared
// where x is zero, subnormal, infinite or NaN or 1/x is subnormal.
__device__ __forceinline__ double rcp_int(double x, bool &ok)
{
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu);
    const uint32_t mhi = (hi & 0xfffffu) | 0x100000u;
    float y0;
    asm("rcp.approx.ftz.f32 %0, %1;"
        : "=f"(y0)
        : "f"(__uint_as_float(0x3f800000u | ((hi & 0xfffffu) << 3) | (lo >> 29))));
    const uint32_t yb = __float_as_uint(y0);  // y0 in (1/2, 1]: biased exponent 126 or 127
    const uint32_t Y = ((yb & 0x7fffffu) | 0x800000u) << ((yb >> 23) - 120u);
    // X Y mod 2^64 for X = mhi 2^32 + lo; 2^82 is 0 mod 2^64
    const uint64_t xy = (uint64_t)lo * Y + ((uint64_t)(mhi * Y) << 32);
    const int64_t E = (int64_t)(0ull - xy);
    const int32_t Eh = (int32_t)(E >> 32);
    const int64_t T = E + (((int64_t)Eh * Eh) >> 18);  // (e + e^2) 2^82
    const int32_t Th = (int32_t)(T >> 32);
    const int64_t corr = ((int64_t)Y * Th + (int64_t)__umulhi(Y, (uint32_t)T)) >> 18;
    const uint64_t R62 = ((uint64_t)Y << 32) + (uint64_t)corr;  // (1/m) 2^62, in (2^61, 2^62]
    double r;
    const bool in_range = pack_sig(R62 << 1, 1024 - e, hi & 0x80000000u, r);
    ok = ok && in_range && (unsigned)(e - 1) < 2046u;
    return r;
}

}  // namespace
}  // namespace pab
