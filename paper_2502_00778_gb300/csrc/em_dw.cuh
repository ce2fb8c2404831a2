// Double-word ("DW") arithmetic on the FP32 pipe.
//
// A DW value is an unevaluated sum h + l of two floats.  The building blocks
// are the classical error-free transformations (Knuth's TwoSum, Dekker's
// Fast2Sum, the FMA-based product error); see e.g. Joldes, Muller & Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 2017.  They give ~2^-48 relative accuracy per
// operation using only FP32 instructions, which on GB300 issue 64x faster
// than FP64 instructions.
//
// Conversions between double and DW are done on the integer pipe (bit
// manipulation), because FP32<->FP64 conversion instructions run on the slow
// FP64 unit of this GPU.
//
// Every operation below is written with the round-to-nearest intrinsics
// (__fadd_rn, __fsub_rn, __fmul_rn) or an explicit fmaf: the compiler never
// fuses those into a multiply-add, whereas a plain "a*b - c" may be contracted
// into one FMA, which silently breaks the error-free transformations.
#pragma once
#include <stdint.h>

namespace em {

struct dw {
    float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dw dw_neg(dw a) { return {-a.h, -a.l}; }

// sign flip by a +-1.0f factor (exact)
__device__ __forceinline__ dw dw_sgn(dw a, float s) { return {__fmul_rn(a.h, s), __fmul_rn(a.l, s)}; }

// a - b, renormalized (|l| <= ulp(h)/2 up to one rounding)
__device__ __forceinline__ dw dw_sub_n(dw a, dw b) {
    float s, e;
    two_sum(a.h, -b.h, s, e);
    e = __fadd_rn(e, __fsub_rn(a.l, b.l));
    float r, q;
    fast_two_sum(s, e, r, q);
    return {r, q};
}

// a + b, not renormalized
__device__ __forceinline__ dw dw_add(dw a, dw b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    return {s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ dw dw_sub(dw a, dw b) {
    float s, e;
    two_sum(a.h, -b.h, s, e);
    return {s, __fadd_rn(e, __fsub_rn(a.l, b.l))};
}

// a * b (a.l * b.l dropped: below 2^-46 relative for renormalized inputs)
__device__ __forceinline__ dw dw_mul(dw a, dw b) {
    float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return {p, e};
}

// a * f for a float constant pair (fh + fl)
__device__ __forceinline__ dw dw_mulc(dw a, float fh, float fl) {
    float p = __fmul_rn(a.h, fh);
    float e = fmaf(a.h, fh, -p);
    e = fmaf(a.h, fl, e);
    e = fmaf(a.l, fh, e);
    return {p, e};
}

// p*q - r*s for DW inputs: the exact difference of the high products plus
// first-order terms
__device__ __forceinline__ dw dw_det2(dw p, dw q, dw r, dw s) {
    float a = __fmul_rn(p.h, q.h);
    float b = __fmul_rn(r.h, s.h);
    float ea = fmaf(p.h, q.h, -a);
    float eb = fmaf(r.h, s.h, -b);
    float h, t;
    two_sum(a, -b, h, t);
    float lo = __fadd_rn(t, __fsub_rn(ea, eb));
    lo = fmaf(p.h, q.l, lo);
    lo = fmaf(p.l, q.h, lo);
    lo = fmaf(-r.h, s.l, lo);
    lo = fmaf(-r.l, s.h, lo);
    return {h, lo};
}

// accumulate v into acc (unnormalized running sum)
__device__ __forceinline__ void dw_acc(dw& acc, dw v) {
    float s, e;
    two_sum(acc.h, v.h, s, e);
    acc.l = __fadd_rn(acc.l, __fadd_rn(e, v.l));
    acc.h = s;
}

__device__ __forceinline__ void dw_acc_f(dw& acc, float v) {
    float s, e;
    two_sum(acc.h, v, s, e);
    acc.l = __fadd_rn(acc.l, e);
    acc.h = s;
}

// double -> DW (truncated high part, remaining bits in the low part);
// values below 2^-126 in magnitude map to 0; NaN, infinities and finite
// values of magnitude 2^128 or more (outside the float range) map to NaN
__device__ __forceinline__ dw dw_from_double(double d) {
    unsigned long long b = (unsigned long long)__double_as_longlong(d);
    int e = (int)((b >> 52) & 0x7ff);
    int ef = e - 1023 + 127;
    if (ef <= 0) return {0.f, 0.f};
    if (ef >= 255) return {__int_as_float(0x7fc00000), __int_as_float(0x7fc00000)};
    unsigned sign = (unsigned)(b >> 63) << 31;
    float hi = __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)((b >> 29) & 0x7fffff));
    unsigned r = (unsigned)(b & 0x1fffffffu);
    int el = e - 1075 + 127;               // exponent of 2^(e - 1075)
    float lo = 0.f;
    if (el > 0) lo = __fmul_rn(__uint2float_rn(r), __uint_as_float((unsigned)el << 23));
    return {hi, sign ? -lo : lo};
}

// double -> float by truncation of the mantissa (integer pipe only)
__device__ __forceinline__ float f_from_double(double d) { return dw_from_double(d).h; }

// DW -> double, correctly rounded up to one ulp, without FP64 instructions;
// a non-finite sum gives NaN
__device__ __forceinline__ double dw_to_double(dw a) {
    float s, e;
    two_sum(a.h, a.l, s, e);
    if (s == 0.f) return 0.0;
    unsigned sb = __float_as_uint(s);
    unsigned sign = sb >> 31;
    int ex = (int)((sb >> 23) & 0xff);
    if (ex == 0) return 0.0;
    if (ex == 255 || e != e) return __longlong_as_double(0x7ff8000000000000LL);
    long long M = (1LL << 52) | ((long long)(sb & 0x7fffff) << 29);
    int k = 0;
    int sc = 306 - ex;                      // e * 2^(179 - ex): e in units of the double ulp of s
    if (e != 0.f && sc > 0 && sc < 255) k = __float2int_rn(__fmul_rn(e, __uint_as_float((unsigned)sc << 23)));
    M += sign ? -(long long)k : (long long)k;
    long long E = ex - 127 + 1023;
    if (M >= (1LL << 53)) {
        M = (M + 1) >> 1;
        E += 1;
    } else if (M < (1LL << 52)) {
        M <<= 1;
        E -= 1;
    }
    unsigned long long bits = ((unsigned long long)sign << 63) | ((unsigned long long)E << 52) |
                              ((unsigned long long)M & ((1ULL << 52) - 1));
    return __longlong_as_double((long long)bits);
}

// float -> double on the integer pipe (exact; denormals map to 0, NaN and
// infinities to NaN)
__device__ __forceinline__ double f_to_double(float f) {
    unsigned b = __float_as_uint(f);
    int ex = (int)((b >> 23) & 0xff);
    if (ex == 0) return 0.0;
    if (ex == 255) return __longlong_as_double(0x7ff8000000000000LL);
    unsigned long long bits = ((unsigned long long)(b >> 31) << 63) | ((unsigned long long)(ex - 127 + 1023) << 52) |
                              ((unsigned long long)(b & 0x7fffff) << 29);
    return __longlong_as_double((long long)bits);
}

}  // namespace em
