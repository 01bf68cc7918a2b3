// Float-float ("double-float") arithmetic: a value is an unevaluated sum hi + lo of two float32 numbers with
// |lo| <= ulp(hi)/2, about 48 significant bits.  Built from the error-free transformations of Knuth's TwoSum
// (TAOCP vol. 2, 4.2.2) and the FMA form of Dekker's TwoProduct (Dekker 1971): every rounding error of a sum or
// product is recovered exactly and carried in lo.  All operations use the _rn intrinsics, so the compiler
// cannot contract or reassociate them.  On GB300 float64 runs at 1/62 of the float32 rate; a float-float
// product or sum costs 4 to 20 float32 operations, so float64-accurate link updates are several times cheaper
// this way.
#pragma once
#include <cuda_runtime.h>

namespace rm {

struct dfl { float hi, lo; };
struct cdfl { dfl re, im; };

__device__ __forceinline__ dfl df_make(float h, float l) { dfl r; r.hi = h; r.lo = l; return r; }
// s + e = a + b exactly (TwoSum)
__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df_make(s, e);
}
// the same when |a| >= |b|
__device__ __forceinline__ dfl quick_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// Conversions between float64 and float pairs from the IEEE-754 bit fields, with integer operations and no
// float64 arithmetic (float64 runs at a small fraction of the float32 rate on this part).  df_split: hi = x
// rounded to 24 significant bits (its 29 low significand bits dropped, rounding half away from zero, a carry
// moving into the exponent), lo = the signed remainder (at most 2^28 units of x's last place) as a float times
// 2^(e - 52); |lo| <= ulp(hi) / 2 and hi + lo = x to 2^-49 |x|.  |x| below 2^-126 gives 0 and |x|
// near or above 2^128 gives +-inf (NaN too); lo is dropped for |x| < 2^-74 (an absolute error below 2^-98).
__device__ __forceinline__ dfl df_split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 1023 - 126) return df_make(__uint_as_float(sign), __uint_as_float(sign));
    const unsigned long long m = b & 0x1fffffffull;
    const bool up = m >= (1ull << 28);
    const unsigned long long bh = (b & ~0x1fffffffull) + (up ? (1ull << 29) : 0ull);
    const int eh = (int)((bh >> 52) & 0x7ff);
    if (eh > 1023 + 127) return df_make(__uint_as_float(sign | 0x7f800000u), 0.f);
    const float hi = __uint_as_float(sign | ((unsigned)(eh - 1023 + 127) << 23) | (unsigned)((bh >> 29) & 0x7fffffu));
    float lo = 0.f;
    if (e >= 949) {   // 2^(e - 1075) is a normal float
        const int r = up ? (int)m - (1 << 29) : (int)m;
        lo = __int2float_rn(r) * __uint_as_float((unsigned)(e - 948) << 23);
        if (sign) lo = -lo;
    }
    return df_make(hi, lo);
}
// a float as a double, from its bit fields (normal numbers, zero, inf and NaN; subnormals give 0)
__device__ __forceinline__ double f_to_d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned fe = (u >> 23) & 0xffu;
    if (fe == 0) return __longlong_as_double((long long)sign);
    const unsigned long long de = fe == 255 ? 0x7ffull : (unsigned long long)(fe - 127 + 1023);
    return __longlong_as_double((long long)(sign | (de << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}
// hi + lo as a double: one float64 addition, exact (the two parts span at most 49 bits)
__device__ __forceinline__ double df_join(dfl a) { return f_to_d_bits(a.hi) + f_to_d_bits(a.lo); }

// a + b with an error below 2^-47 (|a| + |b|): the low parts are added without their own TwoSum, which is
// accurate relative to the operands (not to a cancelled result) -- enough here, where every value is an
// entry or coefficient of order 1 and the link update needs absolute accuracy
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    const dfl s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl df_neg(dfl a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ dfl df_mulf(dfl a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ dfl df_zero() { return df_make(0.f, 0.f); }

__device__ __forceinline__ cdfl cdf_make(dfl re, dfl im) { cdfl r; r.re = re; r.im = im; return r; }
__device__ __forceinline__ cdfl cdf_add(cdfl a, cdfl b) { return cdf_make(df_add(a.re, b.re), df_add(a.im, b.im)); }
__device__ __forceinline__ cdfl cdf_sub(cdfl a, cdfl b) { return cdf_make(df_sub(a.re, b.re), df_sub(a.im, b.im)); }
__device__ __forceinline__ cdfl cdf_conj(cdfl a) { return cdf_make(a.re, df_neg(a.im)); }
__device__ __forceinline__ cdfl cdf_mul(cdfl a, cdfl b) {
    return cdf_make(df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re)));
}
__device__ __forceinline__ cdfl cdf_scale(cdfl a, dfl s) { return cdf_make(df_mul(a.re, s), df_mul(a.im, s)); }
// |a|^2
__device__ __forceinline__ dfl cdf_norm(cdfl a) { return df_add(df_mul(a.re, a.re), df_mul(a.im, a.im)); }

// 1/sqrt(a) for a > 0: float32 estimate, then one Newton step y + y (1 - a y^2) / 2 in float-float
__device__ __forceinline__ dfl df_rsqrt(dfl a) {
    const dfl y = df_make(rsqrtf(a.hi), 0.f);
    const dfl r = df_sub(df_make(1.f, 0.f), df_mul(a, df_mul(y, y)));
    return df_add(y, df_mul(y, df_mulf(r, 0.5f)));
}

}  // namespace rm
