// Double-binary32 ("double-float") arithmetic: a value is hi + lo with two
// binary32 numbers, |lo| <= ulp(hi)/2, about 48 significant bits. Built from
// error-free transformations: Knuth's TwoSum, Dekker's FastTwoSum, and the
// FMA-based TwoProduct (see Ogita, Rump & Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26 (2005)). On a GB300 the binary32 pipes
// run 64 times the binary64 FMA rate, so these ~7-11 binary32 operations per
// double-float operation still outrun native binary64.
//
// The exponent range is binary32's (|x| < 3.4e38; the low part underflows
// below ~1e-38 * 2^-24); the kernels keep every quantity in range by
// construction (scaled node weights, normalised angular sums).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace gfc {

// the binary32/binary64 overloads stay visible next to the df ones below
using ::fabs;
using ::fma;
using ::fmin;

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    // from a binary64 value: hi = nearest binary32, lo = the rest rounded
    __host__ __device__ explicit df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit df(int i) : hi((float)i), lo(0.0f) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

#if defined(__CUDACC__)

__device__ __forceinline__ df df_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df(s, e);
}

// requires |a| >= |b| (or a = 0)
__device__ __forceinline__ df df_fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df(s, e);
}

__device__ __forceinline__ df df_two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return df(p, e);
}

// a + b by Dekker's add: TwoSum of the high parts, the low parts added in
// binary32. Its error is ~2^-48 (|a| + |b|): relative to a + b it grows with
// cancellation, as the rounding already carried by computed a and b does; the
// kernels add no operands that are exact and cancel, so the second TwoSum of
// the fully accurate add (~20 operations instead of ~11) would buy nothing.
__device__ __forceinline__ df operator+(df a, df b)
{
    df s = df_two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b)
{
    df p = df_two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return df_fast_two_sum(p.hi, p.lo);
}

// a b + c in one pass: the product's high part exactly (FMA TwoProduct) with
// its low-order terms gathered before Dekker's add, one renormalisation at the
// end (~15 binary32 operations instead of ~18 for a product, then an add)
__device__ __forceinline__ df fma(df a, df b, df c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, pe));
    df s = df_two_sum(p, c.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(pe, c.lo));
    return df_fast_two_sum(s.hi, s.lo);
}

// Sums of positive products e r without renormalising every term: cascaded
// summation (Ogita, Rump & Oishi 2005, Sum2, with FMA products). The high
// parts accumulate by TwoSum; each TwoSum error, the product's rounding error
// (FMA TwoProduct) and the low-order product terms e.hi r.lo + e.lo r.hi go to
// the low part; pos_finish renormalises once. ~12 binary32 operations a term
// instead of ~18 for a double-float product and add; the rounding error grows
// like n 2^-48 over n positive terms (against ~sqrt(n) 2^-48 renormalising
// every term).
__device__ __forceinline__ void pos_acc(df &s, df e, df r)
{
    const float p = __fmul_rn(e.hi, r.hi);
    const float pe = __fmaf_rn(e.hi, r.hi, -p);
    const float low = __fmaf_rn(e.hi, r.lo, __fmaf_rn(e.lo, r.hi, pe));
    const df t = df_two_sum(s.hi, p);
    s.hi = t.hi;
    s.lo = __fadd_rn(s.lo, __fadd_rn(t.lo, low));
}
__device__ __forceinline__ df pos_finish(df s) { return df_fast_two_sum(s.hi, s.lo); }

// 1/a: binary32 seed r, then one Newton step r (1 + e), e = 1 - a r, which
// doubles the ~23 correct bits of the seed. e is formed almost exactly in
// binary32: a.hi r = p + pe exactly (FMA TwoProduct), 1 - p is exact because
// p is within 2^-22 of 1 (Sterbenz), and a.lo r is below 2^-23; so the only
// double-float work left is the final FastTwoSum.
__device__ __forceinline__ df rcp(df a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a.hi));
    float p = __fmul_rn(a.hi, r);
    float pe = __fmaf_rn(a.hi, r, -p);
    float e = __fmaf_rn(-a.lo, r, __fsub_rn(__fsub_rn(1.0f, p), pe));
    return df_fast_two_sum(r, __fmul_rn(r, e));
}

__device__ __forceinline__ df operator/(df a, df b) { return a * rcp(b); }

// square root: binary32 seed, one Newton step on x = s + (a - s^2)/(2 s)
__device__ __forceinline__ df tsqrt(df a)
{
    if (a.hi <= 0.0f) return df(0.0f, 0.0f);
    float s = sqrtf(a.hi);
    df s2 = df_two_prod(s, s);
    df d = a - s2;
    float corr = __fdiv_rn(d.hi, 2.0f * s);
    return df_fast_two_sum(s, corr);
}

__device__ __forceinline__ df fabs(df a) { return a.hi < 0.0f ? -a : a; }
__device__ __forceinline__ df fmin(df a, df b) { return (a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo)) ? a : b; }
__device__ __forceinline__ bool operator<(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df a, df b) { return b < a; }
__device__ __forceinline__ bool operator>=(df a, df b) { return !(a < b); }
__device__ __forceinline__ bool operator<=(df a, df b) { return !(b < a); }
__device__ __forceinline__ bool operator==(df a, df b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ df &operator+=(df &a, df b) { a = a + b; return a; }
__device__ __forceinline__ df &operator*=(df &a, df b) { a = a * b; return a; }

#endif  // __CUDACC__

}  // namespace gfc
