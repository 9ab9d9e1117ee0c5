// df64.cuh -- float-float ("double-single") arithmetic for an FP64-class
// solve on the FP32 units.
//
// A value is hi + lo with |lo| <= ulp(hi) / 2, about 48 significant bits.
// The building blocks are the error-free transformations of Knuth (two-sum)
// and Dekker (fast two-sum), and the fused multiply-add for the exact
// product error:
//   add: (s, e) = two_sum(a.hi, b.hi); e += a.lo + b.lo; fast_two_sum(s, e)
//        -- the "sloppy" sum, whose error is relative to |a| + |b|, which is
//        the bound an FFT's normwise error analysis uses anyway;
//   mul: p = a.hi b.hi; e = fma(a.hi, b.hi, -p) + a.hi b.lo + a.lo b.hi;
//        fast_two_sum(p, e).
// Only sums and explicit fma() calls appear, so contraction of a * b + c by
// the compiler cannot change the rounding of the error-free steps.
#pragma once
#include <math.h>

namespace isofft {

struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    // exact split of a double into the nearest float and the float nearest
    // to the remainder
    __host__ __device__ constexpr df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr explicit df64(int i) : hi((float)i), lo(0.0f) {}
    __host__ __device__ constexpr double to_double() const { return (double)hi + (double)lo; }
};

__host__ __device__ __forceinline__ df64 df64_fast_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}

__host__ __device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    return df64_fast_two_sum(s, e);
}

// The sum without its closing renormalisation: hi = fl(a.hi + b.hi) and lo
// its exact error plus a.lo + b.lo.  hi + lo is the same sloppy sum, but lo
// may exceed half an ulp of hi (by a few ulps along a chain of such sums,
// and more where hi cancels).  The FFT engine's butterflies chain these and
// renormalise (df64_renorm) before any product, whose error term drops
// lo x lo and so needs |lo| << |hi|.
__host__ __device__ __forceinline__ df64 df64_add_lazy(df64 a, df64 b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return {s, e + (a.lo + b.lo)};
}
// The product without its closing renormalisation (its lo is the exact
// error of hi plus the cross terms, within a few ulps of hi): for products
// that only enter sums.  Both operands must be normalised.
__host__ __device__ __forceinline__ df64 df64_mul_lazy(df64 a, df64 b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return {p, e};
}
__host__ __device__ __forceinline__ df64 df64_renorm(df64 a)
{
    return df64_fast_two_sum(a.hi, a.lo);
}

__host__ __device__ __forceinline__ df64 operator-(df64 a) { return {-a.hi, -a.lo}; }
__host__ __device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__host__ __device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df64_fast_two_sum(p, e);
}

__host__ __device__ __forceinline__ bool operator>(df64 a, df64 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

// The real type an API buffer holds for arithmetic type T (df64 solves read
// and write FP64 arrays).
template <typename T>
struct IoReal {
    using type = T;
    static __host__ __device__ __forceinline__ T in(T v) { return v; }
    static __host__ __device__ __forceinline__ T out(T v) { return v; }
};
template <>
struct IoReal<df64> {
    using type = double;
    static __host__ __device__ __forceinline__ df64 in(double v) { return df64(v); }
    static __host__ __device__ __forceinline__ double out(df64 v) { return v.to_double(); }
};

}  // namespace isofft
