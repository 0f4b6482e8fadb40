// Double-float arithmetic: a real as the unevaluated sum hi + lo of two
// FP32 numbers (|lo| <= ulp(hi) / 2), about 48 significand bits.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so the
// reliable-update residuals r = b - M x can run faster on the FP32 pipes in
// this form than in native FP64.  The algorithms are the classical
// error-free transformations: Knuth's TwoSum (The Art of Computer
// Programming, vol. 2, 4.2.2) and Dekker's product (1971, "A floating-point
// technique for extending the available precision") with the exact product
// error taken from one FMA; additions use the short (non-IEEE) double-double
// form, whose error is bounded by a few units of 2^-48 of the operands'
// magnitude -- enough for residuals required to 1e-10 of |b|.
#pragma once

#include <cuda_runtime.h>

namespace wd {

struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr df64(int v) : hi((float)v), lo(0.0f) {}
    __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly
__device__ __forceinline__ df64 two_sum(float a, float b) {
    const float s = a + b;
    const float v = s - a;
    const float e = (a - (s - v)) + (b - v);
    return df64(s, e);
}
// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ df64 quick_two_sum(float a, float b) {
    const float s = a + b;
    return df64(s, b - (s - a));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
    df64 s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);       // exact error of the leading product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }

}  // namespace wd
