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

struct df64;
__device__ df64 split_double(double d);

struct __align__(8) df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr df64(int v) : hi((float)v), lo(0.0f) {}
    __host__ __device__ df64(double d);
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// hi = d rounded to FP32, lo = (d - hi) rounded to FP32.  On the device the
// split is done on the bit pattern: GB300's FP64 adder runs at a small
// fraction of the FP32 rate (a DADD per element made the canonical-to-
// double-float conversion three times slower than a copy), while integer
// operations and the narrowing conversion do not touch it.  Exact halfway
// cases of hi round away from zero instead of to even.  Zeros, values below
// 2^-74 or from 2^127 in magnitude, infinities and NaNs take the FP64 route.
__device__ __forceinline__ df64 split_double(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((u >> 52) & 0x7FF) - 1023;
    if (e < -74 || e > 126) {
        if ((u << 1) == 0) return df64(__double2float_rn(d), 0.0f);   // +-0
        const float h = __double2float_rn(d);
        return df64(h, __double2float_rn(d - (double)h));
    }
    const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
    unsigned int hb = ((unsigned int)(u >> 32) & 0x80000000u) |
                      ((unsigned int)(e + 127) << 23) | (unsigned int)(m >> 29);
    int r = (int)(m & 0x1FFFFFFFu);          // the 29 bits below hi's last
    if (r >= (1 << 28)) {                    // round hi up, remainder negative
        hb += 1u;
        r -= (1 << 29);
    }
    float lo = __int2float_rn(r) * __int_as_float((e - 52 + 127) << 23);
    if (u >> 63) lo = -lo;
    return df64(__uint_as_float(hb), lo);
}

__host__ __device__ inline df64::df64(double d) {
#ifdef __CUDA_ARCH__
    *this = split_double(d);
#else
    hi = (float)d;
    lo = (float)(d - (double)(float)d);
#endif
}

// The error-free transformations below spell every operation with the
// round-to-nearest intrinsics: nvcc contracts a multiply feeding an add into
// one FMA by default, and a sum s that is not fl(a + b) breaks their
// exactness.

// s + e = a + b exactly
__device__ __forceinline__ df64 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
    return df64(s, e);
}
// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ df64 quick_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
    df64 s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);       // exact error of the leading product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }

// Lazily normalised double-float: the value s + e where s is the FP32 sum of
// the leading parts and e collects, in plain FP32, the exact rounding error
// of every leading addition (TwoSum), the exact error of every leading
// product (one FMA) and the products with the trailing parts.  This is the
// compensated dot product "Dot2" of Ogita, Rump and Oishi (SIAM J. Sci.
// Comput. 26, 2005): a sum of n products comes out as accurate as one
// evaluated with twice the working precision, error <= gamma_n^2 sum |a_i b_i|
// with gamma_n = n u / (1 - n u), u = 2^-24.  Only s forms a serial chain
// (one FP32 add per term); everything else is independent work.
struct dfl {
    float s, e;
    dfl() = default;
    __host__ __device__ constexpr dfl(float s_, float e_) : s(s_), e(e_) {}
    __host__ __device__ constexpr dfl(int v) : s((float)v), e(0.0f) {}
    __host__ __device__ constexpr dfl(df64 a) : s(a.hi), e(a.lo) {}
};

template <int SGN>
__device__ __forceinline__ dfl lazy_add(dfl a, dfl b) {
    const float bs = SGN > 0 ? b.s : -b.s, be = SGN > 0 ? b.e : -b.e;
    const float s = __fadd_rn(a.s, bs);
    const float v = __fsub_rn(s, a.s);
    const float t = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, v)), __fsub_rn(bs, v));
    return dfl(s, a.e + (t + be));
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) { return lazy_add<1>(a, b); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return lazy_add<-1>(a, b); }
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.s, -a.e); }
__device__ __forceinline__ dfl &operator+=(dfl &a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl &operator-=(dfl &a, dfl b) { return a = a - b; }
// a * b as (leading product, exact error of it + cross products with the
// trailing parts); the trailing-times-trailing term is below 2^-48 |a b|.
__device__ __forceinline__ dfl operator*(df64 a, dfl b) {
    const float p = __fmul_rn(a.hi, b.s);
    float c = fmaf(a.hi, b.s, -p);
    c = fmaf(a.hi, b.e, c);
    c = fmaf(a.lo, b.s, c);
    return dfl(p, c);
}
__device__ __forceinline__ dfl operator*(dfl a, df64 b) { return b * a; }
// nearest normalised double-float (TwoSum of the two parts: s and e carry
// no ordering once e has collected several terms)
__device__ __forceinline__ df64 normalise(dfl a) { return two_sum(a.s, a.e); }

}  // namespace wd
