// df64.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo
// of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.  Built
// from error-free transformations: Knuth's TwoSum for sums, the exact
// product error given by an FMA (Dekker's product), and a Newton step for
// 1/sqrt.  On GB300 the FP32 pipe runs ~70x the FP64 rate, so FP64-accurate
// operators computed this way outrun native FP64.
//
// No fast-math: the transformations rely on IEEE round-to-nearest FP32
// additions in program order (nvcc preserves that without --use_fast_math;
// the products use explicit fmaf).
#pragma once

#include <cuda_runtime.h>

namespace fsi {

struct df64 {
    float hi, lo;
    __host__ __device__ df64() {}
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    // exact split of a double into hi + lo (rounded once to 48 bits)
    __host__ __device__ df64(double d)
    {
        hi = (float)d;
        lo = (float)(d - (double)hi);
    }
    __host__ __device__ constexpr explicit df64(float h) : hi(h), lo(0.0f) {}
    // small integers are exact in one float
    __host__ __device__ constexpr df64(int i) : hi((float)i), lo(0.0f) {}
    __host__ __device__ double to_double() const { return (double)hi + (double)lo; }
};

// Split of a double into hi + lo with integer operations only (no FP64
// instruction): hi keeps the sign, the exponent and the leading 24
// significant bits (truncated), lo the next 24 of the remaining 29 bits
// (truncated), so hi + lo equals d to 2^-47 relative.  Zero and magnitudes
// outside the normal float range take the float conversion path.
__device__ __forceinline__ df64 df_split(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
    const int e = (int)((hw >> 20) & 0x7FFu);
    const int fe = e - 1023 + 127;
    if (e == 0 || fe <= 0 || fe >= 255) return df64((float)d, 0.0f);
    const unsigned sign = hw & 0x80000000u;
    const unsigned hm = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | hm);
    const unsigned r = lw & 0x1FFFFFFFu;  // d - hi = r * 2^(e - 1075)
    if (r == 0) return df64(hi, 0.0f);
    const int top = 31 - __clz((int)r);   // leading bit of r, 0..28
    const unsigned mant = top >= 23 ? (r >> (top - 23)) : (r << (23 - top));
    const int le = e - 1075 + top + 127;
    if (le <= 0) return df64(hi, 0.0f);
    return df64(hi, __uint_as_float(sign | ((unsigned)le << 23) | (mant & 0x7FFFFFu)));
}

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df64 df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df64(s, e);
}

// s + e = a + b exactly, given |a| >= |b|
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return df64(s, e);
}

// Sum: exact sum of the high parts, the low parts added in FP32, one
// renormalisation.  The error is bounded by a few units of 2^-47 of
// max(|a|, |b|) (not of |a + b|): enough for FP64-level results unless a
// difference cancels many digits, which the operators' tests bound.
__device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    const df64 s = df_two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return df_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the product
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

// a b + c: the exact product error and the low parts join the sum before
// one renormalisation (the product is not renormalised on its own).  Error
// a few units of 2^-47 of max(|a b|, |c|), like a product followed by a sum.
__device__ __forceinline__ df64 df_fma(df64 a, df64 b, df64 c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const df64 s = df_two_sum(p, c.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

// a b + c d with one renormalisation
__device__ __forceinline__ df64 df_dot2(df64 a, df64 b, df64 c, df64 d)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float q = __fmul_rn(c.hi, d.hi);
    float f = __fmaf_rn(c.hi, d.hi, -q);
    f = __fmaf_rn(c.hi, d.lo, f);
    f = __fmaf_rn(c.lo, d.hi, f);
    const df64 s = df_two_sum(p, q);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, f)));
}

// a b + c in any compute type: the plain expression (contracted to an FMA)
// for float and double, df_fma for double-float
template <typename T> __device__ __forceinline__ T madd(T a, T b, T c) { return a * b + c; }
template <> __device__ __forceinline__ df64 madd<df64>(df64 a, df64 b, df64 c)
{
    return df_fma(a, b, c);
}

__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }

// 1/sqrt(x): float estimate, then one Newton step r += r (1 - x r^2) / 2 in
// double-float (doubles the ~23 correct bits)
__device__ __forceinline__ df64 df_rsqrt(df64 x)
{
    const df64 r(rsqrtf(x.hi), 0.0f);
    const df64 one(1.0f, 0.0f), half(0.5f, 0.0f);
    const df64 corr = one - x * (r * r);
    return r + r * (corr * half);
}

// 1/x: float reciprocal, then one Newton step r += r (1 - x r) in
// double-float (doubles the ~24 correct bits)
__device__ __forceinline__ df64 df_rcp(df64 x)
{
    const df64 r(__frcp_rn(x.hi), 0.0f);
    const df64 one(1.0f, 0.0f);
    return r + r * (one - x * r);
}

__device__ __forceinline__ df64 df_shfl_xor(df64 v, int m)
{
    return df64(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}


// Storage (I/O) type of a compute type: double-float computes on FP64 data.
template <typename C> struct StorageOf {
    using type = C;
};
template <> struct StorageOf<df64> {
    using type = double;
};

template <typename C> __device__ __forceinline__ C to_c(typename StorageOf<C>::type v)
{
    return C(v);
}

template <> __device__ __forceinline__ df64 to_c<df64>(double v) { return df_split(v); }

template <typename C> __device__ __forceinline__ typename StorageOf<C>::type to_s(C v)
{
    return v;
}
template <> __device__ __forceinline__ double to_s<df64>(df64 v) { return v.to_double(); }

template <typename T> __device__ __forceinline__ T shfl_x(T v, int m)
{
    return __shfl_xor_sync(0xffffffffu, v, m);
}
template <> __device__ __forceinline__ df64 shfl_x<df64>(df64 v, int m) { return df_shfl_xor(v, m); }

}  // namespace fsi
