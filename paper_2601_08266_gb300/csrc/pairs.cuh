// pairs.cuh -- two independent values of one compute type carried together.
//
// The sm_100-family FP32 pipe has paired instructions (FADD2, FMUL2, FFMA2):
// one issue slot does the work of two scalar ones on a float2.  The VMS
// operators are bound by issue slots, and the Q1 evaluation/projection
// butterflies run the same instruction sequence for every field, so two fields
// at a time go through these pairs.  float and double-float pairs use the
// paired intrinsics (__fadd2_rn, __fmul2_rn, __ffma2_rn): each half rounds to
// nearest exactly like the scalar operation.  The double-float pair performs
// the scalar double-float sequence operation for operation, so its results
// equal the scalar code's bit for bit; a float pair fixes where a*b + c*d is
// contracted into an FMA, which the compiler chooses freely in scalar code.
// double has no paired form; its pair is two scalars.
#pragma once

#include <cuda_runtime.h>

#include "df64.cuh"

namespace fsi {

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 shfl2(float2 v, int m)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// ---------------------------------------------------------------- float pair
struct f32x2 {
    float2 v;
};
__device__ __forceinline__ f32x2 operator+(f32x2 a, f32x2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ f32x2 operator-(f32x2 a, f32x2 b)
{
    return {__fadd2_rn(a.v, neg2(b.v))};
}
__device__ __forceinline__ f32x2 operator*(f32x2 a, f32x2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ f32x2 pair_fma(f32x2 a, f32x2 b, f32x2 c)
{
    return {__ffma2_rn(a.v, b.v, c.v)};
}
__device__ __forceinline__ f32x2 pair_dot2(f32x2 a, f32x2 b, f32x2 c, f32x2 d)
{
    return {__ffma2_rn(a.v, b.v, __fmul2_rn(c.v, d.v))};
}
__device__ __forceinline__ f32x2 pair_shx(f32x2 a, int m) { return {shfl2(a.v, m)}; }

// --------------------------------------------------------- double-float pair
// The same error-free transformations as df64.cuh, on both halves at once.
struct df64x2 {
    float2 hi, lo;
};
__device__ __forceinline__ df64x2 two_sum2(float2 a, float2 b)
{
    const float2 s = __fadd2_rn(a, b);
    const float2 bb = __fadd2_rn(s, neg2(a));
    const float2 e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(b, neg2(bb)));
    return {s, e};
}
__device__ __forceinline__ df64x2 fast_two_sum2(float2 a, float2 b)
{
    const float2 s = __fadd2_rn(a, b);
    return {s, __fadd2_rn(b, neg2(__fadd2_rn(s, neg2(a))))};
}
__device__ __forceinline__ df64x2 operator+(df64x2 a, df64x2 b)
{
    const df64x2 s = two_sum2(a.hi, b.hi);
    return fast_two_sum2(s.hi, __fadd2_rn(s.lo, __fadd2_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df64x2 operator-(df64x2 a) { return {neg2(a.hi), neg2(a.lo)}; }
__device__ __forceinline__ df64x2 operator-(df64x2 a, df64x2 b) { return a + (-b); }
// exact product error of the high parts plus the cross terms
__device__ __forceinline__ float2 prod_err2(df64x2 a, df64x2 b, float2 p)
{
    float2 e = __ffma2_rn(a.hi, b.hi, neg2(p));
    e = __ffma2_rn(a.hi, b.lo, e);
    return __ffma2_rn(a.lo, b.hi, e);
}
__device__ __forceinline__ df64x2 operator*(df64x2 a, df64x2 b)
{
    const float2 p = __fmul2_rn(a.hi, b.hi);
    return fast_two_sum2(p, prod_err2(a, b, p));
}
__device__ __forceinline__ df64x2 pair_fma(df64x2 a, df64x2 b, df64x2 c)
{
    const float2 p = __fmul2_rn(a.hi, b.hi);
    const float2 e = prod_err2(a, b, p);
    const df64x2 s = two_sum2(p, c.hi);
    return fast_two_sum2(s.hi, __fadd2_rn(s.lo, __fadd2_rn(e, c.lo)));
}
__device__ __forceinline__ df64x2 pair_dot2(df64x2 a, df64x2 b, df64x2 c, df64x2 d)
{
    const float2 p = __fmul2_rn(a.hi, b.hi);
    const float2 e = prod_err2(a, b, p);
    const float2 q = __fmul2_rn(c.hi, d.hi);
    const float2 f = prod_err2(c, d, q);
    const df64x2 s = two_sum2(p, q);
    return fast_two_sum2(s.hi, __fadd2_rn(s.lo, __fadd2_rn(e, f)));
}
__device__ __forceinline__ df64x2 pair_shx(df64x2 a, int m) { return {shfl2(a.hi, m), shfl2(a.lo, m)}; }

// ---------------------------------------------------------------- generic pair
template <typename T> struct pair2 {
    T a, b;
};
template <typename T> __device__ __forceinline__ pair2<T> operator+(pair2<T> x, pair2<T> y)
{
    return {x.a + y.a, x.b + y.b};
}
template <typename T> __device__ __forceinline__ pair2<T> operator-(pair2<T> x, pair2<T> y)
{
    return {x.a - y.a, x.b - y.b};
}
template <typename T> __device__ __forceinline__ pair2<T> operator*(pair2<T> x, pair2<T> y)
{
    return {x.a * y.a, x.b * y.b};
}
template <typename T> __device__ __forceinline__ pair2<T> pair_fma(pair2<T> x, pair2<T> y, pair2<T> z)
{
    return {x.a * y.a + z.a, x.b * y.b + z.b};
}
template <typename T>
__device__ __forceinline__ pair2<T> pair_dot2(pair2<T> x, pair2<T> y, pair2<T> z, pair2<T> w)
{
    return {x.a * y.a + z.a * w.a, x.b * y.b + z.b * w.b};
}
template <typename T> __device__ __forceinline__ pair2<T> pair_shx(pair2<T> x, int m)
{
    return {__shfl_xor_sync(0xffffffffu, x.a, m), __shfl_xor_sync(0xffffffffu, x.b, m)};
}

// ------------------------------------------------- pair type of a compute type
template <typename T> struct PairOf {
    using type = pair2<T>;
    static __device__ __forceinline__ type pack(T a, T b) { return {a, b}; }
    static __device__ __forceinline__ T first(type p) { return p.a; }
    static __device__ __forceinline__ T second(type p) { return p.b; }
};
template <> struct PairOf<float> {
    using type = f32x2;
    static __device__ __forceinline__ type pack(float a, float b) { return {make_float2(a, b)}; }
    static __device__ __forceinline__ float first(type p) { return p.v.x; }
    static __device__ __forceinline__ float second(type p) { return p.v.y; }
};
template <> struct PairOf<df64> {
    using type = df64x2;
    static __device__ __forceinline__ type pack(df64 a, df64 b)
    {
        return {make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)};
    }
    static __device__ __forceinline__ df64 first(type p) { return df64(p.hi.x, p.lo.x); }
    static __device__ __forceinline__ df64 second(type p) { return df64(p.hi.y, p.lo.y); }
};

}  // namespace fsi
