// dfloat.cuh -- double-float arithmetic on the FP32 pipes.
//
// A dfloat is the unevaluated sum h + l of two FP32 numbers with |l| well below |h| (a few ulp(h)
// at most): about 48 significant bits with FP32's exponent range.  GB300 executes FP32 at many
// times its FP64 rate, so an operator evaluated in dfloat gives nearly FP64 accuracy at FP32-pipe
// throughput.
//
// Building blocks (both exact):
//   two_sum(a, b)  -> (s, e): s = fl(a + b), s + e = a + b                (Knuth, TAOCP 2, 4.2.2)
//   two_prod(a, b) -> (p, e): p = fl(a b), e = fma(a, b, -p), p + e = a b
// A product keeps the exact product of the high words plus the two cross terms (the low-low term
// lies below the format's precision) as an unnormalised pair `dprod` -- the cheap double-word
// product of Joldes, Muller and Popescu (ACM TOMS 44(2), 2017) without its final normalisation.
// A sum adds the high words with two_sum and the low words and the rounding error with plain
// adds, and keeps the result unnormalised (the error word of a compensated sum, as in the
// summation of Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26, 2005): a multiply-add costs 12 FP32
// operations and its dependency chain through the high word is one add long.  The absolute error
// of a sum of n such products is a small multiple of n u^2 sum |terms|, u = 2^-24 -- the form of the
// FP64 bound n 2^-53 sum |terms|, with u^2 = 2^-48 in its place.
//
// Every FP32 operation is an explicitly rounded intrinsic, so the compiler neither contracts nor
// reorders them (which would break the error-free transforms).
#pragma once

#include <cuda_runtime.h>

namespace feod {

struct __align__(8) dfloat {
    float h, l;
    dfloat() = default;
    __host__ __device__ constexpr explicit dfloat(int i) : h((float)i), l(0.f) {}
    // nearest dfloat to x: h = fl32(x), l = fl32(x - h) (x - h is exact in FP64)
    __host__ __device__ explicit dfloat(double x) : h((float)x), l((float)(x - (double)(float)x)) {}
    // h + l rounded once to FP64
    __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
};

// unnormalised product: value p + e, |e| of order u |p|
struct dprod {
    float p, e;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ dprod operator*(dfloat x, dfloat y)
{
    dprod r;
    r.p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -r.p);
    e = __fmaf_rn(x.h, y.l, e);
    r.e = __fmaf_rn(x.l, y.h, e);
    return r;
}

// (a1 + a2) + (b1 + b2) with a1, b1 the leading words: two_sum of the leading words, the rest
// into the low word (unnormalised)
__device__ __forceinline__ dfloat df_add(float a1, float a2, float b1, float b2)
{
    dfloat r;
    float e;
    two_sum(a1, b1, r.h, e);
    r.l = __fadd_rn(e, __fadd_rn(a2, b2));
    return r;
}

__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) { return df_add(x.h, x.l, y.h, y.l); }
__device__ __forceinline__ dfloat operator+(dfloat x, dprod y) { return df_add(x.h, x.l, y.p, y.e); }
__device__ __forceinline__ dfloat operator+(dprod x, dfloat y) { return df_add(y.h, y.l, x.p, x.e); }
__device__ __forceinline__ dfloat operator+(dprod x, dprod y) { return df_add(x.p, x.e, y.p, y.e); }
__device__ __forceinline__ dfloat &operator+=(dfloat &x, dfloat y) { return x = x + y; }
__device__ __forceinline__ dfloat &operator+=(dfloat &x, dprod y) { return x = x + y; }

// Two independent dfloats in the two lanes of float2 words, for the packed FP32 instructions
// (fma.rn.f32x2, add.rn.f32x2, mul.rn.f32x2): one packed instruction does the work of two scalar
// ones, and each lane's result is bit for bit that of the scalar operation on that lane.
struct df2 {
    float2 h, l;
};

// A packed coefficient: high words, low words and negated high words (a product's high term is
// formed negated where its exact error needs -p, since there is no packed subtraction).
struct df2c {
    float2 h, l, nh;
};

__host__ __device__ inline df2c df2c_pack(dfloat a, dfloat b)
{
    return df2c{ make_float2(a.h, b.h), make_float2(a.l, b.l), make_float2(-a.h, -b.h) };
}

// the packed two-lane FP32 instructions exist on sm_100 and later (device code only)
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
#define FEOD_F32X2 1
#endif

#ifdef FEOD_F32X2
__device__ __forceinline__ df2 df2_bcast(dfloat x) { return df2{ make_float2(x.h, x.h), make_float2(x.l, x.l) }; }
__device__ __forceinline__ df2c df2c_bcast(dfloat x)
{
    return df2c{ make_float2(x.h, x.h), make_float2(x.l, x.l), make_float2(-x.h, -x.h) };
}
__device__ __forceinline__ df2 df2_pack(dfloat a, dfloat b) { return df2{ make_float2(a.h, b.h), make_float2(a.l, b.l) }; }
__device__ __forceinline__ dfloat df2_lo(const df2 &v) { dfloat r; r.h = v.h.x; r.l = v.l.x; return r; }
__device__ __forceinline__ dfloat df2_hi(const df2 &v) { dfloat r; r.h = v.h.y; r.l = v.l.y; return r; }
__device__ __forceinline__ df2 df2_zero() { return df2{ make_float2(0.f, 0.f), make_float2(0.f, 0.f) }; }

// fl(a - b) lane by lane: fma(b, -1, a) rounds a - b once, as a scalar subtraction does
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// acc += c x lane by lane (the scalar acc + c * x: the product of Joldes, Muller and Popescu
// without normalisation, then the compensated sum)
__device__ __forceinline__ void df2_fma(df2 &acc, const df2c &c, const df2 &x)
{
    const float2 np = __fmul2_rn(c.nh, x.h);          // -fl(ch xh)
    float2 e = __ffma2_rn(c.h, x.h, np);              // ch xh - p, exact
    e = __ffma2_rn(c.h, x.l, e);
    e = __ffma2_rn(c.l, x.h, e);
    // two_sum(acc.h, p) with p = -np: s = fl(acc.h + p), bb = s - acc.h,
    // err = (acc.h - (s - bb)) + (p - bb)
    const float2 s = sub2(acc.h, np);
    const float2 bb = sub2(s, acc.h);
    const float2 e1 = sub2(acc.h, sub2(s, bb));
    const float2 e2 = __fadd2_rn(np, bb);             // -(p - bb)
    const float2 es = sub2(e1, e2);
    acc.l = __fadd2_rn(es, __fadd2_rn(acc.l, e));
    acc.h = s;
}

// the unnormalised product t g lane by lane (the scalar t * g), given ngh = -g.h
struct dprod2 {
    float2 p, e;
};
__device__ __forceinline__ dprod2 df2_mul(const df2 &t, const df2 &g, float2 ngh)
{
    dprod2 r;
    r.p = __fmul2_rn(t.h, g.h);
    const float2 np = __fmul2_rn(t.h, ngh);            // -p exactly
    float2 e = __ffma2_rn(t.h, g.h, np);
    e = __ffma2_rn(t.h, g.l, e);
    r.e = __ffma2_rn(t.l, g.h, e);
    return r;
}

// (a1 + a2) + (b1 + b2) lane by lane, as df_add
__device__ __forceinline__ df2 df2_add(float2 a1, float2 a2, float2 b1, float2 b2)
{
    df2 r;
    r.h = __fadd2_rn(a1, b1);
    const float2 bb = sub2(r.h, a1);
    const float2 e = __fadd2_rn(sub2(a1, sub2(r.h, bb)), sub2(b1, bb));
    r.l = __fadd2_rn(e, __fadd2_rn(a2, b2));
    return r;
}
#endif

template <typename T>
struct is_dfloat { static constexpr bool value = false; };
template <>
struct is_dfloat<dfloat> { static constexpr bool value = true; };

}  // namespace feod
