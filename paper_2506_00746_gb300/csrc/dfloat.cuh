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

template <typename T>
struct is_dfloat { static constexpr bool value = false; };
template <>
struct is_dfloat<dfloat> { static constexpr bool value = true; };

}  // namespace feod
