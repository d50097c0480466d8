// Float-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2
// (|lo| < ulp(hi) for a double split from its bits, ff_split_bits), about 48
// significant bits.  The building blocks are the error-free transformations
// TwoSum (Knuth, TAOCP vol. 2, 4.2.2), Fast2Sum (Dekker 1971) and TwoProduct
// with a fused multiply-add (the product's rounding error is
// fma(a, b, -a*b)); addition, multiplication and the reciprocal square root
// with one Newton correction follow Dekker, "A floating-point technique for
// extending the available precision", Numer. Math. 18 (1971).  GB300 runs
// FP32 about 74 times faster than FP64, so a float-float operation of 10-20
// FP32 instructions costs less than one FP64 operation.  The _rn intrinsics
// keep the compiler from contracting or reordering the error terms.
#pragma once

#include <cuda_runtime.h>

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float a)
{
    ff r;
    r.hi = a;
    r.lo = 0.0f;
    return r;
}

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    ff r;
    r.hi = s;
    r.lo = e;
    return r;
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ ff fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    ff r;
    r.hi = s;
    r.lo = e;
    return r;
}

// p + e = a * b exactly (error of the product from a fused multiply-add)
__device__ __forceinline__ ff two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    ff r;
    r.hi = p;
    r.lo = e;
    return r;
}

__device__ __forceinline__ ff ff_add(ff x, ff y)
{
    const ff s = two_sum(x.hi, y.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_neg(ff x)
{
    ff r;
    r.hi = -x.hi;
    r.lo = -x.lo;
    return r;
}

__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

__device__ __forceinline__ ff ff_mul(ff x, ff y)
{
    const ff p = two_prod(x.hi, y.hi);
    const float e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ ff ff_mulf(ff x, float y)
{
    const ff p = two_prod(x.hi, y);
    const float e = __fmaf_rn(x.lo, y, p.lo);
    return fast_two_sum(p.hi, e);
}

// 1 / sqrt(x) of a positive value: r = rsqrt(hi), one Newton correction
// r + r (1 - x r^2) / 2.  The residual 1 - x r^2, of order 1e-7, by fused
// multiply-adds: hi r = u + v exactly (v from an FMA), 1 - u r by one FMA
// (one rounding of a number of order 1e-7), then - v r - lo r^2; about 11
// instructions against 29 with the residual formed by float-float products
__device__ __forceinline__ ff ff_rsqrt(ff x)
{
    const float r = rsqrtf(x.hi);
    const float u = __fmul_rn(x.hi, r);
    const float v = __fmaf_rn(x.hi, r, -u);
    float e = __fmaf_rn(-u, r, 1.0f);
    e = __fmaf_rn(-v, r, e);
    e = __fmaf_rn(-__fmul_rn(x.lo, r), r, e);
    return fast_two_sum(r, __fmul_rn(__fmul_rn(0.5f, r), e));
}

// a . b of two float-float vectors
__device__ __forceinline__ ff ff_dot3(const ff a[3], const ff b[3])
{
    return ff_add(ff_add(ff_mul(a[0], b[0]), ff_mul(a[1], b[1])), ff_mul(a[2], b[2]));
}

// a . b of two float-float vectors, compensated (the Dot2 scheme of Ogita,
// Rump & Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26
// (2005), with the low parts folded into the error term): exact products of
// the high parts by TwoProduct, their rounding errors, the products with the
// low parts and the TwoSum errors of the running sum accumulated in FP32, one
// renormalisation at the end.  As accurate as ff_dot3 (the result as if
// computed in twice the precision) for about two thirds of its operations.
__device__ __forceinline__ ff ff_dot3_c(const ff a[3], const ff b[3])
{
    ff p = two_prod(a[0].hi, b[0].hi);
    float s = p.hi;
    float e = __fmaf_rn(a[0].hi, b[0].lo, __fmaf_rn(a[0].lo, b[0].hi, p.lo));
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        p = two_prod(a[k].hi, b[k].hi);
        const ff t = two_sum(s, p.hi);
        s = t.hi;
        e = __fadd_rn(e, __fadd_rn(t.lo, __fmaf_rn(a[k].hi, b[k].lo, __fmaf_rn(a[k].lo, b[k].hi, p.lo))));
    }
    return fast_two_sum(s, e);
}

// a_b c_c - a_c c_b for a float a and a float-float c, compensated: one
// component of the cross product a x c
__device__ __forceinline__ ff ff_cross_comp_f(float ab, ff cc, float ac, ff cb)
{
    const ff p = two_prod(ab, cc.hi), q = two_prod(ac, cb.hi);
    const ff t = two_sum(p.hi, -q.hi);
    const float e = __fadd_rn(t.lo, __fmaf_rn(ab, cc.lo, __fmaf_rn(-ac, cb.lo, __fsub_rn(p.lo, q.lo))));
    return fast_two_sum(t.hi, e);
}

// a . b for a float-float vector a and a float vector b
__device__ __forceinline__ ff ff_dot3f(const ff a[3], const float b[3])
{
    return ff_add(ff_add(ff_mulf(a[0], b[0]), ff_mulf(a[1], b[1])), ff_mulf(a[2], b[2]));
}

// a . b for a float-float vector a and a float vector b, compensated as
// ff_dot3_c: the products of the high parts exact (TwoProduct), their
// errors, the products with the low parts and the TwoSum errors of the
// running sum accumulated in FP32, one renormalisation (about 28
// instructions against 40 for ff_dot3f; the error stays at the level of
// eps^2 times the sum of the products' magnitudes)
__device__ __forceinline__ ff ff_dot3f_c(const ff a[3], const float b[3])
{
    ff p = two_prod(a[0].hi, b[0]);
    float s = p.hi;
    float e = __fmaf_rn(a[0].lo, b[0], p.lo);
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        p = two_prod(a[k].hi, b[k]);
        const ff t = two_sum(s, p.hi);
        s = t.hi;
        e = __fadd_rn(e, __fadd_rn(t.lo, __fmaf_rn(a[k].lo, b[k], p.lo)));
    }
    return fast_two_sum(s, e);
}

// a . b of two float vectors, the products exact
__device__ __forceinline__ ff ff_dot3_exact(const float a[3], const float b[3])
{
    return ff_add(ff_add(two_prod(a[0], b[0]), two_prod(a[1], b[1])), two_prod(a[2], b[2]));
}
__device__ __forceinline__ double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }

// symmetry axis (body z) of the rotation by q/|q| in float-float (quaternion
// components exact): 2/|q|^2 (xz + wy, yz - wx, ...) and 1 - 2/|q|^2 (x^2 + y^2)
__device__ __forceinline__ void ff_axis(float w, float x, float y, float z, ff o[3])
{
    const ff q2 = ff_add(ff_add(two_prod(w, w), two_prod(x, x)), ff_add(two_prod(y, y), two_prod(z, z)));
    // s = 2 / |q|^2: float reciprocal plus one correction with the exact residual
    const float r0 = __fdiv_rn(2.0f, q2.hi);
    const ff res = ff_sub(ff_make(2.0f), ff_mulf(q2, r0));
    const ff s = fast_two_sum(r0, __fmul_rn(res.hi, __fmul_rn(r0, 0.5f)));
    o[0] = ff_mul(s, ff_add(two_prod(x, z), two_prod(w, y)));
    o[1] = ff_mul(s, ff_sub(two_prod(y, z), two_prod(w, x)));
    o[2] = ff_sub(ff_make(1.0f), ff_mul(s, ff_add(two_prod(x, x), two_prod(y, y))));
}

// Float-float split of a double with integer and FP32 operations only (no
// FP64-pipe conversion): hi = d truncated to 24 significant bits, lo = the
// next 23 bits, |hi + lo - d| < 2^-46 |d|.  Doubles with |d| < 2^-126
// (zero included) give 0 + 0; |d| >= 2^128 gives +-infinity.
__device__ __forceinline__ ff ff_split_bits(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
    const unsigned int sign = hw & 0x80000000u;
    const int ef = (int)((hw >> 20) & 0x7FFu) - 1023 + 127;  // the float exponent of hi
    ff r;
    if (ef <= 0) {
        r.hi = 0.0f;
        r.lo = 0.0f;
        return r;
    }
    if (ef >= 255) {
        r.hi = __int_as_float(sign | 0x7F800000u);
        r.lo = 0.0f;
        return r;
    }
    // the fraction's top 23 bits (20 of the high word, 3 of the low word)
    r.hi = __int_as_float(sign | ((unsigned int)ef << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
    // the next 23 bits as an exact float (2^23 + m - 2^23), times 2^(e - 46)
    const unsigned int m = (lw & 0x1FFFFFFFu) >> 6;
    const int el = ef - 46;
    float lo = 0.0f;
    if (el > 0) lo = __fmul_rn(__fsub_rn(__int_as_float(0x4B000000u | m), 8388608.0f), __int_as_float((unsigned int)el << 23));
    r.lo = sign ? -lo : lo;
    return r;
}

// ff_split_bits with NaN kept as NaN (ff_split_bits gives infinity for it):
// positions split without the FP64 pipe, a NaN still failing every test
__device__ __forceinline__ ff ff_split_bits_nan(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d) & 0x7FFFFFFFFFFFFFFFull;
    if (b > 0x7FF0000000000000ull) {
        ff r;
        r.hi = __int_as_float(0x7FC00000);
        r.lo = 0.0f;
        return r;
    }
    return ff_split_bits(d);
}
