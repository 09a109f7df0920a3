// gf_df64.cuh -- FP64-class arithmetic on the FP32 pipe ("double-float").
//
// On this GPU the FP64 unit is small (a few FP64 operations per clock per SM)
// while FP32 runs at 128 lanes per clock per SM.  A value is held as an
// unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2, a 48-bit
// significand); sums and products use the error-free transformations of
// Knuth (two-sum), Dekker (fast two-sum) and the FMA-based exact product, so
// every operation has relative error ~2^-47 (about 7e-15).
//
// Storage format DF64_18 keeps each complex link entry as one 16-byte chunk
// (re.hi, re.lo, im.hi, im.lo): the same planes and byte count as FP64-18.
#pragma once

#include "gf_device.cuh"

namespace gf {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo)
{
    df r;
    r.hi = hi;
    r.lo = lo;
    return r;
}

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df df_add(df x, df y)
{
    float s, e;
    two_sum(x.hi, y.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
    df r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df df_neg(df x) { return df_make(-x.hi, -x.lo); }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// x * y: exact product of the high parts (FMA) plus the cross terms
__device__ __forceinline__ df df_mul(df x, df y)
{
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    df r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df df_from_double(double v)
{
    float hi = __double2float_rn(v);
    return df_make(hi, __double2float_rn(v - (double)hi));
}

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

struct cdf {
    df re, im;
};

struct mat3df {
    cdf e[3][3];
};

// acc + x y (complex)
__device__ __forceinline__ cdf cdf_mac(cdf acc, cdf x, cdf y)
{
    cdf r;
    r.re = df_add(acc.re, df_sub(df_mul(x.re, y.re), df_mul(x.im, y.im)));
    r.im = df_add(acc.im, df_add(df_mul(x.re, y.im), df_mul(x.im, y.re)));
    return r;
}

// acc + x conj(y)
__device__ __forceinline__ cdf cdf_mac_conj(cdf acc, cdf x, cdf y)
{
    cdf r;
    r.re = df_add(acc.re, df_add(df_mul(x.re, y.re), df_mul(x.im, y.im)));
    r.im = df_add(acc.im, df_sub(df_mul(x.im, y.re), df_mul(x.re, y.im)));
    return r;
}

// Dot products of three complex double-float numbers with one final
// renormalisation: each real product x y contributes its rounded high part p =
// x.hi y.hi to a running sum (two-sum, error kept) and its exact remainder
// fma(x.hi, y.hi, -p) + x.hi y.lo + x.lo y.hi to a float error accumulator;
// the x.lo y.lo term (relative 2^-48) is dropped.  About 12 FP32 operations
// per real product against 18 for a double-float multiply and add.
struct dacc {
    float s, e;
};

__device__ __forceinline__ void dacc_add_prod(dacc &a, df x, df y)
{
    float p = __fmul_rn(x.hi, y.hi);
    float r = __fmaf_rn(x.hi, y.hi, -p);
    r = __fmaf_rn(x.hi, y.lo, r);
    r = __fmaf_rn(x.lo, y.hi, r);
    float s, t;
    two_sum(a.s, p, s, t);
    a.s = s;
    a.e = __fadd_rn(a.e, __fadd_rn(t, r));
}

// (two-sum, not fast-two-sum: after cancellation the error sum may exceed s)
__device__ __forceinline__ df dacc_result(dacc a)
{
    df r;
    two_sum(a.s, a.e, r.hi, r.lo);
    return r;
}

// sum_l x[l] y[l] (CONJ: sum_l x[l] conj(y[l]))
template <bool CONJ>
__device__ __forceinline__ cdf cdf_dot3(const cdf x[3], const cdf y[3])
{
    dacc re = { 0.f, 0.f }, im = { 0.f, 0.f };
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const df yi = CONJ ? df_make(-y[l].im.hi, -y[l].im.lo) : y[l].im;
        dacc_add_prod(re, x[l].re, y[l].re);
        dacc_add_prod(re, df_make(-x[l].im.hi, -x[l].im.lo), yi);
        dacc_add_prod(im, x[l].re, yi);
        dacc_add_prod(im, x[l].im, y[l].re);
    }
    cdf z;
    z.re = dacc_result(re);
    z.im = dacc_result(im);
    return z;
}

__device__ __forceinline__ cdf cdf_zero()
{
    cdf z;
    z.re = df_make(0.f, 0.f);
    z.im = df_make(0.f, 0.f);
    return z;
}

// ---------------------------------------------------------------------------
// DF64_18 storage: 9 chunks per link, chunk = (re.hi, re.lo, im.hi, im.lo)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_df(const FieldRef &f, int pl0, int h, mat3df &u)
{
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const float4 *pl = reinterpret_cast<const float4 *>(f.base + (pl0 + c) * f.plane_bytes);
        float4 v = pl[h];
        u.e[c / 3][c % 3].re = df_make(v.x, v.y);
        u.e[c / 3][c % 3].im = df_make(v.z, v.w);
    }
}

// second read of a link (volatile: not merged with the first read)
__device__ __forceinline__ void reload_df(const FieldRef &f, int pl0, int h, mat3df &u)
{
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const float4 *p = reinterpret_cast<const float4 *>(f.base + (pl0 + c) * f.plane_bytes) + h;
        float4 v;
        asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
        u.e[c / 3][c % 3].re = df_make(v.x, v.y);
        u.e[c / 3][c % 3].im = df_make(v.z, v.w);
    }
}

// one complex entry (chunk) of a link
__device__ __forceinline__ cdf reload_chunk_df(const FieldRef &f, int plane, int h)
{
    const float4 *p = reinterpret_cast<const float4 *>(f.base + plane * f.plane_bytes) + h;
    float4 v;
    asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    cdf z;
    z.re = df_make(v.x, v.y);
    z.im = df_make(v.z, v.w);
    return z;
}

__device__ __forceinline__ void store_chunk_df(const FieldRef &f, int plane, int h, const cdf &z)
{
    float4 *p = reinterpret_cast<float4 *>(f.base + plane * f.plane_bytes) + h;
    *p = make_float4(z.re.hi, z.re.lo, z.im.hi, z.im.lo);
}

__device__ __forceinline__ void store_df(const FieldRef &f, int pl0, int h, const mat3df &u)
{
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        float4 *pl = reinterpret_cast<float4 *>(f.base + (pl0 + c) * f.plane_bytes);
        const cdf &z = u.e[c / 3][c % 3];
        pl[h] = make_float4(z.re.hi, z.re.lo, z.im.hi, z.im.lo);
    }
}

}  // namespace gf
