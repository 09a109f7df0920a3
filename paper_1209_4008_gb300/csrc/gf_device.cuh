// gf_device.cuh -- device-side building blocks of the gauge-fixing kernels:
// lattice geometry of the checkerboard layout, the four link storage formats,
// SU(2)-subgroup algebra in quaternion form, Philox4x32-10 and the SU(2)
// heatbath draw.  Written for sm_103a; CUDA cores only (SU(3) algebra is not
// a dense contraction).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gf {

// ---------------------------------------------------------------------------
// complex numbers and 3x3 matrices held in registers
// ---------------------------------------------------------------------------
template <class T>
struct cpx {
    T re, im;
};

template <class T>
struct mat3 {
    cpx<T> e[3][3];
};

template <class T>
__device__ __forceinline__ cpx<T> mk(T re, T im)
{
    cpx<T> z;
    z.re = re;
    z.im = im;
    return z;
}

// conj(a*d - b*c): one entry of the third row of an SU(3) matrix from rows 0, 1
template <class T>
__device__ __forceinline__ cpx<T> conj_cross(cpx<T> a, cpx<T> d, cpx<T> b, cpx<T> c)
{
    // one multiply and three FMAs per component
    T re = a.re * d.re;
    re = fma(-a.im, d.im, re);
    re = fma(-b.re, c.re, re);
    re = fma(b.im, c.im, re);
    T im = a.re * d.im;
    im = fma(a.im, d.re, im);
    im = fma(-b.re, c.im, im);
    im = fma(-b.im, c.re, im);
    return mk<T>(re, -im);
}

// row 2 = conj(row0 x row1): unitarity and det = 1 fix the third row (Sec. 4.1)
template <class T>
__device__ __forceinline__ void rebuild_row2(mat3<T> &u)
{
    u.e[2][0] = conj_cross(u.e[0][1], u.e[1][2], u.e[0][2], u.e[1][1]);
    u.e[2][1] = conj_cross(u.e[0][2], u.e[1][0], u.e[0][0], u.e[1][2]);
    u.e[2][2] = conj_cross(u.e[0][0], u.e[1][1], u.e[0][1], u.e[1][0]);
}

template <class T>
__device__ __forceinline__ mat3<T> dagger(const mat3<T> &u)
{
    mat3<T> d;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) d.e[a][b] = mk<T>(u.e[b][a].re, -u.e[b][a].im);
    return d;
}

template <class T>
__device__ __forceinline__ mat3<T> identity3()
{
    mat3<T> u;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) u.e[a][b] = mk<T>(a == b ? T(1) : T(0), T(0));
    return u;
}

// ---------------------------------------------------------------------------
// lattice geometry: per-parity half-site index (Sec. 4.1, RED/BLACK blocks)
// ---------------------------------------------------------------------------
// A site with lexicographic index i = x + Lx (y + Ly (z + Lz t)) has parity
// p = (x+y+z+t) & 1 and half index h = i >> 1 (Lx even makes this a bijection
// onto [0, V/2) for each parity).
struct Geom {
    int L[4];   // Lx, Ly, Lz, Lt
    int Lh0;    // Lx / 2
    int Vh;     // V / 2
    int plane;  // elements per storage plane (Vh rounded up to 64)
};

__device__ __forceinline__ void site_coords(const Geom &g, int p, int h, int c[4])
{
    int r = h / g.Lh0;
    int xh = h - r * g.Lh0;
    int r2 = r / g.L[1];
    c[1] = r - r2 * g.L[1];
    c[3] = r2 / g.L[2];
    c[2] = r2 - c[3] * g.L[2];
    c[0] = 2 * xh + ((p + c[1] + c[2] + c[3]) & 1);
}

__device__ __forceinline__ int lex_index(const Geom &g, const int c[4])
{
    return c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}

// lexicographic stride of direction mu (selects, no local-memory indexing)
__device__ __forceinline__ int lex_stride(const Geom &g, int mu)
{
    int s1 = g.L[0], s2 = s1 * g.L[1], s3 = s2 * g.L[2];
    return mu == 0 ? 1 : (mu == 1 ? s1 : (mu == 2 ? s2 : s3));
}

__device__ __forceinline__ int coord_of(const int c[4], int mu)
{
    return mu == 0 ? c[0] : (mu == 1 ? c[1] : (mu == 2 ? c[2] : c[3]));
}

__device__ __forceinline__ int extent_of(const Geom &g, int mu)
{
    return mu == 0 ? g.L[0] : (mu == 1 ? g.L[1] : (mu == 2 ? g.L[2] : g.L[3]));
}

// half index of x - mu (periodic)
__device__ __forceinline__ int back_half(const Geom &g, const int c[4], int mu)
{
    int i = lex_index(g, c);
    int st = lex_stride(g, mu);
    int d = coord_of(c, mu) == 0 ? (extent_of(g, mu) - 1) * st : -st;
    return (i + d) >> 1;
}

// half index of x + mu (periodic)
__device__ __forceinline__ int fwd_half(const Geom &g, const int c[4], int mu)
{
    int i = lex_index(g, c);
    int st = lex_stride(g, mu);
    int d = coord_of(c, mu) + 1 == extent_of(g, mu) ? -(extent_of(g, mu) - 1) * st : st;
    return (i + d) >> 1;
}

// ---------------------------------------------------------------------------
// link storage formats (per-parity SoA, site index fastest; Sec. 4.1)
// ---------------------------------------------------------------------------
// A field is a sequence of planes, plane (p, mu, c) holding chunk c of link
// U_mu of every site of parity p: plane index (p*4 + mu)*NCHUNK + c, each
// plane g.plane * 16 bytes.  Chunks are 16-byte vectors so that a warp reads
// 512 contiguous bytes per load instruction:
//   F64_18: 9 double2 (one complex each, row-major)
//   F64_12: 6 double2 (rows 0, 1; row 2 rebuilt)
//   F32_18: 4 float4 (two complex each, row-major) + 1 float2 (entry 2,2)
//   F32_12: 3 float4 (rows 0, 1; row 2 rebuilt)
//   DF64_18: 9 float4 (re.hi, re.lo, im.hi, im.lo): FP64-class values as pairs of
//            FP32 (hi + lo), for the FP32-pipe kernels of gf_df64.cuh
enum Format { F64_18 = 0, F64_12 = 1, F32_18 = 2, F32_12 = 3, DF64_18 = 4 };

struct FieldRef {
    char *base;
    size_t plane_bytes;
};

template <int FMT>
struct Store;

template <>
struct Store<F64_18> {
    typedef double T;
    static constexpr int NCHUNK = 9;
    static constexpr int REALS = 18;
    static __device__ __forceinline__ void load(const FieldRef &f, int pl0, int h, mat3<double> &u)
    {
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const double2 *pl = reinterpret_cast<const double2 *>(f.base + (pl0 + c) * f.plane_bytes);
            double2 v = pl[h];
            u.e[c / 3][c % 3] = mk<double>(v.x, v.y);
        }
    }
    static __device__ __forceinline__ void store(const FieldRef &f, int pl0, int h, const mat3<double> &u)
    {
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            double2 *pl = reinterpret_cast<double2 *>(f.base + (pl0 + c) * f.plane_bytes);
            pl[h] = make_double2(u.e[c / 3][c % 3].re, u.e[c / 3][c % 3].im);
        }
    }
};

template <>
struct Store<F64_12> {
    typedef double T;
    static constexpr int NCHUNK = 6;
    static constexpr int REALS = 12;
    static __device__ __forceinline__ void load(const FieldRef &f, int pl0, int h, mat3<double> &u)
    {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const double2 *pl = reinterpret_cast<const double2 *>(f.base + (pl0 + c) * f.plane_bytes);
            double2 v = pl[h];
            u.e[c / 3][c % 3] = mk<double>(v.x, v.y);
        }
        rebuild_row2(u);
    }
    static __device__ __forceinline__ void store(const FieldRef &f, int pl0, int h, const mat3<double> &u)
    {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            double2 *pl = reinterpret_cast<double2 *>(f.base + (pl0 + c) * f.plane_bytes);
            pl[h] = make_double2(u.e[c / 3][c % 3].re, u.e[c / 3][c % 3].im);
        }
    }
};

template <>
struct Store<F32_18> {
    typedef float T;
    static constexpr int NCHUNK = 5;
    static constexpr int REALS = 18;
    static __device__ __forceinline__ void load(const FieldRef &f, int pl0, int h, mat3<float> &u)
    {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float4 *pl = reinterpret_cast<const float4 *>(f.base + (pl0 + c) * f.plane_bytes);
            float4 v = pl[h];
            int e0 = 2 * c, e1 = 2 * c + 1;
            u.e[e0 / 3][e0 % 3] = mk<float>(v.x, v.y);
            u.e[e1 / 3][e1 % 3] = mk<float>(v.z, v.w);
        }
        const float2 *pl = reinterpret_cast<const float2 *>(f.base + (pl0 + 4) * f.plane_bytes);
        float2 v = pl[h];
        u.e[2][2] = mk<float>(v.x, v.y);
    }
    static __device__ __forceinline__ void store(const FieldRef &f, int pl0, int h, const mat3<float> &u)
    {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float4 *pl = reinterpret_cast<float4 *>(f.base + (pl0 + c) * f.plane_bytes);
            int e0 = 2 * c, e1 = 2 * c + 1;
            pl[h] = make_float4(u.e[e0 / 3][e0 % 3].re, u.e[e0 / 3][e0 % 3].im, u.e[e1 / 3][e1 % 3].re,
                                u.e[e1 / 3][e1 % 3].im);
        }
        float2 *pl = reinterpret_cast<float2 *>(f.base + (pl0 + 4) * f.plane_bytes);
        pl[h] = make_float2(u.e[2][2].re, u.e[2][2].im);
    }
};

template <>
struct Store<F32_12> {
    typedef float T;
    static constexpr int NCHUNK = 3;
    static constexpr int REALS = 12;
    static __device__ __forceinline__ void load(const FieldRef &f, int pl0, int h, mat3<float> &u)
    {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 *pl = reinterpret_cast<const float4 *>(f.base + (pl0 + c) * f.plane_bytes);
            float4 v = pl[h];
            int e0 = 2 * c, e1 = 2 * c + 1;
            u.e[e0 / 3][e0 % 3] = mk<float>(v.x, v.y);
            u.e[e1 / 3][e1 % 3] = mk<float>(v.z, v.w);
        }
        rebuild_row2(u);
    }
    static __device__ __forceinline__ void store(const FieldRef &f, int pl0, int h, const mat3<float> &u)
    {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float4 *pl = reinterpret_cast<float4 *>(f.base + (pl0 + c) * f.plane_bytes);
            int e0 = 2 * c, e1 = 2 * c + 1;
            pl[h] = make_float4(u.e[e0 / 3][e0 % 3].re, u.e[e0 / 3][e0 % 3].im, u.e[e1 / 3][e1 % 3].re,
                                u.e[e1 / 3][e1 % 3].im);
        }
    }
};

// FP64 view of DF64_18 (value = hi + lo), used by the whole-field kernels
template <>
struct Store<DF64_18> {
    typedef double T;
    static constexpr int NCHUNK = 9;
    static constexpr int REALS = 18;
    static __device__ __forceinline__ void load(const FieldRef &f, int pl0, int h, mat3<double> &u)
    {
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const float4 *pl = reinterpret_cast<const float4 *>(f.base + (pl0 + c) * f.plane_bytes);
            float4 v = pl[h];
            u.e[c / 3][c % 3] = mk<double>((double)v.x + (double)v.y, (double)v.z + (double)v.w);
        }
    }
    static __device__ __forceinline__ void store(const FieldRef &f, int pl0, int h, const mat3<double> &u)
    {
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            float4 *pl = reinterpret_cast<float4 *>(f.base + (pl0 + c) * f.plane_bytes);
            double re = u.e[c / 3][c % 3].re, im = u.e[c / 3][c % 3].im;
            float rh = __double2float_rn(re), ih = __double2float_rn(im);
            pl[h] = make_float4(rh, __double2float_rn(re - (double)rh), ih, __double2float_rn(im - (double)ih));
        }
    }
};

// ---------------------------------------------------------------------------
// SU(2) subgroups in quaternion form (Sec. 2, Cabibbo-Marinari)
// ---------------------------------------------------------------------------
// r = (r0, r1, r2, r3) is R = r0 1 + i r.sigma = [[r0 + i r3, r2 + i r1],
// [-r2 + i r1, r0 - i r3]].  For a complex 2x2 block w, Re tr[R w] = r . k
// with k = (Re(w00 + w11), -Im(w01 + w10), Re(w10 - w01), Im(w11 - w00)), so
// the SU(2) maximiser of eq. (localsolution) is k/|k|.
__device__ __forceinline__ void subgroup_rows(int sg, int &a, int &b)
{
    a = (sg == 1) ? 1 : 0;
    b = (sg == 0) ? 1 : 2;
}

template <class T>
__device__ __forceinline__ void add_block_quaternion(const mat3<T> &x, int a, int b, T k[4])
{
    k[0] += x.e[a][a].re + x.e[b][b].re;
    k[1] -= x.e[a][b].im + x.e[b][a].im;
    k[2] += x.e[b][a].re - x.e[a][b].re;
    k[3] += x.e[b][b].im - x.e[a][a].im;
}

// rows a, b of x <- R (rows a, b)
template <class T>
__device__ __forceinline__ void rotate_rows(mat3<T> &x, int a, int b, const T r[4])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cpx<T> xa = x.e[a][c], xb = x.e[b][c];
        x.e[a][c].re = r[0] * xa.re - r[3] * xa.im + r[2] * xb.re - r[1] * xb.im;
        x.e[a][c].im = r[0] * xa.im + r[3] * xa.re + r[2] * xb.im + r[1] * xb.re;
        x.e[b][c].re = r[0] * xb.re + r[3] * xb.im - r[2] * xa.re - r[1] * xa.im;
        x.e[b][c].im = r[0] * xb.im - r[3] * xb.re - r[2] * xa.im + r[1] * xa.re;
    }
}

// Overrelaxation exponent and SU(2) projection (Alg. 1, 19 flop form):
// b = (omega a0^2 + |a|^2) / (a0^2 + |a|^2), r = (a0, b a) / sqrt(a0^2 + b^2 |a|^2).
// Returns false when k = 0 (the subgroup is then left unchanged).
__device__ __forceinline__ bool overrelax_quat(const float k[4], float omega, float r[4])
{
    float a0sq = k[0] * k[0];
    float aisq = k[1] * k[1] + k[2] * k[2] + k[3] * k[3];
    float n = a0sq + aisq;
    if (n == 0.0f) return false;
    float b = __fdiv_rn(omega * a0sq + aisq, n);
    float c = rsqrtf(a0sq + b * b * aisq);
    float bc = b * c;
    r[0] = c * k[0];
    r[1] = bc * k[1];
    r[2] = bc * k[2];
    r[3] = bc * k[3];
    return true;
}

// FP64: the same rational map written without a division (one reciprocal
// square root), since FP64 divides are costly on this part:
// r = (n a0, B a) / sqrt(n^2 a0^2 + B^2 |a|^2), n = a0^2 + |a|^2, B = omega a0^2 + |a|^2.
__device__ __forceinline__ bool overrelax_quat(const double k[4], double omega, double r[4])
{
    double a0sq = k[0] * k[0];
    double aisq = k[1] * k[1] + k[2] * k[2] + k[3] * k[3];
    double n = a0sq + aisq;
    if (n == 0.0) return false;
    double B = omega * a0sq + aisq;
    double na = n * k[0];
    double c = rsqrt(na * na + B * B * aisq);
    double bc = B * c;
    r[0] = na * c;
    r[1] = bc * k[1];
    r[2] = bc * k[2];
    r[3] = bc * k[3];
    return true;
}

// Other readings of g -> g^omega (Sec. 2 leaves the form open), selected by
// the context option "or_variant": 1 = first order, r = normalise((1 - omega)
// 1 + omega k/|k|); 2 = the exact power, r = (cos(omega phi), sin(omega phi) n)
// for k/|k| = (cos phi, sin phi n), left unchanged when n is undefined.
template <class T>
struct quat_ok {
    T r0, r1, r2, r3;
    int ok;
};

// (out of line, arguments and result by value: the default reading pays no
// registers or local memory for these paths)
template <class T>
__device__ __noinline__ quat_ok<T> overrelax_first_order(T k0, T k1, T k2, T k3, T omega)
{
    quat_ok<T> q = { T(0), T(0), T(0), T(0), 0 };
    T n = sqrt(k0 * k0 + k1 * k1 + k2 * k2 + k3 * k3);
    if (n == T(0)) return q;
    T v0 = (T(1) - omega) + omega * (k0 / n), v1 = omega * (k1 / n), v2 = omega * (k2 / n), v3 = omega * (k3 / n);
    T m = sqrt(v0 * v0 + v1 * v1 + v2 * v2 + v3 * v3);
    if (m == T(0)) return q;
    q.r0 = v0 / m;
    q.r1 = v1 / m;
    q.r2 = v2 / m;
    q.r3 = v3 / m;
    q.ok = 1;
    return q;
}

template <class T>
__device__ __noinline__ quat_ok<T> overrelax_exact_power(T k0, T k1, T k2, T k3, T omega)
{
    quat_ok<T> q = { T(0), T(0), T(0), T(0), 0 };
    T a = sqrt(k1 * k1 + k2 * k2 + k3 * k3);
    if (a == T(0)) {
        if (!(k0 > T(0))) return q;
        q.r0 = T(1);
        q.ok = 1;
        return q;
    }
    T phi = atan2(a, k0);
    T c = cos(omega * phi), sn = sin(omega * phi);
    q.r0 = c;
    q.r1 = sn * (k1 / a);
    q.r2 = sn * (k2 / a);
    q.r3 = sn * (k3 / a);
    q.ok = 1;
    return q;
}

template <class T>
__device__ __forceinline__ bool overrelax_step(const T k[4], T omega, int variant, T r[4])
{
    if (variant == 0) return overrelax_quat(k, omega, r);
    quat_ok<T> q = variant == 1 ? overrelax_first_order(k[0], k[1], k[2], k[3], omega)
                                : overrelax_exact_power(k[0], k[1], k[2], k[3], omega);
    r[0] = q.r0;
    r[1] = q.r1;
    r[2] = q.r2;
    r[3] = q.r3;
    return q.ok != 0;
}

// ---------------------------------------------------------------------------
// Maximally Abelian gauge (Sec. 6): F = sum |U_ii|^2.  For subgroup (a,b) and
// a held matrix X (forward link U, or U^dagger of a backward link), the
// diagonal weight after X <- R X, R = [[alpha, beta], [-beta*, alpha*]], is
// |alpha X_aa + beta X_ba|^2 + |alpha conj(X_bb) - beta conj(X_ab)|^2 =
// z^dagger H z with z = (alpha, beta) and H the 2x2 Hermitian matrix summed
// below.  Its maximiser over |z| = 1 is the top eigenvector of H, unique up to
// the phase of the residual U(1); the phase is fixed by alpha >= 0 (the
// maximiser closest to the identity).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void add_mag_terms(const mat3<T> &x, int a, int b, T h[4])
{
    const cpx<T> xaa = x.e[a][a], xab = x.e[a][b], xba = x.e[b][a], xbb = x.e[b][b];
    // (accumulated as FMA chains)
    h[0] = fma(xaa.re, xaa.re, fma(xaa.im, xaa.im, fma(xbb.re, xbb.re, fma(xbb.im, xbb.im, h[0]))));  // h11
    h[1] = fma(xba.re, xba.re, fma(xba.im, xba.im, fma(xab.re, xab.re, fma(xab.im, xab.im, h[1]))));  // h22
    // h12 += conj(xaa) xba - xbb conj(xab)
    h[2] = fma(xaa.re, xba.re, fma(xaa.im, xba.im, fma(-xbb.re, xab.re, fma(-xbb.im, xab.im, h[2]))));
    h[3] = fma(xaa.re, xba.im, fma(-xaa.im, xba.re, fma(-xbb.im, xab.re, fma(xbb.re, xab.im, h[3]))));
}

// quaternion r of the maximiser (r0 = |alpha|, r3 = 0, r2 + i r1 = beta);
// false (no change) when H is a multiple of the identity
template <class T>
__device__ __forceinline__ bool mag_element(const T h[4], T r[4])
{
    const T d = T(0.5) * (h[0] - h[1]);
    const T n12 = h[2] * h[2] + h[3] * h[3];
    if (n12 == T(0) && d >= T(0)) {  // already optimal (or degenerate): identity
        return false;
    }
    const T rt = sqrt(d * d + n12);
    // top eigenvector: (lambda - h22, conj(h12)) when h11 >= h22, else (h12, lambda - h11)
    T v1re, v1im, v2re, v2im;
    if (d >= T(0)) {
        v1re = d + rt;
        v1im = T(0);
        v2re = h[2];
        v2im = -h[3];
    } else {
        v1re = h[2];
        v1im = h[3];
        v2re = rt - d;
        v2im = T(0);
    }
    const T n1 = sqrt(v1re * v1re + v1im * v1im);
    const T nv = sqrt(v1re * v1re + v1im * v1im + v2re * v2re + v2im * v2im);
    if (n1 > T(0)) {  // alpha = |v1|, beta = v2 conj(v1) / |v1|
        r[0] = n1 / nv;
        r[3] = T(0);
        r[2] = (v2re * v1re + v2im * v1im) / (n1 * nv);
        r[1] = (v2im * v1re - v2re * v1im) / (n1 * nv);
    } else {  // no maximiser near the identity: alpha = 0, beta = |v2|
        r[0] = T(0);
        r[3] = T(0);
        r[2] = T(1);
        r[1] = T(0);
    }
    return true;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// (w + 1/2) / 2^32, exact in double
__device__ __forceinline__ double u01(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

#define GF_TWO_PI 6.283185307179586476925286766559
#define GF_SA_TAG 1u
#define GF_SA_DIRECTION 255u
#define GF_SA_ALPHA_SWITCH 2.0

// SU(2) heatbath for weight exp(r.k / T) dHaar(r): s0 from
// sqrt(1 - s0^2) exp(alpha s0), alpha = |k|/T (Creutz 1980 below alpha = 2,
// Kennedy-Pendleton 1985 above), direction of the imaginary part uniform on
// the sphere, then r = s k/|k| (quaternion product).  FP64 throughout so that
// accept/reject decisions follow the FP64 definition.  st = 1 on success,
// 0 when cap attempts were rejected, 2 when k = 0 (nothing to do; r unset).
// Not inlined: a site update draws for three subgroups, and three inlined
// copies of this FP64 code (log, exp, cos, sincos, sqrt) overflow the
// instruction cache of the larger site-update kernels.
struct HeatbathDraw {
    double r0, r1, r2, r3;
    int st;
};

static __device__ __noinline__ HeatbathDraw heatbath_draw(double k0, double k1, double k2, double k3, double T,
                                                   uint32_t site, uint32_t sweep, int sg, int cap, uint2 key,
                                                   uint32_t tag)
{
    HeatbathDraw d;
    d.r0 = d.r1 = d.r2 = d.r3 = 0.0;
    d.st = 2;
    double kn = sqrt(k0 * k0 + k1 * k1 + k2 * k2 + k3 * k3);
    if (kn == 0.0) return d;
    double alpha = kn / T;
    double s0 = 0.0;
    bool ok = false;
    for (int a = 0; a < cap && a < (int)GF_SA_DIRECTION; ++a) {
        uint4 w = philox4x32_10(make_uint4(site, sweep, (uint32_t)sg * 256u + (uint32_t)a, tag), key);
        if (alpha < GF_SA_ALPHA_SWITCH) {
            double u = u01(w.x);
            double e = exp(-2.0 * alpha);
            double s = 1.0 + log(e + u * (1.0 - e)) / alpha;
            if (u01(w.y) <= sqrt(1.0 - s * s)) {
                s0 = s;
                ok = true;
                break;
            }
        } else {
            double c = cos(GF_TWO_PI * u01(w.y));
            double lam2 = -(log(u01(w.x)) + c * c * log(u01(w.z))) / (2.0 * alpha);
            double v = u01(w.w);
            if (v * v <= 1.0 - lam2) {
                s0 = 1.0 - 2.0 * lam2;
                ok = true;
                break;
            }
        }
    }
    if (!ok) {
        d.st = 0;
        return d;
    }
    uint4 w = philox4x32_10(make_uint4(site, sweep, (uint32_t)sg * 256u + GF_SA_DIRECTION, tag), key);
    double ct = 2.0 * u01(w.x) - 1.0;
    double phi = GF_TWO_PI * u01(w.y);
    double st = sqrt(1.0 - ct * ct);
    double rho = sqrt(1.0 - s0 * s0);
    double sp, cp;
    sincos(phi, &sp, &cp);
    double s[4] = { s0, rho * st * cp, rho * st * sp, rho * ct };
    const double ikn = 1.0 / kn;  // one FP64 division instead of four
    double kh[4] = { k0 * ikn, k1 * ikn, k2 * ikn, k3 * ikn };
    // r = s kh (product of the SU(2) matrices)
    d.r0 = s[0] * kh[0] - (s[1] * kh[1] + s[2] * kh[2] + s[3] * kh[3]);
    d.r1 = s[0] * kh[1] + kh[0] * s[1] - (s[2] * kh[3] - s[3] * kh[2]);
    d.r2 = s[0] * kh[2] + kh[0] * s[2] - (s[3] * kh[1] - s[1] * kh[3]);
    d.r3 = s[0] * kh[3] + kh[0] * s[3] - (s[1] * kh[2] - s[2] * kh[1]);
    d.st = 1;
    return d;
}

// open-interval uniform (0,1) in FP32 from the top 23 bits of a word: ((w >> 9) + 1/2) / 2^23, exact
__device__ __forceinline__ float u01f(uint32_t w) { return __fmul_rn(__fadd_rn((float)(w >> 9), 0.5f), 1.0f / 8388608.0f); }

#define GF_TWO_PI_F 6.28318530717958647692f

// The FP32 reading of the same draw (option "sa_draw" 1, annealing only):
// alpha = |k|/T in FP64 rounded once to FP32, uniforms u01f, every later
// operation one FP32 operation in the order written (the _rn intrinsics keep
// the compiler from contracting them into fused multiply-adds, so only the
// library's expf, logf, cosf and sinf may differ from another correctly
// written implementation, by an ulp); the drawn element is widened to FP64 and
// normalised in FP64 before the product with k/|k|, so that the rotation stays
// unitary to FP64 rounding.  The FP32 pipe and the special-function units do
// the transcendental work that the FP64 reading leaves to the small FP64 unit.
static __device__ __noinline__ HeatbathDraw heatbath_draw_f32(double k0, double k1, double k2, double k3, double T,
                                                              uint32_t site, uint32_t sweep, int sg, int cap, uint2 key,
                                                              uint32_t tag)
{
    HeatbathDraw d;
    d.r0 = d.r1 = d.r2 = d.r3 = 0.0;
    d.st = 2;
    double kn = sqrt(k0 * k0 + k1 * k1 + k2 * k2 + k3 * k3);
    if (kn == 0.0) return d;
    const float alpha = __double2float_rn(kn / T);
    float s0 = 0.0f;
    bool ok = false;
    for (int a = 0; a < cap && a < (int)GF_SA_DIRECTION; ++a) {
        uint4 w = philox4x32_10(make_uint4(site, sweep, (uint32_t)sg * 256u + (uint32_t)a, tag), key);
        if (alpha < (float)GF_SA_ALPHA_SWITCH) {
            const float u = u01f(w.x);
            const float e = expf(__fmul_rn(-2.0f, alpha));
            const float s = __fadd_rn(1.0f, __fdiv_rn(logf(__fadd_rn(e, __fmul_rn(u, __fsub_rn(1.0f, e)))), alpha));
            if (u01f(w.y) <= __fsqrt_rn(__fsub_rn(1.0f, __fmul_rn(s, s)))) {
                s0 = s;
                ok = true;
                break;
            }
        } else {
            const float c = cosf(__fmul_rn(GF_TWO_PI_F, u01f(w.y)));
            const float lam2 = -__fdiv_rn(__fadd_rn(logf(u01f(w.x)), __fmul_rn(__fmul_rn(c, c), logf(u01f(w.z)))),
                                          __fmul_rn(2.0f, alpha));
            const float v = u01f(w.w);
            if (__fmul_rn(v, v) <= __fsub_rn(1.0f, lam2)) {
                s0 = __fsub_rn(1.0f, __fmul_rn(2.0f, lam2));
                ok = true;
                break;
            }
        }
    }
    if (!ok) {
        d.st = 0;
        return d;
    }
    uint4 w = philox4x32_10(make_uint4(site, sweep, (uint32_t)sg * 256u + GF_SA_DIRECTION, tag), key);
    const float ct = __fsub_rn(__fmul_rn(2.0f, u01f(w.x)), 1.0f);
    const float phi = __fmul_rn(GF_TWO_PI_F, u01f(w.y));
    const float st = __fsqrt_rn(__fsub_rn(1.0f, __fmul_rn(ct, ct)));
    const float rho = __fsqrt_rn(__fsub_rn(1.0f, __fmul_rn(s0, s0)));
    const float rs = __fmul_rn(rho, st);
    double s[4] = { (double)s0, (double)__fmul_rn(rs, cosf(phi)), (double)__fmul_rn(rs, sinf(phi)),
                    (double)__fmul_rn(rho, ct) };
    const double sn = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3]);
#pragma unroll
    for (int c = 0; c < 4; ++c) s[c] /= sn;
    const double ikn = 1.0 / kn;
    double kh[4] = { k0 * ikn, k1 * ikn, k2 * ikn, k3 * ikn };
    d.r0 = s[0] * kh[0] - (s[1] * kh[1] + s[2] * kh[2] + s[3] * kh[3]);
    d.r1 = s[0] * kh[1] + kh[0] * s[1] - (s[2] * kh[3] - s[3] * kh[2]);
    d.r2 = s[0] * kh[2] + kh[0] * s[2] - (s[3] * kh[1] - s[1] * kh[3]);
    d.r3 = s[0] * kh[3] + kh[0] * s[3] - (s[1] * kh[2] - s[2] * kh[1]);
    d.st = 1;
    return d;
}

// the draw above (fp32: its FP32 reading); r is written only on success (return value 1)
__device__ __forceinline__ int heatbath_quat(const double k[4], double T, uint32_t site, uint32_t sweep, int sg,
                                             int cap, uint2 key, double r[4], uint32_t tag = GF_SA_TAG,
                                             bool fp32 = false)
{
    const HeatbathDraw d = fp32 ? heatbath_draw_f32(k[0], k[1], k[2], k[3], T, site, sweep, sg, cap, key, tag)
                                : heatbath_draw(k[0], k[1], k[2], k[3], T, site, sweep, sg, cap, key, tag);
    if (d.st == 1) {
        r[0] = d.r0;
        r[1] = d.r1;
        r[2] = d.r2;
        r[3] = d.r3;
    }
    return d.st;
}

// Stochastic relaxation: the maximiser r* = k/|k|, replaced with probability
// p by r*^2 (the microcanonical reflection through the maximum).  The draw is
// the first word of Philox counter (site, sweep, 256 * subgroup, 2); the
// decision u < p is taken in FP64.  Returns false when k = 0.
#define GF_SR_TAG 2u
template <class T>
__device__ __forceinline__ bool sr_quat(const T k[4], double p, uint32_t site, uint32_t sweep, int sg, uint2 key,
                                        T r[4])
{
    T n2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2] + k[3] * k[3];
    if (n2 == T(0)) return false;
    T inv = T(1) / sqrt(n2);
#pragma unroll
    for (int c = 0; c < 4; ++c) r[c] = k[c] * inv;
    uint4 w = philox4x32_10(make_uint4(site, sweep, (uint32_t)sg * 256u, GF_SR_TAG), key);
    if (u01(w.x) < p) {
        T r0 = r[0];
        r[0] = T(2) * r0 * r0 - T(1);
        r[1] = T(2) * r0 * r[1];
        r[2] = T(2) * r0 * r[2];
        r[3] = T(2) * r0 * r[3];
    }
    return true;
}

}  // namespace gf
