// gf_field.cu -- whole-field kernels: conversion between the canonical
// array-of-structures field and the per-parity structure-of-arrays storage
// (Sec. 4.1), reunitarisation, FP32 -> FP64 widening, application of the
// gauge transformation accumulated during the FP32 phase, and the
// deterministic FP64 reductions of F (eq. F_g), theta (eq. theta) and the
// plaquette.
#include "gf_internal.h"

namespace gf {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
template <int FMT>
__device__ __forceinline__ mat3<double> load_d(const FieldRef &f, int pl0, int h)
{
    typedef Store<FMT> S;
    mat3<typename S::T> u;
    S::load(f, pl0, h, u);
    mat3<double> d;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) d.e[a][b] = mk<double>((double)u.e[a][b].re, (double)u.e[a][b].im);
    if (S::REALS == 12) rebuild_row2(d);
    return d;
}

template <int FMT>
__device__ __forceinline__ void store_d(const FieldRef &f, int pl0, int h, const mat3<double> &d)
{
    typedef Store<FMT> S;
    typedef typename S::T T;
    mat3<T> u;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) u.e[a][b] = mk<T>((T)d.e[a][b].re, (T)d.e[a][b].im);
    S::store(f, pl0, h, u);
}

__device__ __forceinline__ mat3<double> load_aos(const double *aos, long link)
{
    const double2 *p = reinterpret_cast<const double2 *>(aos + link * 18);
    mat3<double> u;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        double2 v = p[c];
        u.e[c / 3][c % 3] = mk<double>(v.x, v.y);
    }
    return u;
}

__device__ __forceinline__ void store_aos(double *aos, long link, const mat3<double> &u)
{
    double2 *p = reinterpret_cast<double2 *>(aos + link * 18);
#pragma unroll
    for (int c = 0; c < 9; ++c) p[c] = make_double2(u.e[c / 3][c % 3].re, u.e[c / 3][c % 3].im);
}

// Gram-Schmidt on rows 0, 1, then row 2 = conj(row0 x row1): projects onto SU(3)
__device__ __forceinline__ void reunitarize3(mat3<double> &u)
{
    double n0 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) n0 += u.e[0][c].re * u.e[0][c].re + u.e[0][c].im * u.e[0][c].im;
    n0 = rsqrt(n0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        u.e[0][c].re *= n0;
        u.e[0][c].im *= n0;
    }
    double ipr = 0.0, ipi = 0.0;  // <row0, row1> = sum conj(row0) row1
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        ipr += u.e[0][c].re * u.e[1][c].re + u.e[0][c].im * u.e[1][c].im;
        ipi += u.e[0][c].re * u.e[1][c].im - u.e[0][c].im * u.e[1][c].re;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        u.e[1][c].re -= ipr * u.e[0][c].re - ipi * u.e[0][c].im;
        u.e[1][c].im -= ipr * u.e[0][c].im + ipi * u.e[0][c].re;
    }
    double n1 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) n1 += u.e[1][c].re * u.e[1][c].re + u.e[1][c].im * u.e[1][c].im;
    n1 = rsqrt(n1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        u.e[1][c].re *= n1;
        u.e[1][c].im *= n1;
    }
    rebuild_row2(u);
}

__device__ __forceinline__ mat3<double> mul3(const mat3<double> &x, const mat3<double> &y)
{
    mat3<double> z;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                re += x.e[a][c].re * y.e[c][b].re - x.e[a][c].im * y.e[c][b].im;
                im += x.e[a][c].re * y.e[c][b].im + x.e[a][c].im * y.e[c][b].re;
            }
            z.e[a][b] = mk<double>(re, im);
        }
    return z;
}

__device__ __forceinline__ void coords_of_lex(const Geom &g, int i, int c[4])
{
    int r = i / g.L[0];
    c[0] = i - r * g.L[0];
    int r2 = r / g.L[1];
    c[1] = r - r2 * g.L[1];
    c[3] = r2 / g.L[2];
    c[2] = r2 - c[3] * g.L[2];
}

// ---------------------------------------------------------------------------
// codec
// ---------------------------------------------------------------------------
template <int FMT>
__global__ void k_encode(const double *__restrict__ aos, FieldRef f, Geom g)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;  // link = site*4 + mu
    if (t >= 8L * g.Vh) return;
    int i = (int)(t >> 2), mu = (int)(t & 3);
    int c[4];
    coords_of_lex(g, i, c);
    int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    store_d<FMT>(f, (p * 4 + mu) * Store<FMT>::NCHUNK, i >> 1, load_aos(aos, t));
}

template <int FMT>
__global__ void k_decode(FieldRef f, Geom g, double *__restrict__ aos)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8L * g.Vh) return;
    int i = (int)(t >> 2), mu = (int)(t & 3);
    int c[4];
    coords_of_lex(g, i, c);
    int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    store_aos(aos, t, load_d<FMT>(f, (p * 4 + mu) * Store<FMT>::NCHUNK, i >> 1));
}

// one thread per (parity, mu, half site)
template <int SRC, int DST>
__global__ void k_transcode(FieldRef src, FieldRef dst, Geom g)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8L * g.Vh) return;
    int h = (int)(t % g.Vh), pm = (int)(t / g.Vh);  // pm = p*4 + mu
    mat3<double> u = load_d<SRC>(src, pm * Store<SRC>::NCHUNK, h);
    reunitarize3(u);
    store_d<DST>(dst, pm * Store<DST>::NCHUNK, h, u);
}

__global__ void k_gauge_identity(FieldRef gt, Geom g)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2L * g.Vh) return;
    int h = (int)(t % g.Vh), p = (int)(t / g.Vh);
    Store<F32_12>::store(gt, p * 3, h, identity3<float>());
}

// dst_mu(x) = g(x) U_mu(x) g(x+mu)^dagger with g taken from the FP32 site
// field, rebuilt and reunitarised in FP64 (eq. 1 applied to the exact input)
template <int DST>
__global__ void k_apply_tracked_gauge(const double *__restrict__ aos, FieldRef gt, FieldRef dst, Geom g)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8L * g.Vh) return;
    int i = (int)(t >> 2), mu = (int)(t & 3);
    int c[4];
    coords_of_lex(g, i, c);
    int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    mat3<double> gx = load_d<F32_12>(gt, p * 3, i >> 1);
    mat3<double> gy = load_d<F32_12>(gt, (p ^ 1) * 3, fwd_half(g, c, mu));
    reunitarize3(gx);
    reunitarize3(gy);
    mat3<double> u = mul3(mul3(gx, load_aos(aos, t)), dagger(gy));
    store_d<DST>(dst, (p * 4 + mu) * Store<DST>::NCHUNK, i >> 1, u);
}

// ---------------------------------------------------------------------------
// reductions: fixed-order two-level FP64 sums (deterministic run to run)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_sum2(double a, double b, double *out2)
{
    __shared__ double sa[32], sb[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        a = l < nw ? sa[l] : 0.0;
        b = l < nw ? sb[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (l == 0) {
            out2[0] = a;
            out2[1] = b;
        }
    }
}

__global__ void k_finalize(const double *__restrict__ partials, int n, double sa, double sb, double *out)
{
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
    __shared__ double r[2];
    block_sum2(a, b, r);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = r[0] * sa;
        out[1] = r[1] * sb;
    }
}

// A = (U - U^dagger)/(2i) is Hermitian: accumulate D += s A(U) on the upper
// triangle (diagonal real).
template <class T>
__device__ __forceinline__ void add_antiherm(const mat3<T> &u, double s, double dre[3][3], double dim[3][3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dre[a][a] += s * (double)u.e[a][a].im;
#pragma unroll
        for (int b = a + 1; b < 3; ++b) {
            dre[a][b] += s * 0.5 * ((double)u.e[a][b].im + (double)u.e[b][a].im);
            dim[a][b] -= s * 0.5 * ((double)u.e[a][b].re - (double)u.e[b][a].re);
        }
    }
}

// tr[D D^dagger] of the traceless part of the Hermitian D
__device__ __forceinline__ double traceless_norm2(double dre[3][3], double dim[3][3])
{
    double tr = (dre[0][0] + dre[1][1] + dre[2][2]) * (1.0 / 3.0);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double d = dre[a][a] - tr;
        s += d * d;
#pragma unroll
        for (int b = a + 1; b < 3; ++b) s += 2.0 * (dre[a][b] * dre[a][b] + dim[a][b] * dim[a][b]);
    }
    return s;
}

template <int FMT, bool COULOMB>
__global__ void __launch_bounds__(kReduceBlock) k_measure(FieldRef f, Geom g, double *partials)
{
    typedef Store<FMT> S;
    typedef typename S::T T;
    constexpr int NK = COULOMB ? 3 : 4;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    double fsum = 0.0, tsum = 0.0;
    if (t < 2 * g.Vh) {
        int p = t >= g.Vh ? 1 : 0;
        int h = t - p * g.Vh;
        int c[4];
        site_coords(g, p, h, c);
        double dre[3][3] = { { 0 } }, dim[3][3] = { { 0 } };
#pragma unroll
        for (int mu = 0; mu < NK; ++mu) {
            mat3<T> u;
            S::load(f, (p * 4 + mu) * S::NCHUNK, h, u);
            fsum += (double)u.e[0][0].re + (double)u.e[1][1].re + (double)u.e[2][2].re;
            add_antiherm(u, 1.0, dre, dim);
            S::load(f, ((p ^ 1) * 4 + mu) * S::NCHUNK, back_half(g, c, mu), u);
            add_antiherm(u, -1.0, dre, dim);
        }
        tsum = traceless_norm2(dre, dim);
    }
    block_sum2(fsum, tsum, partials + 2 * blockIdx.x);
}

template <bool COULOMB>
__global__ void __launch_bounds__(kReduceBlock) k_measure_aos(const double *__restrict__ aos, Geom g,
                                                              double *partials)
{
    constexpr int NK = COULOMB ? 3 : 4;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double fsum = 0.0, tsum = 0.0;
    if (i < 2 * g.Vh) {
        int c[4];
        coords_of_lex(g, i, c);
        double dre[3][3] = { { 0 } }, dim[3][3] = { { 0 } };
#pragma unroll
        for (int mu = 0; mu < NK; ++mu) {
            mat3<double> u = load_aos(aos, 4L * i + mu);
            fsum += u.e[0][0].re + u.e[1][1].re + u.e[2][2].re;
            add_antiherm(u, 1.0, dre, dim);
            int st = lex_stride(g, mu);
            int j = coord_of(c, mu) == 0 ? i + (extent_of(g, mu) - 1) * st : i - st;
            add_antiherm(load_aos(aos, 4L * j + mu), -1.0, dre, dim);
        }
        tsum = traceless_norm2(dre, dim);
    }
    block_sum2(fsum, tsum, partials + 2 * blockIdx.x);
}

__global__ void __launch_bounds__(kReduceBlock) k_plaquette_aos(const double *__restrict__ aos, Geom g,
                                                                double *partials)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < 2 * g.Vh) {
        int c[4];
        coords_of_lex(g, i, c);
        for (int mu = 0; mu < 4; ++mu) {
            int smu = lex_stride(g, mu);
            int imu = coord_of(c, mu) + 1 == extent_of(g, mu) ? i - (extent_of(g, mu) - 1) * smu : i + smu;
            for (int nu = mu + 1; nu < 4; ++nu) {
                int snu = lex_stride(g, nu);
                int inu = coord_of(c, nu) + 1 == extent_of(g, nu) ? i - (extent_of(g, nu) - 1) * snu : i + snu;
                mat3<double> a = load_aos(aos, 4L * i + mu);
                mat3<double> b = load_aos(aos, 4L * imu + nu);
                mat3<double> cc = load_aos(aos, 4L * inu + mu);
                mat3<double> d = load_aos(aos, 4L * i + nu);
                // Re tr[a b c^+ d^+] = Re tr[(a b)(d c)^+] = sum_xy Re[(ab)_xy conj((dc)_xy)]
                mat3<double> ab = mul3(a, b), dc = mul3(d, cc);
                double re = 0.0;
#pragma unroll
                for (int x = 0; x < 3; ++x)
#pragma unroll
                    for (int y = 0; y < 3; ++y)
                        re += ab.e[x][y].re * dc.e[x][y].re + ab.e[x][y].im * dc.e[x][y].im;
                s += re;
            }
        }
    }
    block_sum2(s, 0.0, partials + 2 * blockIdx.x);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline int nblocks(long n, int b) { return (int)((n + b - 1) / b); }

#define GF_FMT_SWITCH(fmt, CALL)                \
    switch (fmt) {                              \
    case F64_18: CALL(F64_18); break;           \
    case F64_12: CALL(F64_12); break;           \
    case F32_18: CALL(F32_18); break;           \
    case F32_12: CALL(F32_12); break;           \
    default: return cudaErrorInvalidValue;      \
    }

cudaError_t launch_encode(int fmt, const double *aos, FieldRef f, const Geom &g, cudaStream_t s)
{
#define GF_CALL(F) k_encode<F><<<nblocks(8L * g.Vh, 256), 256, 0, s>>>(aos, f, g)
    GF_FMT_SWITCH(fmt, GF_CALL)
#undef GF_CALL
    return cudaGetLastError();
}

cudaError_t launch_decode(int fmt, FieldRef f, const Geom &g, double *aos, cudaStream_t s)
{
#define GF_CALL(F) k_decode<F><<<nblocks(8L * g.Vh, 256), 256, 0, s>>>(f, g, aos)
    GF_FMT_SWITCH(fmt, GF_CALL)
#undef GF_CALL
    return cudaGetLastError();
}

cudaError_t launch_reunitarize(int fmt, FieldRef f, const Geom &g, cudaStream_t s)
{
#define GF_CALL(F) k_transcode<F, F><<<nblocks(8L * g.Vh, 256), 256, 0, s>>>(f, f, g)
    GF_FMT_SWITCH(fmt, GF_CALL)
#undef GF_CALL
    return cudaGetLastError();
}

cudaError_t launch_widen(int src_fmt, FieldRef src, int dst_fmt, FieldRef dst, const Geom &g, cudaStream_t s)
{
    int n = nblocks(8L * g.Vh, 256);
    if (src_fmt == F32_12 && dst_fmt == F64_18) k_transcode<F32_12, F64_18><<<n, 256, 0, s>>>(src, dst, g);
    else if (src_fmt == F32_12 && dst_fmt == F64_12) k_transcode<F32_12, F64_12><<<n, 256, 0, s>>>(src, dst, g);
    else if (src_fmt == F32_18 && dst_fmt == F64_18) k_transcode<F32_18, F64_18><<<n, 256, 0, s>>>(src, dst, g);
    else if (src_fmt == F32_18 && dst_fmt == F64_12) k_transcode<F32_18, F64_12><<<n, 256, 0, s>>>(src, dst, g);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_gauge_identity(FieldRef gt, const Geom &g, cudaStream_t s)
{
    k_gauge_identity<<<nblocks(2L * g.Vh, 256), 256, 0, s>>>(gt, g);
    return cudaGetLastError();
}

cudaError_t launch_apply_tracked_gauge(const double *aos, FieldRef gt, int dst_fmt, FieldRef dst, const Geom &g,
                                       cudaStream_t s)
{
    int n = nblocks(8L * g.Vh, 128);
    if (dst_fmt == F64_18) k_apply_tracked_gauge<F64_18><<<n, 128, 0, s>>>(aos, gt, dst, g);
    else if (dst_fmt == F64_12) k_apply_tracked_gauge<F64_12><<<n, 128, 0, s>>>(aos, gt, dst, g);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

int measure_blocks(const Geom &g) { return nblocks(2L * g.Vh, kReduceBlock); }
int aos_blocks(const Geom &g) { return nblocks(2L * g.Vh, kReduceBlock); }

cudaError_t launch_measure(int fmt, FieldRef f, const Geom &g, int coulomb, double *partials, double *out,
                           cudaStream_t s)
{
    int n = measure_blocks(g);
#define GF_CALL(F)                                                               \
    if (coulomb) k_measure<F, true><<<n, kReduceBlock, 0, s>>>(f, g, partials);  \
    else k_measure<F, false><<<n, kReduceBlock, 0, s>>>(f, g, partials)
    GF_FMT_SWITCH(fmt, GF_CALL)
#undef GF_CALL
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double V = 2.0 * g.Vh;
    k_finalize<<<1, 256, 0, s>>>(partials, n, 1.0 / (3.0 * (coulomb ? 3 : 4) * V), 1.0 / (3.0 * V), out);
    return cudaGetLastError();
}

cudaError_t launch_measure_aos(const double *aos, const Geom &g, int coulomb, double *partials, double *out,
                               cudaStream_t s)
{
    int n = aos_blocks(g);
    if (coulomb) k_measure_aos<true><<<n, kReduceBlock, 0, s>>>(aos, g, partials);
    else k_measure_aos<false><<<n, kReduceBlock, 0, s>>>(aos, g, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double V = 2.0 * g.Vh;
    k_finalize<<<1, 256, 0, s>>>(partials, n, 1.0 / (3.0 * (coulomb ? 3 : 4) * V), 1.0 / (3.0 * V), out);
    return cudaGetLastError();
}

cudaError_t launch_plaquette_aos(const double *aos, const Geom &g, double *partials, double *out, cudaStream_t s)
{
    int n = aos_blocks(g);
    k_plaquette_aos<<<n, kReduceBlock, 0, s>>>(aos, g, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double V = 2.0 * g.Vh;
    k_finalize<<<1, 256, 0, s>>>(partials, n, 1.0 / (18.0 * V), 0.0, out);
    return cudaGetLastError();
}

}  // namespace gf
