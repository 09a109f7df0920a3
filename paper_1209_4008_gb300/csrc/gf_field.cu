// gf_field.cu -- whole-field kernels: conversion between the canonical
// array-of-structures field and the per-parity structure-of-arrays storage
// (Sec. 4.1), reunitarisation, FP32 -> FP64 widening, application of the
// gauge transformation accumulated during the FP32 phase, and the
// deterministic FP64 reductions of F (eq. F_g), theta (eq. theta) and the
// plaquette.
#include "gf.h"
#include "gf_fieldops.cuh"

namespace gf {

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

template <int FMT, bool COULOMB>
__global__ void __launch_bounds__(kReduceBlock) k_measure(FieldRef f, Geom g, double *partials)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    double fsum = 0.0, tsum = 0.0;
    if (t < 2 * g.Vh) {
        int p = t >= g.Vh ? 1 : 0;
        measure_site<FMT, COULOMB>(f, g, p, t - p * g.Vh, fsum, tsum);
    }
    block_sum2(fsum, tsum, partials + 2 * blockIdx.x);
}

// per timeslice: block (b, t) covers sites b*blockDim .. of timeslice t (both
// parities; the half-sites of a timeslice are contiguous, Lx Ly Lz / 2 of each)
template <int FMT, bool COULOMB>
__global__ void __launch_bounds__(kReduceBlock) k_measure_slices(FieldRef f, Geom g, double *partials)
{
    const int hs = g.Vh / g.L[3];  // half-sites per timeslice and parity
    const int t = blockIdx.y;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    double fsum = 0.0, tsum = 0.0;
    if (j < 2 * hs) {
        int p = j >= hs ? 1 : 0;
        measure_site<FMT, COULOMB>(f, g, p, t * hs + (j - p * hs), fsum, tsum);
    }
    block_sum2(fsum, tsum, partials + 2 * ((long)t * gridDim.x + blockIdx.x));
}

// slices[2t], slices[2t+1] = F_t, theta_t (fixed-order sums of the block partials)
__global__ void k_finalize_slices(const double *__restrict__ partials, int nb, double sa, double sb,
                                  double *slices)
{
    const int t = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += partials[2 * ((long)t * nb + i)];
        b += partials[2 * ((long)t * nb + i) + 1];
    }
    __shared__ double r[2];
    block_sum2(a, b, r);
    __syncthreads();
    if (threadIdx.x == 0) {
        slices[2 * t] = r[0] * sa;
        slices[2 * t + 1] = r[1] * sb;
    }
}

// out[0] = mean of F_t (the global F), out[1] = max of theta_t
__global__ void k_slices_summary(const double *__restrict__ slices, int Lt, double *out)
{
    if (threadIdx.x != 0) return;
    double f = 0.0, m = 0.0;
    for (int t = 0; t < Lt; ++t) {
        f += slices[2 * t];
        m = fmax(m, slices[2 * t + 1]);
    }
    out[0] = f / (double)Lt;
    out[1] = m;
}

template <int FMT>
__global__ void __launch_bounds__(kReduceBlock) k_measure_mag(FieldRef f, Geom g, double *partials)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    double fsum = 0.0, tsum = 0.0;
    if (t < 2 * g.Vh) {
        int p = t >= g.Vh ? 1 : 0;
        measure_site_mag<FMT>(f, g, p, t - p * g.Vh, fsum, tsum);
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
    case DF64_18: CALL(DF64_18); break;         \
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
    else if (src_fmt == F32_12 && dst_fmt == DF64_18) k_transcode<F32_12, DF64_18><<<n, 256, 0, s>>>(src, dst, g);
    else if (src_fmt == F32_18 && dst_fmt == DF64_18) k_transcode<F32_18, DF64_18><<<n, 256, 0, s>>>(src, dst, g);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_narrow(int src_fmt, FieldRef src, int dst_fmt, FieldRef dst, const Geom &g, cudaStream_t s)
{
    int n = nblocks(8L * g.Vh, 256);
    if (src_fmt == F64_18 && dst_fmt == F32_12) k_transcode<F64_18, F32_12><<<n, 256, 0, s>>>(src, dst, g);
    else if (src_fmt == F64_18 && dst_fmt == F32_18) k_transcode<F64_18, F32_18><<<n, 256, 0, s>>>(src, dst, g);
    else if (src_fmt == F64_12 && dst_fmt == F32_12) k_transcode<F64_12, F32_12><<<n, 256, 0, s>>>(src, dst, g);
    else if (src_fmt == F64_12 && dst_fmt == F32_18) k_transcode<F64_12, F32_18><<<n, 256, 0, s>>>(src, dst, g);
    else if (src_fmt == DF64_18 && dst_fmt == F32_12) k_transcode<DF64_18, F32_12><<<n, 256, 0, s>>>(src, dst, g);
    else if (src_fmt == DF64_18 && dst_fmt == F32_18) k_transcode<DF64_18, F32_18><<<n, 256, 0, s>>>(src, dst, g);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_to_df(int src_fmt, FieldRef src, FieldRef dst, const Geom &g, cudaStream_t s)
{
    int n = nblocks(8L * g.Vh, 256);
    if (src_fmt == F64_18) k_transcode<F64_18, DF64_18><<<n, 256, 0, s>>>(src, dst, g);
    else if (src_fmt == F64_12) k_transcode<F64_12, DF64_18><<<n, 256, 0, s>>>(src, dst, g);
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
    else if (dst_fmt == DF64_18) k_apply_tracked_gauge<DF64_18><<<n, 128, 0, s>>>(aos, gt, dst, g);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

int measure_blocks(const Geom &g) { return nblocks(2L * g.Vh, kReduceBlock); }
int aos_blocks(const Geom &g) { return nblocks(2L * g.Vh, kReduceBlock); }

cudaError_t launch_measure(int fmt, FieldRef f, const Geom &g, int coulomb, double *partials, double *out,
                           cudaStream_t s)
{
    int n = measure_blocks(g);
    if (coulomb == GF_MAG) {  // maximally Abelian gauge: F_MAG and theta_MAG
        if (fmt == DF64_18) return cudaErrorInvalidValue;
#define GF_CALL(F) k_measure_mag<F><<<n, kReduceBlock, 0, s>>>(f, g, partials)
        GF_FMT_SWITCH(fmt, GF_CALL)
#undef GF_CALL
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        double V = 2.0 * g.Vh;
        k_finalize<<<1, 256, 0, s>>>(partials, n, 1.0 / (3.0 * 4.0 * V), 1.0 / (3.0 * V), out);
        return cudaGetLastError();
    }
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

int slice_blocks(const Geom &g) { return nblocks(2L * (g.Vh / g.L[3]), kReduceBlock); }

cudaError_t launch_measure_slices(int fmt, FieldRef f, const Geom &g, int coulomb, double *partials,
                                  double *slices, double *out, cudaStream_t s)
{
    int nb = slice_blocks(g);
    dim3 grid(nb, g.L[3]);
#define GF_CALL(F)                                                                   \
    if (coulomb) k_measure_slices<F, true><<<grid, kReduceBlock, 0, s>>>(f, g, partials); \
    else k_measure_slices<F, false><<<grid, kReduceBlock, 0, s>>>(f, g, partials)
    GF_FMT_SWITCH(fmt, GF_CALL)
#undef GF_CALL
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double Ls = 2.0 * g.Vh / g.L[3];
    k_finalize_slices<<<g.L[3], 256, 0, s>>>(partials, nb, 1.0 / (3.0 * (coulomb ? 3 : 4) * Ls), 1.0 / (3.0 * Ls),
                                             slices);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_slices_summary<<<1, 32, 0, s>>>(slices, g.L[3], out);
    return cudaGetLastError();
}

// maximally Abelian gauge on a canonical field (see measure_site_mag)
__global__ void __launch_bounds__(kReduceBlock) k_measure_aos_mag(const double *__restrict__ aos, Geom g,
                                                                  double *partials)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double fsum = 0.0, tsum = 0.0;
    if (i < 2 * g.Vh) {
        int c[4];
        coords_of_lex(g, i, c);
        double hs[3][4] = { { 0 } };
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            mat3<double> u = load_aos(aos, 4L * i + mu);
#pragma unroll
            for (int a = 0; a < 3; ++a) fsum += u.e[a][a].re * u.e[a][a].re + u.e[a][a].im * u.e[a][a].im;
            int st = lex_stride(g, mu);
            int j = coord_of(c, mu) == 0 ? i + (extent_of(g, mu) - 1) * st : i - st;
            const mat3<double> x = dagger(load_aos(aos, 4L * j + mu));
#pragma unroll
            for (int sg = 0; sg < 3; ++sg) {
                int a, b;
                subgroup_rows(sg, a, b);
                add_mag_terms(u, a, b, hs[sg]);
                add_mag_terms(x, a, b, hs[sg]);
            }
        }
#pragma unroll
        for (int sg = 0; sg < 3; ++sg) tsum += hs[sg][2] * hs[sg][2] + hs[sg][3] * hs[sg][3];
    }
    block_sum2(fsum, tsum, partials + 2 * blockIdx.x);
}

cudaError_t launch_measure_aos(const double *aos, const Geom &g, int coulomb, double *partials, double *out,
                               cudaStream_t s)
{
    int n = aos_blocks(g);
    if (coulomb == GF_MAG) {
        k_measure_aos_mag<<<n, kReduceBlock, 0, s>>>(aos, g, partials);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        double V = 2.0 * g.Vh;
        k_finalize<<<1, 256, 0, s>>>(partials, n, 1.0 / (3.0 * 4.0 * V), 1.0 / (3.0 * V), out);
        return cudaGetLastError();
    }
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
