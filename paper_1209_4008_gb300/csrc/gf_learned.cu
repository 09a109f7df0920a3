// gf_learned.cu -- field-side kernels of the learned warm start: the network's
// inputs from the resident FP64 field, the algebra coefficients of the tracked
// gauge transformation (training labels), and the application of a predicted
// gauge transformation g(x) = exp(i s sum_a c_a lambda_a / 2) to the resident
// field as an exact FP64 gauge transformation (eq. 1).
#include <cuda_bf16.h>

#include "gf_fieldops.cuh"

namespace gf {

// tr(lambda_a X) for the Hermitian X given by its real diagonal and upper
// triangle (dre, dim), a = 1..8 (Gell-Mann basis, tr(lambda_a lambda_b) = 2 delta)
__device__ __forceinline__ void gell_mann_components(const double dre[3][3], const double dim[3][3], double out[8])
{
    const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
    out[0] = 2.0 * dre[0][1];
    out[1] = -2.0 * dim[0][1];
    out[2] = dre[0][0] - dre[1][1];
    out[3] = 2.0 * dre[0][2];
    out[4] = -2.0 * dim[0][2];
    out[5] = 2.0 * dre[1][2];
    out[6] = -2.0 * dim[1][2];
    out[7] = (dre[0][0] + dre[1][1] - 2.0 * dre[2][2]) * r3;
}

// lex site -> (parity, half index)
__device__ __forceinline__ void parity_half(const Geom &g, int i, int &p, int &h, int c[4])
{
    coords_of_lex(g, i, c);
    p = (c[0] + c[1] + c[2] + c[3]) & 1;
    h = i >> 1;
}

// network inputs: 72 forward-link reals, then tr(lambda_a Delta(x)) * inv_scale
template <int FMT>
__global__ void k_features(FieldRef f, Geom g, double inv_scale, __nv_bfloat16 *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * g.Vh) return;
    int c[4], p, h;
    parity_half(g, i, p, h, c);
    __nv_bfloat16 *o = out + (long)i * 80;
    double dre[3][3] = { { 0 } }, dim[3][3] = { { 0 } };
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        mat3<double> u = load_d<FMT>(f, (p * 4 + mu) * Store<FMT>::NCHUNK, h);
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            o[mu * 18 + 2 * e] = __double2bfloat16(u.e[e / 3][e % 3].re);
            o[mu * 18 + 2 * e + 1] = __double2bfloat16(u.e[e / 3][e % 3].im);
        }
        add_antiherm(u, 1.0, dre, dim);
        add_antiherm(load_d<FMT>(f, ((p ^ 1) * 4 + mu) * Store<FMT>::NCHUNK, back_half(g, c, mu)), -1.0, dre,
                     dim);
    }
    double d8[8];
    gell_mann_components(dre, dim, d8);
#pragma unroll
    for (int a = 0; a < 8; ++a) o[72 + a] = __double2bfloat16(d8[a] * inv_scale);
}

// labels: tr(lambda_a (g - g^+)/(2i)) * inv_scale of the tracked g (first-order log)
__global__ void k_gauge_algebra(FieldRef gt, Geom g, double inv_scale, float *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * g.Vh) return;
    int c[4], p, h;
    parity_half(g, i, p, h, c);
    mat3<double> u = load_d<F32_12>(gt, p * 3, h);
    reunitarize3(u);
    double dre[3][3] = { { 0 } }, dim[3][3] = { { 0 } };
    add_antiherm(u, 1.0, dre, dim);
    double d8[8];
    gell_mann_components(dre, dim, d8);
#pragma unroll
    for (int a = 0; a < 8; ++a) out[(long)i * 8 + a] = (float)(d8[a] * inv_scale);
}

// exp(i H), H = s sum_a c_a lambda_a / 2: Taylor series of order 12 after
// halving until the Frobenius norm of H is below 1/8, then squaring back
__device__ mat3<double> expmap_su3(const float *c8, double s)
{
    const double r3 = 0.57735026918962576451;
    double c[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) c[a] = 0.5 * s * (double)c8[a];
    mat3<double> H;
    H.e[0][0] = mk<double>(c[2] + c[7] * r3, 0.0);
    H.e[1][1] = mk<double>(-c[2] + c[7] * r3, 0.0);
    H.e[2][2] = mk<double>(-2.0 * c[7] * r3, 0.0);
    H.e[0][1] = mk<double>(c[0], -c[1]);
    H.e[0][2] = mk<double>(c[3], -c[4]);
    H.e[1][2] = mk<double>(c[5], -c[6]);
    H.e[1][0] = mk<double>(c[0], c[1]);
    H.e[2][0] = mk<double>(c[3], c[4]);
    H.e[2][1] = mk<double>(c[5], c[6]);
    double n2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) n2 += H.e[a][b].re * H.e[a][b].re + H.e[a][b].im * H.e[a][b].im;
    double nrm = sqrt(n2);
    int sq = 0;
    while (nrm > 0.125 && sq < 60) {
        nrm *= 0.5;
        ++sq;
    }
    double sc = ldexp(1.0, -sq);
    mat3<double> A;  // i H sc
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) A.e[a][b] = mk<double>(-H.e[a][b].im * sc, H.e[a][b].re * sc);
    mat3<double> E = identity3<double>(), T = identity3<double>();
    for (int k = 1; k <= 12; ++k) {
        T = mul3(T, A);
        double inv = 1.0 / (double)k;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                T.e[a][b].re *= inv;
                T.e[a][b].im *= inv;
                E.e[a][b].re += T.e[a][b].re;
                E.e[a][b].im += T.e[a][b].im;
            }
    }
    for (int k = 0; k < sq; ++k) E = mul3(E, E);
    return E;
}

__global__ void k_expmap_to_gauge(const float *__restrict__ c, double s, FieldRef gt, Geom g)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * g.Vh) return;
    int cc[4], p, h;
    parity_half(g, i, p, h, cc);
    store_d<F32_12>(gt, p * 3, h, expmap_su3(c + (long)i * 8, s));
}

// resident FP64 field <- g(x) U_mu(x) g(x+mu)^dagger, g from the FP32 site
// field reunitarised in FP64; one thread per (parity, mu, half site), in place
template <int FMT>
__global__ void k_gauge_transform_resident(FieldRef f, FieldRef gt, Geom g)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8L * g.Vh) return;
    int h = (int)(t % g.Vh), pm = (int)(t / g.Vh);
    int p = pm >> 2, mu = pm & 3;
    int c[4];
    site_coords(g, p, h, c);
    mat3<double> gx = load_d<F32_12>(gt, p * 3, h);
    mat3<double> gy = load_d<F32_12>(gt, (p ^ 1) * 3, fwd_half(g, c, mu));
    reunitarize3(gx);
    reunitarize3(gy);
    mat3<double> u = load_d<FMT>(f, pm * Store<FMT>::NCHUNK, h);
    store_d<FMT>(f, pm * Store<FMT>::NCHUNK, h, mul3(mul3(gx, u), dagger(gy)));
}

// U_mu(x) := g(x) U_mu(x) g(x+mu)^dagger in FP64 with g = 1 + E read from the
// double-float site field ge (E = g - 1 as tracked by the double-float sweeps),
// reunitarised in FP64: the FP64 field stays a gauge transform of its input to
// FP64 rounding
template <int FMT>
__global__ void k_apply_gauge_e(FieldRef f, FieldRef ge, Geom g)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8L * g.Vh) return;
    int h = (int)(t % g.Vh), pm = (int)(t / g.Vh);
    int p = pm >> 2, mu = pm & 3;
    int c[4];
    site_coords(g, p, h, c);
    mat3<double> gx = load_d<DF64_18>(ge, p * 9, h);
    mat3<double> gy = load_d<DF64_18>(ge, (p ^ 1) * 9, fwd_half(g, c, mu));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        gx.e[i][i].re += 1.0;
        gy.e[i][i].re += 1.0;
    }
    reunitarize3(gx);
    reunitarize3(gy);
    mat3<double> u = load_d<FMT>(f, pm * Store<FMT>::NCHUNK, h);
    store_d<FMT>(f, pm * Store<FMT>::NCHUNK, h, mul3(mul3(gx, u), dagger(gy)));
}

// tracked g as a canonical site field double g[V][3][3][2] (reunitarised)
__global__ void k_decode_gauge(FieldRef gt, Geom g, double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * g.Vh) return;
    int c[4], p, h;
    parity_half(g, i, p, h, c);
    mat3<double> u = load_d<F32_12>(gt, p * 3, h);
    reunitarize3(u);
    store_aos(out, i, u);  // 18 doubles per site
}

static inline int nb(long n, int b) { return (int)((n + b - 1) / b); }

cudaError_t launch_features(int fmt, FieldRef f, const Geom &g, double inv_scale, void *out, cudaStream_t s)
{
    __nv_bfloat16 *o = static_cast<__nv_bfloat16 *>(out);
    if (fmt == F64_18) k_features<F64_18><<<nb(2L * g.Vh, 128), 128, 0, s>>>(f, g, inv_scale, o);
    else if (fmt == F64_12) k_features<F64_12><<<nb(2L * g.Vh, 128), 128, 0, s>>>(f, g, inv_scale, o);
    else if (fmt == DF64_18) k_features<DF64_18><<<nb(2L * g.Vh, 128), 128, 0, s>>>(f, g, inv_scale, o);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_gauge_algebra(FieldRef gt, const Geom &g, double inv_scale, float *out, cudaStream_t s)
{
    k_gauge_algebra<<<nb(2L * g.Vh, 128), 128, 0, s>>>(gt, g, inv_scale, out);
    return cudaGetLastError();
}

cudaError_t launch_expmap_to_gauge(const float *c, double scale, FieldRef gt, const Geom &g, cudaStream_t s)
{
    k_expmap_to_gauge<<<nb(2L * g.Vh, 128), 128, 0, s>>>(c, scale, gt, g);
    return cudaGetLastError();
}

cudaError_t launch_gauge_transform_resident(int fmt, FieldRef f, FieldRef gt, const Geom &g, cudaStream_t s)
{
    int n = nb(8L * g.Vh, 128);
    if (fmt == F64_18) k_gauge_transform_resident<F64_18><<<n, 128, 0, s>>>(f, gt, g);
    else if (fmt == F64_12) k_gauge_transform_resident<F64_12><<<n, 128, 0, s>>>(f, gt, g);
    else if (fmt == DF64_18) k_gauge_transform_resident<DF64_18><<<n, 128, 0, s>>>(f, gt, g);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_apply_gauge_e(int fmt, FieldRef f, FieldRef ge, const Geom &g, cudaStream_t s)
{
    int n = nb(8L * g.Vh, 128);
    if (fmt == F64_18) k_apply_gauge_e<F64_18><<<n, 128, 0, s>>>(f, ge, g);
    else if (fmt == F64_12) k_apply_gauge_e<F64_12><<<n, 128, 0, s>>>(f, ge, g);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_decode_gauge(FieldRef gt, const Geom &g, double *out, cudaStream_t s)
{
    k_decode_gauge<<<nb(2L * g.Vh, 128), 128, 0, s>>>(gt, g, out);
    return cudaGetLastError();
}

}  // namespace gf
