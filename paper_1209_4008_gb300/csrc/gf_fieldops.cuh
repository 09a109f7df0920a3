// gf_fieldops.cuh -- device helpers shared by the whole-field kernels and the
// batched kernels: FP64 views of stored links, canonical-layout access,
// reunitarisation, 3x3 products, the per-site measurement of F and theta,
// and the fixed-order block sum.
#pragma once

#include "gf_internal.h"

namespace gf {

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

// x y, accumulated as one multiply and FMAs per component (no separate adds)
__device__ __forceinline__ mat3<double> mul3(const mat3<double> &x, const mat3<double> &y)
{
    mat3<double> z;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            double re = x.e[a][0].re * y.e[0][b].re;
            double im = x.e[a][0].re * y.e[0][b].im;
            re = fma(-x.e[a][0].im, y.e[0][b].im, re);
            im = fma(x.e[a][0].im, y.e[0][b].re, im);
#pragma unroll
            for (int c = 1; c < 3; ++c) {
                re = fma(x.e[a][c].re, y.e[c][b].re, re);
                re = fma(-x.e[a][c].im, y.e[c][b].im, re);
                im = fma(x.e[a][c].re, y.e[c][b].im, im);
                im = fma(x.e[a][c].im, y.e[c][b].re, im);
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

// fixed-order block sum of two doubles; thread 0 of warp 0 writes out2[0..1]
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

// the same accumulation in the storage precision A (FP32 fields: the FP32
// phase only decides theta against thresholds >= 1e-12, far above FP32
// rounding of the O(1) link entries, ~1e-7 in Delta)
template <class T, class A>
__device__ __forceinline__ void add_antiherm_p(const mat3<T> &u, A s, A dre[3][3], A dim[3][3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dre[a][a] += s * (A)u.e[a][a].im;
#pragma unroll
        for (int b = a + 1; b < 3; ++b) {
            dre[a][b] += s * A(0.5) * ((A)u.e[a][b].im + (A)u.e[b][a].im);
            dim[a][b] -= s * A(0.5) * ((A)u.e[a][b].re - (A)u.e[b][a].re);
        }
    }
}

template <class A>
__device__ __forceinline__ double traceless_norm2_p(A dre[3][3], A dim[3][3])
{
    A tr = (dre[0][0] + dre[1][1] + dre[2][2]) * A(1.0 / 3.0);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        A d = dre[a][a] - tr;
        s += (double)(d * d);
#pragma unroll
        for (int b = a + 1; b < 3; ++b) s += 2.0 * (double)(dre[a][b] * dre[a][b] + dim[a][b] * dim[a][b]);
    }
    return s;
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


// Re tr U_mu(x) (mu < NK) and tr[D D^dagger] of the traceless D(x) =
// sum_mu [A_mu(x) - A_mu(x - mu)] for half-site h of parity p of a stored field
template <int FMT, bool COULOMB>
__device__ __forceinline__ void measure_site(const FieldRef &f, const Geom &g, int p, int h, double &fsum,
                                             double &tsum)
{
    typedef Store<FMT> S;
    typedef typename S::T T;  // per-site sums in the storage precision, totals in FP64
    constexpr int NK = COULOMB ? 3 : 4;
    int c[4];
    site_coords(g, p, h, c);
    T dre[3][3] = { { T(0) } }, dim[3][3] = { { T(0) } };
    T fs = T(0);
#pragma unroll
    for (int mu = 0; mu < NK; ++mu) {
        mat3<T> u;
        S::load(f, (p * 4 + mu) * S::NCHUNK, h, u);
        fs += u.e[0][0].re + u.e[1][1].re + u.e[2][2].re;
        add_antiherm_p<T, T>(u, T(1), dre, dim);
        S::load(f, ((p ^ 1) * 4 + mu) * S::NCHUNK, back_half(g, c, mu), u);
        add_antiherm_p<T, T>(u, T(-1), dre, dim);
    }
    fsum = (double)fs;
    tsum = traceless_norm2_p<T>(dre, dim);
}

// Maximally Abelian gauge: F part sum_mu sum_i |U_mu(x)_ii|^2, theta part
// sum over the three subgroups of |h12|^2, h12 the off-diagonal element of the
// local matrix H of the subgroup step at the identity (the squared gradient of
// the local functional along the directions that are not the residual U(1))
template <int FMT>
__device__ __forceinline__ void measure_site_mag(const FieldRef &f, const Geom &g, int p, int h, double &fsum,
                                                 double &tsum)
{
    typedef Store<FMT> S;
    typedef typename S::T T;
    int c[4];
    site_coords(g, p, h, c);
    T hs[3][4] = { { T(0) } };
    T fs = T(0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        mat3<T> u;
        S::load(f, (p * 4 + mu) * S::NCHUNK, h, u);
#pragma unroll
        for (int i = 0; i < 3; ++i) fs += u.e[i][i].re * u.e[i][i].re + u.e[i][i].im * u.e[i][i].im;
#pragma unroll
        for (int sg = 0; sg < 3; ++sg) {
            int a, b;
            subgroup_rows(sg, a, b);
            add_mag_terms(u, a, b, hs[sg]);
        }
        S::load(f, ((p ^ 1) * 4 + mu) * S::NCHUNK, back_half(g, c, mu), u);
        const mat3<T> x = dagger(u);
#pragma unroll
        for (int sg = 0; sg < 3; ++sg) {
            int a, b;
            subgroup_rows(sg, a, b);
            add_mag_terms(x, a, b, hs[sg]);
        }
    }
    fsum = (double)fs;
    double t = 0.0;
#pragma unroll
    for (int sg = 0; sg < 3; ++sg) t += (double)hs[sg][2] * (double)hs[sg][2] + (double)hs[sg][3] * (double)hs[sg][3];
    tsum = t;
}

}  // namespace gf
