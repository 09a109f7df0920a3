// gf_sweep.cuh -- the half-sweep kernel: overrelaxation (Alg. 1) and the
// simulated-annealing heatbath share one skeleton.
//
// One site of the active parity is served by TPS threads (TPS = 1, 2, 4, 8;
// the paper's Fermi kernel used 8, Sec. 4.2).  The 8 links touching the site
// are split among them; every thread keeps its links in registers for the
// whole update.  A backward link U_mu(x - mu) is held as X = U^dagger, so
// that M = sum_l X_l for all eight links and both updates
//     U_mu(x) <- g U_mu(x),  U_mu(x - mu) <- U_mu(x - mu) g^dagger
// become the same row rotation X <- g X.  Per SU(2) subgroup each thread
// projects its links' 2x2 blocks to a quaternion, the TPS partial sums are
// combined with xor shuffles (identical bits in every lane), every lane
// computes the same subgroup element, and rotates its own links.
#pragma once

#include "gf_device.cuh"
#include "gf_internal.h"

namespace gf {

// MODE_MAG: overrelaxation towards the maximally Abelian gauge (Sec. 6), the
// subgroup element from the 2x2 matrix H of add_mag_terms (per-subgroup form only)
enum Mode { MODE_OR = 0, MODE_SA = 1, MODE_SR = 2, MODE_MAG = 3 };

// ---------------------------------------------------------------------------
// accumulate form (one thread per site)
// ---------------------------------------------------------------------------
// Because every rotation acts on the rows of all eight held matrices X_l
// (U_mu(x) and U_mu(x-mu)^dagger), M = sum_l X_l transforms as M -> R M: the
// three subgroup steps of Alg. 1 can run on M alone while G = R3 R2 R1 is
// accumulated, and G is applied once per link at the end.  Same arithmetic
// result as the per-subgroup form in exact arithmetic; fewer operations, one
// thread per site, and the links are read a second time (from cache) instead
// of being held in registers.

// re-read of a stored link (volatile: not merged with the first read)
template <int FMT>
__device__ __forceinline__ void reload(const FieldRef &f, int pl0, int h, mat3<typename Store<FMT>::T> &u);

template <>
__device__ __forceinline__ void reload<F64_18>(const FieldRef &f, int pl0, int h, mat3<double> &u)
{
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const double2 *p = reinterpret_cast<const double2 *>(f.base + (pl0 + c) * f.plane_bytes) + h;
        double2 v;
        asm volatile("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
        u.e[c / 3][c % 3] = mk<double>(v.x, v.y);
    }
}

template <>
__device__ __forceinline__ void reload<F64_12>(const FieldRef &f, int pl0, int h, mat3<double> &u)
{
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const double2 *p = reinterpret_cast<const double2 *>(f.base + (pl0 + c) * f.plane_bytes) + h;
        double2 v;
        asm volatile("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
        u.e[c / 3][c % 3] = mk<double>(v.x, v.y);
    }
    rebuild_row2(u);
}

template <>
__device__ __forceinline__ void reload<F32_18>(const FieldRef &f, int pl0, int h, mat3<float> &u)
{
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float4 *p = reinterpret_cast<const float4 *>(f.base + (pl0 + c) * f.plane_bytes) + h;
        float4 v;
        asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
        int e0 = 2 * c, e1 = 2 * c + 1;
        u.e[e0 / 3][e0 % 3] = mk<float>(v.x, v.y);
        u.e[e1 / 3][e1 % 3] = mk<float>(v.z, v.w);
    }
    const float2 *p = reinterpret_cast<const float2 *>(f.base + (pl0 + 4) * f.plane_bytes) + h;
    float2 v;
    asm volatile("ld.global.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    u.e[2][2] = mk<float>(v.x, v.y);
}

template <>
__device__ __forceinline__ void reload<F32_12>(const FieldRef &f, int pl0, int h, mat3<float> &u)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float4 *p = reinterpret_cast<const float4 *>(f.base + (pl0 + c) * f.plane_bytes) + h;
        float4 v;
        asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
        int e0 = 2 * c, e1 = 2 * c + 1;
        u.e[e0 / 3][e0 % 3] = mk<float>(v.x, v.y);
        u.e[e1 / 3][e1 % 3] = mk<float>(v.z, v.w);
    }
    rebuild_row2(u);
}

template <>
__device__ __forceinline__ void reload<DF64_18>(const FieldRef &f, int pl0, int h, mat3<double> &u)
{
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const float4 *p = reinterpret_cast<const float4 *>(f.base + (pl0 + c) * f.plane_bytes) + h;
        float4 v;
        asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
        u.e[c / 3][c % 3] = mk<double>((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    }
}


// ---------------------------------------------------------------------------
// SU(2) subgroup element as R = [[alpha, beta], [-conj(beta), conj(alpha)]],
// alpha = r0 + i r3, beta = r2 + i r1 (the quaternion convention of rotate_rows)
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ cpx<T> cconj(cpx<T> z) { return mk<T>(z.re, -z.im); }
template <class T>
__device__ __forceinline__ cpx<T> cneg(cpx<T> z) { return mk<T>(-z.re, -z.im); }
template <class T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> x, cpx<T> y)
{
    return mk<T>(x.re * y.re - x.im * y.im, x.re * y.im + x.im * y.re);
}
// new row a: alpha x_a + beta x_b
template <class T>
__device__ __forceinline__ cpx<T> lin_a(cpx<T> al, cpx<T> be, cpx<T> xa, cpx<T> xb)
{
    return mk<T>(al.re * xa.re - al.im * xa.im + be.re * xb.re - be.im * xb.im,
                 al.re * xa.im + al.im * xa.re + be.re * xb.im + be.im * xb.re);
}
// new row b: -conj(beta) x_a + conj(alpha) x_b
template <class T>
__device__ __forceinline__ cpx<T> lin_b(cpx<T> al, cpx<T> be, cpx<T> xa, cpx<T> xb)
{
    return mk<T>(al.re * xb.re + al.im * xb.im - be.re * xa.re - be.im * xa.im,
                 al.re * xb.im - al.im * xb.re - be.re * xa.im + be.im * xa.re);
}

template <class T>
struct quat {
    T k[4];
};

// quaternion of the 2x2 block [[xaa, xab], [xba, xbb]] (see add_block_quaternion)
template <class T>
__device__ __forceinline__ quat<T> block_quaternion(cpx<T> xaa, cpx<T> xab, cpx<T> xba, cpx<T> xbb)
{
    quat<T> q;
    q.k[0] = xaa.re + xbb.re;
    q.k[1] = -(xab.im + xba.im);
    q.k[2] = xba.re - xab.re;
    q.k[3] = xbb.im - xaa.im;
    return q;
}

// the subgroup's new element from its quaternion k (overrelaxation, heatbath
// draw or stochastic relaxation); the identity when the step leaves it unchanged
template <int MODE, class T>
__device__ __forceinline__ void subgroup_element(const SweepArgs &a, quat<T> q, uint32_t site, int sg, cpx<T> &al,
                                                 cpx<T> &be)
{
    T r[4];
    bool ok;
    if (MODE == MODE_OR) {
        ok = overrelax_step(q.k, (T)a.omega, a.orv, r);
    } else if (MODE == MODE_SR) {
        ok = sr_quat(q.k, a.prob, site, a.sweep, sg, a.key, r);
    } else {
        double kd[4] = { (double)q.k[0], (double)q.k[1], (double)q.k[2], (double)q.k[3] };
        double rd[4];
        int st = heatbath_quat(kd, a.T, site, a.sweep, sg, a.cap, a.key, rd, GF_SA_TAG, a.sa_fp32 != 0);
        if (st == 0) atomicAdd(a.status, 1);
        ok = (st == 1);
#pragma unroll
        for (int i = 0; i < 4; ++i) r[i] = (T)rd[i];
    }
    if (!ok) {
        r[0] = T(1);
        r[1] = r[2] = r[3] = T(0);
    }
    al = mk<T>(r[0], r[3]);
    be = mk<T>(r[2], r[1]);
}

// rows 0 and 1 of a stored link, re-read (volatile); row 2 is left unset
template <int FMT>
__device__ __forceinline__ void reload_rows01(const FieldRef &f, int pl0, int h, mat3<typename Store<FMT>::T> &u);

template <>
__device__ __forceinline__ void reload_rows01<F64_18>(const FieldRef &f, int pl0, int h, mat3<double> &u)
{
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const double2 *p = reinterpret_cast<const double2 *>(f.base + (pl0 + c) * f.plane_bytes) + h;
        double2 v;
        asm volatile("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
        u.e[c / 3][c % 3] = mk<double>(v.x, v.y);
    }
}

template <>
__device__ __forceinline__ void reload_rows01<F64_12>(const FieldRef &f, int pl0, int h, mat3<double> &u)
{
    reload_rows01<F64_18>(f, pl0, h, u);  // the same first six chunks
}

template <>
__device__ __forceinline__ void reload_rows01<F32_18>(const FieldRef &f, int pl0, int h, mat3<float> &u)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float4 *p = reinterpret_cast<const float4 *>(f.base + (pl0 + c) * f.plane_bytes) + h;
        float4 v;
        asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
        int e0 = 2 * c, e1 = 2 * c + 1;
        u.e[e0 / 3][e0 % 3] = mk<float>(v.x, v.y);
        u.e[e1 / 3][e1 % 3] = mk<float>(v.z, v.w);
    }
}

template <>
__device__ __forceinline__ void reload_rows01<F32_12>(const FieldRef &f, int pl0, int h, mat3<float> &u)
{
    reload_rows01<F32_18>(f, pl0, h, u);  // the same first three chunks
}

template <>
__device__ __forceinline__ void reload_rows01<DF64_18>(const FieldRef &f, int pl0, int h, mat3<double> &u)
{
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const float4 *p = reinterpret_cast<const float4 *>(f.base + (pl0 + c) * f.plane_bytes) + h;
        float4 v;
        asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
        u.e[c / 3][c % 3] = mk<double>((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    }
}

// Products of 3x3 complex matrices, written as explicit FMA chains: an
// update "re += a*b - c*d" would round the difference first and cost an extra
// add per term.

// z = x y for 3x3 complex matrices; rows >= ROWS of z are not computed
template <class T, int ROWS>
__device__ __forceinline__ void mul_rows(const mat3<T> &x, const mat3<T> &y, mat3<T> &z)
{
#pragma unroll
    for (int a = 0; a < ROWS; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            T re = x.e[a][0].re * y.e[0][b].re;
            T im = x.e[a][0].re * y.e[0][b].im;
            re = fma(-x.e[a][0].im, y.e[0][b].im, re);
            im = fma(x.e[a][0].im, y.e[0][b].re, im);
#pragma unroll
            for (int c = 1; c < 3; ++c) {
                re = fma(x.e[a][c].re, y.e[c][b].re, re);
                re = fma(-x.e[a][c].im, y.e[c][b].im, re);
                im = fma(x.e[a][c].re, y.e[c][b].im, im);
                im = fma(x.e[a][c].im, y.e[c][b].re, im);
            }
            z.e[a][b] = mk<T>(re, im);
        }
}

// z = x y^dagger, rows >= ROWS of z not computed
template <class T, int ROWS>
__device__ __forceinline__ void mul_rows_dagger(const mat3<T> &x, const mat3<T> &y, mat3<T> &z)
{
#pragma unroll
    for (int a = 0; a < ROWS; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            // sum_c x[a][c] conj(y[b][c])
            T re = x.e[a][0].re * y.e[b][0].re;
            T im = x.e[a][0].im * y.e[b][0].re;
            re = fma(x.e[a][0].im, y.e[b][0].im, re);
            im = fma(-x.e[a][0].re, y.e[b][0].im, im);
#pragma unroll
            for (int c = 1; c < 3; ++c) {
                re = fma(x.e[a][c].re, y.e[b][c].re, re);
                re = fma(x.e[a][c].im, y.e[b][c].im, re);
                im = fma(x.e[a][c].im, y.e[b][c].re, im);
                im = fma(-x.e[a][c].re, y.e[b][c].im, im);
            }
            z.e[a][b] = mk<T>(re, im);
        }
}

// row 2 of z = x y
template <class T>
__device__ __forceinline__ void mul_row2(const mat3<T> &x, const mat3<T> &y, mat3<T> &z)
{
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        T re = x.e[2][0].re * y.e[0][b].re;
        T im = x.e[2][0].re * y.e[0][b].im;
        re = fma(-x.e[2][0].im, y.e[0][b].im, re);
        im = fma(x.e[2][0].im, y.e[0][b].re, im);
#pragma unroll
        for (int c = 1; c < 3; ++c) {
            re = fma(x.e[2][c].re, y.e[c][b].re, re);
            re = fma(-x.e[2][c].im, y.e[c][b].im, re);
            im = fma(x.e[2][c].re, y.e[c][b].im, im);
            im = fma(x.e[2][c].im, y.e[c][b].re, im);
        }
        z.e[2][b] = mk<T>(re, im);
    }
}

// how strongly G mixes row 2 with rows 0, 1: |G20|^2 + |G21|^2
template <class T>
__device__ __forceinline__ T row2_mixing(const mat3<T> &G)
{
    return G.e[2][0].re * G.e[2][0].re + G.e[2][0].im * G.e[2][0].im + G.e[2][1].re * G.e[2][1].re +
           G.e[2][1].im * G.e[2][1].im;
}

// below this mixing the third row of an 18-real link is rebuilt from rows 0, 1
// (error growth at most 1 + 1e-4 per update); above it, multiplied out
constexpr double kCrossRow2 = 1e-4;

// Gram-Schmidt of rows 0 and 1 (row 2 is implied by them in 12-real storage)
template <class T>
__device__ __forceinline__ void normalize_rows01(mat3<T> &u)
{
    T n0 = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) n0 += u.e[0][c].re * u.e[0][c].re + u.e[0][c].im * u.e[0][c].im;
    T i0 = rsqrt(n0);
#pragma unroll
    for (int c = 0; c < 3; ++c) u.e[0][c] = mk<T>(u.e[0][c].re * i0, u.e[0][c].im * i0);
    // row1 -= <row0, row1> row0
    T pre = T(0), pim = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        pre += u.e[0][c].re * u.e[1][c].re + u.e[0][c].im * u.e[1][c].im;
        pim += u.e[0][c].re * u.e[1][c].im - u.e[0][c].im * u.e[1][c].re;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        u.e[1][c] = mk<T>(u.e[1][c].re - (pre * u.e[0][c].re - pim * u.e[0][c].im),
                          u.e[1][c].im - (pre * u.e[0][c].im + pim * u.e[0][c].re));
    T n1 = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) n1 += u.e[1][c].re * u.e[1][c].re + u.e[1][c].im * u.e[1][c].im;
    T i1 = rsqrt(n1);
#pragma unroll
    for (int c = 0; c < 3; ++c) u.e[1][c] = mk<T>(u.e[1][c].re * i1, u.e[1][c].im * i1);
}

// U_mu(x) <- G U_mu(x), U_mu(x-mu) <- U_mu(x-mu) G^dagger for mu = 0..3, each
// link re-read; CROSS: rows 0, 1 multiplied out and row 2 = conj(row0 x row1)
// (the backward link re-read without its third row), else row 2 multiplied
// out too (18-real storage only)
template <int FMT, bool CROSS>
__device__ __forceinline__ void apply_links(const SweepArgs &a, int p, int h, const int hb[4],
                                            const mat3<typename Store<FMT>::T> &G)
{
    typedef Store<FMT> S;
    typedef typename S::T T;
    constexpr int ROWS = S::REALS == 12 ? 2 : 3;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        mat3<T> u, v;
        reload<FMT>(a.f, (p * 4 + mu) * S::NCHUNK, h, u);
        mul_rows<T, 2>(G, u, v);
        if (ROWS == 3) {
            if (CROSS) rebuild_row2(v);
            else mul_row2(G, u, v);
        }
        S::store(a.f, (p * 4 + mu) * S::NCHUNK, h, v);
        if (CROSS) {
            reload_rows01<FMT>(a.f, ((p ^ 1) * 4 + mu) * S::NCHUNK, hb[mu], u);
            mul_rows_dagger<T, 2>(u, G, v);
            if (ROWS == 3) rebuild_row2(v);
        } else {
            reload<FMT>(a.f, ((p ^ 1) * 4 + mu) * S::NCHUNK, hb[mu], u);
            mul_rows_dagger<T, ROWS>(u, G, v);
        }
        S::store(a.f, ((p ^ 1) * 4 + mu) * S::NCHUNK, hb[mu], v);
    }
}

template <int FMT, bool COULOMB, int MODE, bool TRACKG>
__device__ __forceinline__ void sweep_site_acc(const SweepArgs &a, int h)
{
    typedef Store<FMT> S;
    typedef typename S::T T;
    constexpr int ROWS = S::REALS == 12 ? 2 : 3;  // rows of a link that are stored
    const int p = a.parity;
    int c[4];
    site_coords(a.g, p, h, c);
    int hb[4];
    // M = sum over the gauge's directions of U_mu(x) + U_mu(x-mu)^dagger
    mat3<T> M;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M.e[i][j] = mk<T>(T(0), T(0));
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        hb[mu] = back_half(a.g, c, mu);
        if (COULOMB && mu == 3) continue;
        mat3<T> u;
        S::load(a.f, (p * 4 + mu) * S::NCHUNK, h, u);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                M.e[i][j].re += u.e[i][j].re;
                M.e[i][j].im += u.e[i][j].im;
            }
        S::load(a.f, ((p ^ 1) * 4 + mu) * S::NCHUNK, hb[mu], u);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                M.e[i][j].re += u.e[j][i].re;
                M.e[i][j].im -= u.e[j][i].im;
            }
    }
    const uint32_t site = (uint32_t)lex_index(a.g, c);
    // The three subgroups in Alg. 1 order, (0,1), (1,2), (0,2).  Of each rotated
    // M only the entries that the next subgroup's quaternion reads are formed:
    // R1 M rows 0 (cols 0, 2) and 1 (cols 0..2), then R2 R1 M row 2 (cols 0, 2).
    cpx<T> al[3], be[3];
    subgroup_element<MODE>(a, block_quaternion(M.e[0][0], M.e[0][1], M.e[1][0], M.e[1][1]), site, 0, al[0],
                           be[0]);
    const cpx<T> m00 = lin_a(al[0], be[0], M.e[0][0], M.e[1][0]);
    const cpx<T> m02 = lin_a(al[0], be[0], M.e[0][2], M.e[1][2]);
    const cpx<T> m10 = lin_b(al[0], be[0], M.e[0][0], M.e[1][0]);
    const cpx<T> m11 = lin_b(al[0], be[0], M.e[0][1], M.e[1][1]);
    const cpx<T> m12 = lin_b(al[0], be[0], M.e[0][2], M.e[1][2]);
    subgroup_element<MODE>(a, block_quaternion(m11, m12, M.e[2][1], M.e[2][2]), site, 1, al[1], be[1]);
    const cpx<T> n20 = lin_b(al[1], be[1], m10, M.e[2][0]);
    const cpx<T> n22 = lin_b(al[1], be[1], m12, M.e[2][2]);
    subgroup_element<MODE>(a, block_quaternion(m00, m02, n20, n22), site, 2, al[2], be[2]);
    // G = R3 R2 R1 in closed form (the zero pattern of the embedded factors
    // saves most of the three full row rotations)
    mat3<T> G;
    {
        const cpx<T> a1c = cconj(al[0]), b1c = cconj(be[0]), b2c = cconj(be[1]);
        const cpx<T> g20 = cmul(b2c, b1c), g21 = cneg(cmul(b2c, a1c)), g22 = cconj(al[1]);
        G.e[1][0] = cneg(cmul(al[1], b1c));
        G.e[1][1] = cmul(al[1], a1c);
        G.e[1][2] = be[1];
        G.e[0][0] = lin_a(al[2], be[2], al[0], g20);
        G.e[0][1] = lin_a(al[2], be[2], be[0], g21);
        G.e[0][2] = cmul(be[2], g22);
        G.e[2][0] = lin_b(al[2], be[2], al[0], g20);
        G.e[2][1] = lin_b(al[2], be[2], be[0], g21);
        G.e[2][2] = cmul(cconj(al[2]), g22);
    }
    // apply G: U_mu(x) <- G U_mu(x), U_mu(x-mu) <- U_mu(x-mu) G^dagger.  Rows 0, 1
    // are multiplied out.  Row 2 of an 18-real link: when G hardly mixes row 2
    // with rows 0, 1 (w = |G20|^2 + |G21|^2 below kCrossRow2, as near
    // convergence), conj(row0 x row1) -- the product's third row for SU(3)
    // factors (Sec. 4.1) at 2/3 of the cost, the backward link re-read without
    // its third row; otherwise the direct product, because the rebuilt row
    // feeds the unitarity error of rows 0, 1 back with gain up to 1 + w per
    // update (an unbounded growth under the large rotations of annealing).
    // the choice is made per warp (all its sites below the threshold), so that a
    // warp never runs both paths
    const bool cross = ROWS == 2 || __all_sync(__activemask(), row2_mixing(G) < T(kCrossRow2));
    if (cross) apply_links<FMT, true>(a, p, h, hb, G);
    else apply_links<FMT, false>(a, p, h, hb, G);
    if (TRACKG) {
        mat3<float> gx, gy;
        Store<F32_12>::load(a.gt, p * 3, h, gx);
        mat3<float> Gf;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Gf.e[i][j] = mk<float>((float)G.e[i][j].re, (float)G.e[i][j].im);
        mul_rows<float, 2>(Gf, gx, gy);
        normalize_rows01(gy);  // 12-real storage: keep the rebuilt third row from amplifying errors
        Store<F32_12>::store(a.gt, p * 3, h, gy);
    }
}

// mask of the TPS lanes that serve one site (all in the same warp)
template <int TPS>
__device__ __forceinline__ unsigned site_group_mask()
{
    const unsigned lane = threadIdx.x & 31u;
    return (TPS == 1) ? (1u << lane) : (((1u << TPS) - 1u) << (lane & ~(unsigned)(TPS - 1)));
}

// The update of half-site h of parity a.parity by lane j (0 <= j < TPS) of its
// site group: load the 8 links, three subgroup steps, store.
template <int FMT, int TPS, bool COULOMB, int MODE, bool TRACKG>
__device__ __forceinline__ void sweep_site(const SweepArgs &a, int h, int j, unsigned gmask)
{
    typedef Store<FMT> S;
    typedef typename S::T T;
    constexpr int NL = 8 / TPS;
    constexpr int HALF = (NL / 2 > 0) ? NL / 2 : 1;
    const int p = a.parity;

    int c[4];
    site_coords(a.g, p, h, c);

    mat3<T> x[NL];
    int hb[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const bool bwd = (TPS == 8) ? (j >= 4) : (l >= NL / 2);
        const int mu = (TPS == 8) ? (j & 3) : ((l % HALF) * TPS + j);
        if (!bwd) {
            hb[l] = h;
            S::load(a.f, (p * 4 + mu) * S::NCHUNK, h, x[l]);
        } else {
            hb[l] = back_half(a.g, c, mu);
            mat3<T> u;
            S::load(a.f, ((p ^ 1) * 4 + mu) * S::NCHUNK, hb[l], u);
            x[l] = dagger(u);
        }
    }

    mat3<float> gx;
    if (TRACKG && j == 0) Store<F32_12>::load(a.gt, p * 3, h, gx);

    const uint32_t site = (uint32_t)lex_index(a.g, c);

#pragma unroll
    for (int sg = 0; sg < 3; ++sg) {
        int ra, rb;
        subgroup_rows(sg, ra, rb);
        T k[4] = { T(0), T(0), T(0), T(0) };  // quaternion of K, or H of the MAG step
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const int mu = (TPS == 8) ? (j & 3) : ((l % HALF) * TPS + j);
            if (COULOMB && mu == 3) continue;  // Coulomb: K from spatial links only
            if (MODE == MODE_MAG) add_mag_terms(x[l], ra, rb, k);
            else add_block_quaternion(x[l], ra, rb, k);
        }
#pragma unroll
        for (int o = 1; o < TPS; o <<= 1)
#pragma unroll
            for (int i = 0; i < 4; ++i) k[i] += __shfl_xor_sync(gmask, k[i], o);

        T r[4];
        bool ok;
        if (MODE == MODE_MAG) {
            T rm[4];
            ok = mag_element(k, rm) && overrelax_step(rm, (T)a.omega, a.orv, r);
        } else if (MODE == MODE_OR) {
            ok = overrelax_step(k, (T)a.omega, a.orv, r);
        } else if (MODE == MODE_SR) {
            ok = sr_quat(k, a.prob, site, a.sweep, sg, a.key, r);
        } else {
            double kd[4] = { (double)k[0], (double)k[1], (double)k[2], (double)k[3] };
            double rd[4];
            int st = heatbath_quat(kd, a.T, site, a.sweep, sg, a.cap, a.key, rd, GF_SA_TAG, a.sa_fp32 != 0);
            if (st == 0 && j == 0) atomicAdd(a.status, 1);
            ok = (st == 1);
#pragma unroll
            for (int i = 0; i < 4; ++i) r[i] = (T)rd[i];
        }
        if (ok) {
#pragma unroll
            for (int l = 0; l < NL; ++l) rotate_rows(x[l], ra, rb, r);
            if (TRACKG && j == 0) {
                float rf[4] = { (float)r[0], (float)r[1], (float)r[2], (float)r[3] };
                rotate_rows(gx, ra, rb, rf);
            }
        }
    }

#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const bool bwd = (TPS == 8) ? (j >= 4) : (l >= NL / 2);
        const int mu = (TPS == 8) ? (j & 3) : ((l % HALF) * TPS + j);
        if (!bwd)
            S::store(a.f, (p * 4 + mu) * S::NCHUNK, h, x[l]);
        else
            S::store(a.f, ((p ^ 1) * 4 + mu) * S::NCHUNK, hb[l], dagger(x[l]));
    }
    if (TRACKG && j == 0) {
        normalize_rows01(gx);
        Store<F32_12>::store(a.gt, p * 3, h, gx);
    }
}

template <int FMT, bool COULOMB, int MODE, bool TRACKG>
__global__ void __launch_bounds__(256) k_sweep_acc(SweepArgs a)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= a.g.Vh) return;
    sweep_site_acc<FMT, COULOMB, MODE, TRACKG>(a, h);
}

// the same with a register budget (the autotuner tries both for FP64
// storage): RC = 1: 168 per thread (3 blocks of 128 threads per SM), RC = 2:
// 128 (2 blocks of 256)
template <int FMT, bool COULOMB, int MODE, bool TRACKG, int RC>
__global__ void __launch_bounds__(RC == 1 ? 128 : 256, RC == 1 ? 3 : 2) k_sweep_acc_rc(SweepArgs a)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= a.g.Vh) return;
    sweep_site_acc<FMT, COULOMB, MODE, TRACKG>(a, h);
}

template <int FMT, int TPS, bool COULOMB, int MODE, bool TRACKG>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs a)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int h = tid / TPS;
    const int j = tid & (TPS - 1);
    if (h >= a.g.Vh) return;
    sweep_site<FMT, TPS, COULOMB, MODE, TRACKG>(a, h, j, site_group_mask<TPS>());
}

// TPS <= 0 selects the accumulate form (one thread per site) with register
// budget RC = -TPS (GF_ACC, GF_ACC_R168, GF_ACC_R128)
template <int FMT, int TPS, bool COULOMB, int MODE, bool TRACKG>
static cudaError_t launch_k_sweep(const SweepArgs &a, int block, cudaStream_t s)
{
    long threads = (long)a.g.Vh * (TPS <= 0 ? 1 : TPS);
    int grid = (int)((threads + block - 1) / block);
    if (TPS == GF_ACC_R168 && block > 128) return cudaErrorInvalidValue;
    if constexpr (MODE == MODE_MAG && TPS <= 0) {
        return cudaErrorInvalidValue;  // the MAG step needs the links: per-subgroup form only
    } else {
        if (TPS == 0) k_sweep_acc<FMT, COULOMB, MODE, TRACKG><<<grid, block, 0, s>>>(a);
        else if (TPS < 0) k_sweep_acc_rc<FMT, COULOMB, MODE, TRACKG, (TPS < 0 ? -TPS : 1)><<<grid, block, 0, s>>>(a);
        else k_sweep<FMT, (TPS <= 0 ? 1 : TPS), COULOMB, MODE, TRACKG><<<grid, block, 0, s>>>(a);
        return cudaGetLastError();
    }
}

template <int FMT, int TPS, bool TRACKG>
static cudaError_t dispatch_gauge_mode(const SweepArgs &a, int coulomb, int mode, int block, cudaStream_t s)
{
    if (mode == MODE_OR) {
        return coulomb ? launch_k_sweep<FMT, TPS, true, MODE_OR, TRACKG>(a, block, s)
                       : launch_k_sweep<FMT, TPS, false, MODE_OR, TRACKG>(a, block, s);
    }
    if (mode == MODE_MAG) {
        if constexpr (FMT == DF64_18) {
            return cudaErrorInvalidValue;
        } else {
            if (coulomb) return cudaErrorInvalidValue;
            return launch_k_sweep<FMT, TPS, false, MODE_MAG, TRACKG>(a, block, s);
        }
    }
    if (TRACKG) return cudaErrorInvalidValue;  // annealing and stochastic relaxation never track g
    if (mode == MODE_SR)
        return coulomb ? launch_k_sweep<FMT, TPS, true, MODE_SR, false>(a, block, s)
                       : launch_k_sweep<FMT, TPS, false, MODE_SR, false>(a, block, s);
    return coulomb ? launch_k_sweep<FMT, TPS, true, MODE_SA, false>(a, block, s)
                   : launch_k_sweep<FMT, TPS, false, MODE_SA, false>(a, block, s);
}

template <int FMT, bool TRACKG>
static cudaError_t dispatch_tps(const SweepArgs &a, int tps, int coulomb, int mode, int block, cudaStream_t s)
{
    switch (tps) {
    case GF_ACC_R168:
        if constexpr (FMT == F64_18 || FMT == F64_12)
            return dispatch_gauge_mode<FMT, GF_ACC_R168, TRACKG>(a, coulomb, mode, block, s);
        return cudaErrorInvalidValue;
    case GF_ACC_R128:
        if constexpr (FMT == F64_18 || FMT == F64_12)
            return dispatch_gauge_mode<FMT, GF_ACC_R128, TRACKG>(a, coulomb, mode, block, s);
        return cudaErrorInvalidValue;
    case 0: return dispatch_gauge_mode<FMT, 0, TRACKG>(a, coulomb, mode, block, s);
    case 1: return dispatch_gauge_mode<FMT, 1, TRACKG>(a, coulomb, mode, block, s);
    case 2: return dispatch_gauge_mode<FMT, 2, TRACKG>(a, coulomb, mode, block, s);
    case 4: return dispatch_gauge_mode<FMT, 4, TRACKG>(a, coulomb, mode, block, s);
    case 8: return dispatch_gauge_mode<FMT, 8, TRACKG>(a, coulomb, mode, block, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gf
