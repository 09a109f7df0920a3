// gf_sweep_df64.cuh -- the double-float site update (DF64_18 storage): the
// accumulate form of gf_sweep.cuh (M = sum of the eight links, three subgroup
// steps on M with G = R3 R2 R1 accumulated, G applied once per link) with M,
// G and the link products in double-float arithmetic on the FP32 pipe; only
// the scalar step of each subgroup (quaternion k to the SU(2) element r) runs
// in FP64.  Used by the single-lattice kernels (gf_sweep_df64.cu) and by the
// batched persistent kernel (gf_batch.cu).
#pragma once

#include "gf_df64.cuh"
#include "gf_sweep.cuh"

namespace gf {


__device__ __forceinline__ cdf cdf_conj(cdf z)
{
    z.im = df_neg(z.im);
    return z;
}

__device__ __forceinline__ cdf cdf_neg(cdf z)
{
    z.re = df_neg(z.re);
    z.im = df_neg(z.im);
    return z;
}

__device__ __forceinline__ cdf cdf_mul(cdf x, cdf y)
{
    cdf r;
    r.re = df_sub(df_mul(x.re, y.re), df_mul(x.im, y.im));
    r.im = df_add(df_mul(x.re, y.im), df_mul(x.im, y.re));
    return r;
}

// alpha x_a + beta x_b (new row a of an SU(2) rotation)
__device__ __forceinline__ cdf lin_a_df(cdf al, cdf be, cdf xa, cdf xb)
{
    cdf p = cdf_mul(al, xa), q = cdf_mul(be, xb);
    p.re = df_add(p.re, q.re);
    p.im = df_add(p.im, q.im);
    return p;
}

// -conj(beta) x_a + conj(alpha) x_b (new row b)
__device__ __forceinline__ cdf lin_b_df(cdf al, cdf be, cdf xa, cdf xb)
{
    cdf p = cdf_mul(cdf_conj(al), xb), q = cdf_mul(cdf_conj(be), xa);
    p.re = df_sub(p.re, q.re);
    p.im = df_sub(p.im, q.im);
    return p;
}

// conj(a d - b c), each component one double-float dot product of four terms
__device__ __forceinline__ cdf conj_cross_df(cdf a, cdf d, cdf b, cdf c)
{
    dacc re = { 0.f, 0.f }, im = { 0.f, 0.f };
    dacc_add_prod(re, a.re, d.re);
    dacc_add_prod(re, df_neg(a.im), d.im);
    dacc_add_prod(re, df_neg(b.re), c.re);
    dacc_add_prod(re, b.im, c.im);
    dacc_add_prod(im, df_neg(a.re), d.im);  // the imaginary part of a d - b c, negated
    dacc_add_prod(im, df_neg(a.im), d.re);
    dacc_add_prod(im, b.re, c.im);
    dacc_add_prod(im, b.im, c.re);
    cdf r;
    r.re = dacc_result(re);
    r.im = dacc_result(im);
    return r;
}

// third row of an SU(3) link from its first two rows, stored
__device__ __forceinline__ void store_row2_df(const FieldRef &f, int pl0, int h, const cdf v[2][3])
{
    store_chunk_df(f, pl0 + 6, h, conj_cross_df(v[0][1], v[1][2], v[0][2], v[1][1]));
    store_chunk_df(f, pl0 + 7, h, conj_cross_df(v[0][2], v[1][0], v[0][0], v[1][2]));
    store_chunk_df(f, pl0 + 8, h, conj_cross_df(v[0][0], v[1][1], v[0][1], v[1][0]));
}

// subgroup element from the 2x2 block [[xaa, xab], [xba, xbb]]: the quaternion
// in FP64, the scalar step in FP64 (overrelaxation, stochastic choice or
// heatbath draw), the result as R = [[alpha, beta], [-conj(beta), conj(alpha)]]
template <int MODE>
__device__ __forceinline__ void subgroup_element_df(const SweepArgs &a, cdf xaa, cdf xab, cdf xba, cdf xbb,
                                                    uint32_t site, int sg, cdf &al, cdf &be)
{
    double k[4];
    k[0] = df_to_double(df_add(xaa.re, xbb.re));
    k[1] = -df_to_double(df_add(xab.im, xba.im));
    k[2] = df_to_double(df_sub(xba.re, xab.re));
    k[3] = df_to_double(df_sub(xbb.im, xaa.im));
    double rd[4];
    bool ok;
    if (MODE == MODE_OR) {
        ok = overrelax_step(k, a.omega, a.orv, rd);
    } else if (MODE == MODE_SR) {
        ok = sr_quat(k, a.prob, site, a.sweep, sg, a.key, rd);
    } else {
        int st = heatbath_quat(k, a.T, site, a.sweep, sg, a.cap, a.key, rd, GF_SA_TAG, a.sa_fp32 != 0);
        if (st == 0) atomicAdd(a.status, 1);
        ok = (st == 1);
    }
    if (!ok) {
        rd[0] = 1.0;
        rd[1] = rd[2] = rd[3] = 0.0;
    }
    al.re = df_from_double(rd[0]);
    al.im = df_from_double(rd[3]);
    be.re = df_from_double(rd[2]);
    be.im = df_from_double(rd[1]);
}

// U_mu(x) <- G U_mu(x) (one column of U at a time) and U_mu(x-mu) <- U_mu(x-mu)
// G^dagger (one row at a time) for mu = 0..3.  Rows 0 and 1 are multiplied
// out; row 2 is rebuilt as conj(row0 x row1) when cross is set, else
// multiplied out as well.  cross is uniform in a warp, and both ways share one
// loop body: two full copies of this loop overflow the instruction cache of the
// double-float kernels (most of their stalls were instruction fetches).
__device__ __forceinline__ void apply_links_df(const SweepArgs &a, int p, int h, const int hb[4], const mat3df &G,
                                               bool cross)
{
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
        const int pf = (p * 4 + mu) * 9, pb = ((p ^ 1) * 4 + mu) * 9;
        cdf v[2][3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cdf col[3];
#pragma unroll
            for (int l = 0; l < 3; ++l) col[l] = reload_chunk_df(a.f, pf + 3 * l + j, h);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                v[i][j] = cdf_dot3<false>(G.e[i], col);
                store_chunk_df(a.f, pf + 3 * i + j, h, v[i][j]);
            }
            if (!cross) store_chunk_df(a.f, pf + 6 + j, h, cdf_dot3<false>(G.e[2], col));
        }
        if (cross) store_row2_df(a.f, pf, h, v);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            cdf row[3];
#pragma unroll
            for (int l = 0; l < 3; ++l) row[l] = reload_chunk_df(a.f, pb + 3 * i + l, hb[mu]);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                v[i][j] = cdf_dot3<true>(row, G.e[j]);
                store_chunk_df(a.f, pb + 3 * i + j, hb[mu], v[i][j]);
            }
        }
        if (cross) {
            store_row2_df(a.f, pb, hb[mu], v);
        } else {
            cdf row[3];
#pragma unroll
            for (int l = 0; l < 3; ++l) row[l] = reload_chunk_df(a.f, pb + 6 + l, hb[mu]);
#pragma unroll
            for (int j = 0; j < 3; ++j) store_chunk_df(a.f, pb + 6 + j, hb[mu], cdf_dot3<true>(row, G.e[j]));
        }
    }
}

// Prefetch of this thread's E (9 chunks of 16 bytes) into shared memory with
// cp.async at the start of the site update, so that the load latency hides
// behind the update itself; slot c of thread t at epre[c * nthreads + t].
__device__ __forceinline__ void prefetch_e_df(const SweepArgs &a, int p, int h, float4 *epre, int t, int nthreads)
{
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const float4 *src = reinterpret_cast<const float4 *>(a.ge.base + (size_t)(p * 9 + c) * a.ge.plane_bytes) + h;
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(epre + c * nthreads + t);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// g <- G g for the gauge transformation tracked as E = g - 1 in double-float
// (a DF64_18 site field, planes p * 9 + c): E <- (G - 1) + G E.  E stays small
// where g is close to the identity, so its double-float rounding is relative
// to |g - 1|, not to |g| = 1; g = 1 + E is applied to an FP64 field in FP64
// afterwards (k_apply_gauge_e).
// epre: this thread's prefetched E (prefetch_e_df), or nullptr to read E from
// global memory.  One column of E at a time (12 floats live besides G).
__device__ __forceinline__ void track_e_df(const SweepArgs &a, int p, int h, const mat3df &G,
                                           const float4 *epre = nullptr, int t = 0, int nthreads = 0)
{
    if (epre) asm volatile("cp.async.wait_all;" ::: "memory");
    // rolled over the columns: the site-update kernels are large enough that
    // code size (instruction-cache misses) matters more than the loop overhead
#pragma unroll 1
    for (int j = 0; j < 3; ++j) {
        cdf col[3];
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const int c = 3 * l + j;
            if (epre) {
                const float4 v = epre[c * nthreads + t];
                col[l].re = df_make(v.x, v.y);
                col[l].im = df_make(v.z, v.w);
            } else {
                col[l] = reload_chunk_df(a.ge, p * 9 + c, h);
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            cdf s = cdf_dot3<false>(G.e[i], col);
            // (G - 1)_ij without a dynamically indexed register array
            cdf d = j == 0 ? G.e[i][0] : (j == 1 ? G.e[i][1] : G.e[i][2]);
            if (i == j) d.re = df_sub(d.re, df_make(1.f, 0.f));
            s.re = df_add(s.re, d.re);
            s.im = df_add(s.im, d.im);
            store_chunk_df(a.ge, p * 9 + 3 * i + j, h, s);
        }
    }
}

template <bool COULOMB, int MODE, bool TRACKG, bool TRACKE = false>
__device__ __forceinline__ void sweep_site_df(const SweepArgs &a, int h, const float4 *epre = nullptr, int t = 0,
                                              int nthreads = 0)
{
    const int p = a.parity;
    int c[4];
    site_coords(a.g, p, h, c);
    int hb[4];
    mat3df M;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M.e[i][j] = cdf_zero();
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        hb[mu] = back_half(a.g, c, mu);
        if (COULOMB && mu == 3) continue;
        mat3df u;
        load_df(a.f, (p * 4 + mu) * 9, h, u);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                M.e[i][j].re = df_add(M.e[i][j].re, u.e[i][j].re);
                M.e[i][j].im = df_add(M.e[i][j].im, u.e[i][j].im);
            }
        load_df(a.f, ((p ^ 1) * 4 + mu) * 9, hb[mu], u);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {  // + U^dagger
                M.e[i][j].re = df_add(M.e[i][j].re, u.e[j][i].re);
                M.e[i][j].im = df_sub(M.e[i][j].im, u.e[j][i].im);
            }
    }
    const uint32_t site = (uint32_t)lex_index(a.g, c);
    // subgroups (0,1), (1,2), (0,2) as in the FP64 accumulate form: only the
    // entries of the rotated M that the next quaternion reads are formed
    cdf al[3], be[3];
    subgroup_element_df<MODE>(a, M.e[0][0], M.e[0][1], M.e[1][0], M.e[1][1], site, 0, al[0], be[0]);
    const cdf m00 = lin_a_df(al[0], be[0], M.e[0][0], M.e[1][0]);
    const cdf m02 = lin_a_df(al[0], be[0], M.e[0][2], M.e[1][2]);
    const cdf m10 = lin_b_df(al[0], be[0], M.e[0][0], M.e[1][0]);
    const cdf m11 = lin_b_df(al[0], be[0], M.e[0][1], M.e[1][1]);
    const cdf m12 = lin_b_df(al[0], be[0], M.e[0][2], M.e[1][2]);
    subgroup_element_df<MODE>(a, m11, m12, M.e[2][1], M.e[2][2], site, 1, al[1], be[1]);
    const cdf n20 = lin_b_df(al[1], be[1], m10, M.e[2][0]);
    const cdf n22 = lin_b_df(al[1], be[1], m12, M.e[2][2]);
    subgroup_element_df<MODE>(a, m00, m02, n20, n22, site, 2, al[2], be[2]);
    // G = R3 R2 R1 in closed form
    mat3df G;
    {
        const cdf a1c = cdf_conj(al[0]), b1c = cdf_conj(be[0]), b2c = cdf_conj(be[1]);
        const cdf g20 = cdf_mul(b2c, b1c), g21 = cdf_neg(cdf_mul(b2c, a1c)), g22 = cdf_conj(al[1]);
        G.e[1][0] = cdf_neg(cdf_mul(al[1], b1c));
        G.e[1][1] = cdf_mul(al[1], a1c);
        G.e[1][2] = be[1];
        G.e[0][0] = lin_a_df(al[2], be[2], al[0], g20);
        G.e[0][1] = lin_a_df(al[2], be[2], be[0], g21);
        G.e[0][2] = cdf_mul(be[2], g22);
        G.e[2][0] = lin_b_df(al[2], be[2], al[0], g20);
        G.e[2][1] = lin_b_df(al[2], be[2], be[0], g21);
        G.e[2][2] = cdf_mul(cdf_conj(al[2]), g22);
    }
    // U_mu(x) <- G U_mu(x) and U_mu(x-mu) <- U_mu(x-mu) G^dagger: rows 0, 1
    // multiplied out (forward: one column of U at a time; backward: one row);
    // row 2 = conj(row0 x row1) when G hardly mixes row 2 (as in the FP64
    // accumulate form, kCrossRow2), else multiplied out as well
    const float w = G.e[2][0].re.hi * G.e[2][0].re.hi + G.e[2][0].im.hi * G.e[2][0].im.hi +
                    G.e[2][1].re.hi * G.e[2][1].re.hi + G.e[2][1].im.hi * G.e[2][1].im.hi;
    apply_links_df(a, p, h, hb, G, __all_sync(__activemask(), w < (float)kCrossRow2));  // per warp
    if (TRACKE) track_e_df(a, p, h, G, epre, t, nthreads);
    if (TRACKG) {
        mat3<float> gx, gy, Gf;
        Store<F32_12>::load(a.gt, p * 3, h, gx);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                Gf.e[i][j] = mk<float>(G.e[i][j].re.hi + G.e[i][j].re.lo, G.e[i][j].im.hi + G.e[i][j].im.lo);
        mul_rows<float, 2>(Gf, gx, gy);
        normalize_rows01(gy);
        Store<F32_12>::store(a.gt, p * 3, h, gy);
    }
}

}  // namespace gf
