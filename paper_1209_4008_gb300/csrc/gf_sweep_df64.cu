// Half-sweep kernels for DF64_18 storage (FP64-class values as FP32 pairs).
//
// The site update is the accumulate form of gf_sweep.cuh (M = sum of the
// eight links, three subgroup steps on M with G = R3 R2 R1 accumulated, G
// applied once per link), with M, G and the link products in double-float
// arithmetic on the FP32 pipe.  Only the scalar step of each subgroup --
// the quaternion k to the SU(2) element r (overrelaxation exponent or heatbath
// draw) -- runs in FP64, a few dozen FP64 operations per site instead of the
// ~1500 of an FP64 site update.
#include "gf_df64.cuh"
#include "gf_sweep.cuh"

namespace gf {

// rows a, b of x <- R (rows a, b), R the SU(2) element r (quaternion)
__device__ __forceinline__ void rotate_rows_df(mat3df &x, int a, int b, const df r[4])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cdf xa = x.e[a][c], xb = x.e[b][c];
        x.e[a][c].re = df_add(df_sub(df_mul(r[0], xa.re), df_mul(r[3], xa.im)),
                              df_sub(df_mul(r[2], xb.re), df_mul(r[1], xb.im)));
        x.e[a][c].im = df_add(df_add(df_mul(r[0], xa.im), df_mul(r[3], xa.re)),
                              df_add(df_mul(r[2], xb.im), df_mul(r[1], xb.re)));
        x.e[b][c].re = df_sub(df_add(df_mul(r[0], xb.re), df_mul(r[3], xb.im)),
                              df_add(df_mul(r[2], xa.re), df_mul(r[1], xa.im)));
        x.e[b][c].im = df_add(df_sub(df_mul(r[0], xb.im), df_mul(r[3], xb.re)),
                              df_sub(df_mul(r[1], xa.re), df_mul(r[2], xa.im)));
    }
}

template <bool COULOMB, int MODE, bool TRACKG>
__device__ __forceinline__ void sweep_site_df(const SweepArgs &a, int h)
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
    mat3df G;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            G.e[i][j] = cdf_zero();
            if (i == j) G.e[i][j].re = df_make(1.f, 0.f);
        }
#pragma unroll
    for (int sg = 0; sg < 3; ++sg) {
        int ra, rb;
        subgroup_rows(sg, ra, rb);
        // quaternion of the (ra, rb) block of M (see add_block_quaternion)
        double k[4];
        k[0] = df_to_double(df_add(M.e[ra][ra].re, M.e[rb][rb].re));
        k[1] = -df_to_double(df_add(M.e[ra][rb].im, M.e[rb][ra].im));
        k[2] = df_to_double(df_sub(M.e[rb][ra].re, M.e[ra][rb].re));
        k[3] = df_to_double(df_sub(M.e[rb][rb].im, M.e[ra][ra].im));
        double rd[4];
        bool ok;
        if (MODE == MODE_OR) {
            ok = overrelax_quat(k, a.omega, rd);
        } else if (MODE == MODE_SR) {
            ok = sr_quat(k, a.prob, site, a.sweep, sg, a.key, rd);
        } else {
            int st = heatbath_quat(k, a.T, site, a.sweep, sg, a.cap, a.key, rd);
            if (st == 0) atomicAdd(a.status, 1);
            ok = (st == 1);
        }
        if (ok) {
            df r[4] = { df_from_double(rd[0]), df_from_double(rd[1]), df_from_double(rd[2]), df_from_double(rd[3]) };
            rotate_rows_df(M, ra, rb, r);
            rotate_rows_df(G, ra, rb, r);
        }
    }
    // U_mu(x) <- G U_mu(x): one column of U at a time, each output chunk stored
    // as soon as it is formed (few live registers);
    // U_mu(x-mu) <- U_mu(x-mu) G^dagger: one row of U at a time
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
        const int pf = (p * 4 + mu) * 9, pb = ((p ^ 1) * 4 + mu) * 9;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cdf col[3];
#pragma unroll
            for (int l = 0; l < 3; ++l) col[l] = reload_chunk_df(a.f, pf + 3 * l + j, h);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                cdf s = cdf_zero();
#pragma unroll
                for (int l = 0; l < 3; ++l) s = cdf_mac(s, G.e[i][l], col[l]);
                store_chunk_df(a.f, pf + 3 * i + j, h, s);
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            cdf row[3];
#pragma unroll
            for (int l = 0; l < 3; ++l) row[l] = reload_chunk_df(a.f, pb + 3 * i + l, hb[mu]);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                cdf s = cdf_zero();
#pragma unroll
                for (int l = 0; l < 3; ++l) s = cdf_mac_conj(s, row[l], G.e[j][l]);
                store_chunk_df(a.f, pb + 3 * i + j, hb[mu], s);
            }
        }
    }
    if (TRACKG) {
        mat3<float> gx, gy, Gf;
        Store<F32_12>::load(a.gt, p * 3, h, gx);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                Gf.e[i][j] = mk<float>(G.e[i][j].re.hi + G.e[i][j].re.lo, G.e[i][j].im.hi + G.e[i][j].im.lo);
        mul_rows<float, 2>(Gf, gx, gy);
        Store<F32_12>::store(a.gt, p * 3, h, gy);
    }
}

// at most 128 registers: occupancy matters more than registers here (long
// dependent chains of double-float operations)
template <bool COULOMB, int MODE, bool TRACKG>
__global__ void __launch_bounds__(256, 2) k_sweep_df(SweepArgs a)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= a.g.Vh) return;
    sweep_site_df<COULOMB, MODE, TRACKG>(a, h);
}

template <bool TRACKG>
static cudaError_t launch_df(const SweepArgs &a, int coulomb, int mode, int block, cudaStream_t s)
{
    int grid = (a.g.Vh + block - 1) / block;
    if (mode == MODE_OR) {
        if (coulomb) k_sweep_df<true, MODE_OR, TRACKG><<<grid, block, 0, s>>>(a);
        else k_sweep_df<false, MODE_OR, TRACKG><<<grid, block, 0, s>>>(a);
    } else if (mode == MODE_SR) {
        if (TRACKG) return cudaErrorInvalidValue;
        if (coulomb) k_sweep_df<true, MODE_SR, false><<<grid, block, 0, s>>>(a);
        else k_sweep_df<false, MODE_SR, false><<<grid, block, 0, s>>>(a);
    } else {
        if (TRACKG) return cudaErrorInvalidValue;
        if (coulomb) k_sweep_df<true, MODE_SA, false><<<grid, block, 0, s>>>(a);
        else k_sweep_df<false, MODE_SA, false><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// threads per site 0: the double-float accumulate kernel above; 1, 2, 4, 8:
// the per-subgroup kernels on the FP64 view of the same storage
cudaError_t launch_sweep_df64(const SweepArgs &a, int tps, int coulomb, int mode, bool trackg, int block,
                              cudaStream_t s)
{
    if (tps == 0) return trackg ? launch_df<true>(a, coulomb, mode, block, s) : launch_df<false>(a, coulomb, mode, block, s);
    switch (tps) {
    case 1: return trackg ? dispatch_gauge_mode<DF64_18, 1, true>(a, coulomb, mode, block, s)
                          : dispatch_gauge_mode<DF64_18, 1, false>(a, coulomb, mode, block, s);
    case 2: return trackg ? dispatch_gauge_mode<DF64_18, 2, true>(a, coulomb, mode, block, s)
                          : dispatch_gauge_mode<DF64_18, 2, false>(a, coulomb, mode, block, s);
    case 4: return trackg ? dispatch_gauge_mode<DF64_18, 4, true>(a, coulomb, mode, block, s)
                          : dispatch_gauge_mode<DF64_18, 4, false>(a, coulomb, mode, block, s);
    case 8: return trackg ? dispatch_gauge_mode<DF64_18, 8, true>(a, coulomb, mode, block, s)
                          : dispatch_gauge_mode<DF64_18, 8, false>(a, coulomb, mode, block, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gf
