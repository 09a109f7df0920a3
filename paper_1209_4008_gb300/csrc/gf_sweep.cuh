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

enum Mode { MODE_OR = 0, MODE_SA = 1 };

template <int FMT, int TPS, bool COULOMB, int MODE, bool TRACKG>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs a)
{
    typedef Store<FMT> S;
    typedef typename S::T T;
    constexpr int NL = 8 / TPS;
    constexpr int HALF = (NL / 2 > 0) ? NL / 2 : 1;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int h = tid / TPS;
    const int j = tid & (TPS - 1);
    if (h >= a.g.Vh) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned gmask = (TPS == 1) ? (1u << lane) : (((1u << TPS) - 1u) << (lane & ~(unsigned)(TPS - 1)));
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
        T k[4] = { T(0), T(0), T(0), T(0) };
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const int mu = (TPS == 8) ? (j & 3) : ((l % HALF) * TPS + j);
            if (COULOMB && mu == 3) continue;  // Coulomb: K from spatial links only
            add_block_quaternion(x[l], ra, rb, k);
        }
#pragma unroll
        for (int o = 1; o < TPS; o <<= 1)
#pragma unroll
            for (int i = 0; i < 4; ++i) k[i] += __shfl_xor_sync(gmask, k[i], o);

        T r[4];
        bool ok;
        if (MODE == MODE_OR) {
            ok = overrelax_quat(k, (T)a.omega, r);
        } else {
            double kd[4] = { (double)k[0], (double)k[1], (double)k[2], (double)k[3] };
            double rd[4];
            int st = heatbath_quat(kd, a.T, site, a.sweep, sg, a.cap, a.key, rd);
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
    if (TRACKG && j == 0) Store<F32_12>::store(a.gt, p * 3, h, gx);
}

template <int FMT, int TPS, bool COULOMB, int MODE, bool TRACKG>
static cudaError_t launch_k_sweep(const SweepArgs &a, int block, cudaStream_t s)
{
    long threads = (long)a.g.Vh * TPS;
    int grid = (int)((threads + block - 1) / block);
    k_sweep<FMT, TPS, COULOMB, MODE, TRACKG><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int FMT, int TPS, bool TRACKG>
static cudaError_t dispatch_gauge_mode(const SweepArgs &a, int coulomb, int mode, int block, cudaStream_t s)
{
    if (mode == MODE_OR) {
        return coulomb ? launch_k_sweep<FMT, TPS, true, MODE_OR, TRACKG>(a, block, s)
                       : launch_k_sweep<FMT, TPS, false, MODE_OR, TRACKG>(a, block, s);
    }
    if (TRACKG) return cudaErrorInvalidValue;  // annealing never tracks g
    return coulomb ? launch_k_sweep<FMT, TPS, true, MODE_SA, false>(a, block, s)
                   : launch_k_sweep<FMT, TPS, false, MODE_SA, false>(a, block, s);
}

template <int FMT, bool TRACKG>
static cudaError_t dispatch_tps(const SweepArgs &a, int tps, int coulomb, int mode, int block, cudaStream_t s)
{
    switch (tps) {
    case 1: return dispatch_gauge_mode<FMT, 1, TRACKG>(a, coulomb, mode, block, s);
    case 2: return dispatch_gauge_mode<FMT, 2, TRACKG>(a, coulomb, mode, block, s);
    case 4: return dispatch_gauge_mode<FMT, 4, TRACKG>(a, coulomb, mode, block, s);
    case 8: return dispatch_gauge_mode<FMT, 8, TRACKG>(a, coulomb, mode, block, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gf
