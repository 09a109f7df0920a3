// gf_wilson.cu -- gauge-field generation with the Wilson action, to give the
// gauge fixing thermalised inputs like the paper's ensembles (Sec. 5).
//
// S = beta sum_P (1 - Re tr U_P / 3).  The link U = U_mu(x) enters S through
// -(beta/3) Re tr(U A), A the sum of its six staples.  Cabibbo-Marinari: for
// each SU(2) subgroup the link is multiplied from the left by R, and
// Re tr(R U A) = r.k with k the quaternion of the subgroup block of W = U A;
// the heatbath draws r with weight exp((beta/3) r.k) -- the SU(2) draw of the
// annealing at T = 3/beta, Philox counter (4 x + mu, sweep, 256 subgroup +
// draw, 3) -- and the overrelaxation step is the microcanonical r = (k/|k|)^2,
// which keeps Re tr(U A).  One launch updates every link U_mu(x) of one
// direction and one parity (they share no staple); one thread per link.
#include "gf_fieldops.cuh"
#include "gf_internal.h"

namespace gf {

#define GF_WILSON_TAG 3u

// coordinates of x + d mu (periodic), MU a compile-time direction
template <int MU>
__device__ __forceinline__ void shift_coords(const Geom &g, const int c[4], int d, int out[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = c[k];
    int v = c[MU] + d;
    const int L = g.L[MU];
    out[MU] = v < 0 ? v + L : (v >= L ? v - L : v);
}

template <int FMT, int MU>
__global__ void __launch_bounds__(128) k_wilson(FieldRef f, Geom g, int parity, double beta, int mode, uint2 key,
                                                uint32_t sweep, int cap, int *status)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    constexpr int NC = Store<FMT>::NCHUNK;
    const int p = parity, q = parity ^ 1;
    int c[4];
    site_coords(g, p, h, c);
    int cp[4];
    shift_coords<MU>(g, c, 1, cp);
    mat3<double> A;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) A.e[a][b] = mk<double>(0.0, 0.0);
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == MU) continue;
        int cn[4], cm[4], cpm[4];
        // (shift along the compile-time nu of the unrolled loop)
        if (nu == 0) {
            shift_coords<0>(g, c, 1, cn);
            shift_coords<0>(g, c, -1, cm);
            shift_coords<0>(g, cp, -1, cpm);
        } else if (nu == 1) {
            shift_coords<1>(g, c, 1, cn);
            shift_coords<1>(g, c, -1, cm);
            shift_coords<1>(g, cp, -1, cpm);
        } else if (nu == 2) {
            shift_coords<2>(g, c, 1, cn);
            shift_coords<2>(g, c, -1, cm);
            shift_coords<2>(g, cp, -1, cpm);
        } else {
            shift_coords<3>(g, c, 1, cn);
            shift_coords<3>(g, c, -1, cm);
            shift_coords<3>(g, cp, -1, cpm);
        }
        // upper staple U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
        const mat3<double> ua = load_d<FMT>(f, (q * 4 + nu) * NC, lex_index(g, cp) >> 1);
        const mat3<double> ub = load_d<FMT>(f, (q * 4 + MU) * NC, lex_index(g, cn) >> 1);
        const mat3<double> uc = load_d<FMT>(f, (p * 4 + nu) * NC, h);
        const mat3<double> up = mul3(mul3(ua, dagger(ub)), dagger(uc));
        // lower staple U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)
        const mat3<double> ud = load_d<FMT>(f, (p * 4 + nu) * NC, lex_index(g, cpm) >> 1);
        const mat3<double> ue = load_d<FMT>(f, (q * 4 + MU) * NC, lex_index(g, cm) >> 1);
        const mat3<double> uf = load_d<FMT>(f, (q * 4 + nu) * NC, lex_index(g, cm) >> 1);
        const mat3<double> lo = mul3(mul3(dagger(ud), dagger(ue)), uf);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                A.e[a][b] = mk<double>(A.e[a][b].re + (up.e[a][b].re + lo.e[a][b].re),
                                       A.e[a][b].im + (up.e[a][b].im + lo.e[a][b].im));
    }
    mat3<double> u = load_d<FMT>(f, (p * 4 + MU) * NC, h);
    mat3<double> W = mul3(u, A);
    const uint32_t site = 4u * (uint32_t)lex_index(g, c) + (uint32_t)MU;
#pragma unroll
    for (int sg = 0; sg < 3; ++sg) {
        int ra, rb;
        subgroup_rows(sg, ra, rb);
        double k[4] = { 0.0, 0.0, 0.0, 0.0 };
        add_block_quaternion(W, ra, rb, k);
        double r[4];
        bool ok;
        if (mode == 0) {
            const int st = heatbath_quat(k, 3.0 / beta, site, sweep, sg, cap, key, r, GF_WILSON_TAG);
            if (st == 0) atomicAdd(status, 1);
            ok = st == 1;
        } else {  // microcanonical: the square of the relaxation element
            const double n = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2] + k[3] * k[3]);
            ok = n > 0.0;
            if (ok) {
                const double h0 = k[0] / n;
                r[0] = 2.0 * h0 * h0 - 1.0;
#pragma unroll
                for (int i = 1; i < 4; ++i) r[i] = 2.0 * h0 * (k[i] / n);
            }
        }
        if (ok) {
            rotate_rows(u, ra, rb, r);
            rotate_rows(W, ra, rb, r);
        }
    }
    store_d<FMT>(f, (p * 4 + MU) * NC, h, u);
}

template <int FMT>
static cudaError_t launch_wilson_fmt(FieldRef f, const Geom &g, int mu, int parity, double beta, int mode,
                                     uint2 key, uint32_t sweep, int cap, int *status, cudaStream_t s)
{
    const int grid = (g.Vh + 127) / 128;
    switch (mu) {
    case 0: k_wilson<FMT, 0><<<grid, 128, 0, s>>>(f, g, parity, beta, mode, key, sweep, cap, status); break;
    case 1: k_wilson<FMT, 1><<<grid, 128, 0, s>>>(f, g, parity, beta, mode, key, sweep, cap, status); break;
    case 2: k_wilson<FMT, 2><<<grid, 128, 0, s>>>(f, g, parity, beta, mode, key, sweep, cap, status); break;
    case 3: k_wilson<FMT, 3><<<grid, 128, 0, s>>>(f, g, parity, beta, mode, key, sweep, cap, status); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_wilson(int fmt, FieldRef f, const Geom &g, int mu, int parity, double beta, int mode, uint2 key,
                          uint32_t sweep, int cap, int *status, cudaStream_t s)
{
    if (fmt == F64_18) return launch_wilson_fmt<F64_18>(f, g, mu, parity, beta, mode, key, sweep, cap, status, s);
    if (fmt == F64_12) return launch_wilson_fmt<F64_12>(f, g, mu, parity, beta, mode, key, sweep, cap, status, s);
    return cudaErrorInvalidValue;  // generation runs on FP64 storage
}

}  // namespace gf
