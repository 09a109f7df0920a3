// Half-sweep kernels for DF64_18 storage (FP64-class values as FP32 pairs).
//
// The site update is the accumulate form of gf_sweep.cuh (M = sum of the
// eight links, three subgroup steps on M with G = R3 R2 R1 accumulated, G
// applied once per link), with M, G and the link products in double-float
// arithmetic on the FP32 pipe.  Only the scalar step of each subgroup --
// the quaternion k to the SU(2) element r (overrelaxation exponent or heatbath
// draw) -- runs in FP64, a few dozen FP64 operations per site instead of the
// ~1500 of an FP64 site update.
#include "gf_sweep_df64.cuh"

namespace gf {

// Occupancy matters more than registers here (long dependent chains of
// double-float operations): at most 96 registers for overrelaxation and
// stochastic relaxation (five blocks of at most 128 threads per SM; the
// E-tracked half-sweep ran 6 % faster than with 128 registers), 128 for the
// heatbath, which spills around its draw at 96.
constexpr int kDfBlockMax = 128;
template <bool COULOMB, int MODE, bool TRACKG, bool TRACKE = false>
__global__ void __launch_bounds__(MODE == MODE_SA ? 256 : kDfBlockMax, MODE == MODE_SA ? 2 : 5)
    k_sweep_df(SweepArgs a)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= a.g.Vh) return;
    if (TRACKE) {  // E arrives in shared memory while the site update runs (9 x 16 bytes per thread)
        extern __shared__ float4 epre[];
        prefetch_e_df(a, a.parity, h, epre, threadIdx.x, blockDim.x);
        sweep_site_df<COULOMB, MODE, TRACKG, TRACKE>(a, h, epre, threadIdx.x, blockDim.x);
    } else {
        sweep_site_df<COULOMB, MODE, TRACKG, TRACKE>(a, h);
    }
}

// overrelaxation or heatbath with E = g - 1 tracked in double-float (a.ge)
static cudaError_t launch_df_e(const SweepArgs &a, int coulomb, int mode, int block, cudaStream_t s)
{
    if (mode != MODE_SA && block > kDfBlockMax) block = kDfBlockMax;
    int grid = (a.g.Vh + block - 1) / block;
    const size_t smem = 9 * sizeof(float4) * (size_t)block;  // prefetched E, at most 36 KiB
    if (mode == MODE_OR) {
        if (coulomb) k_sweep_df<true, MODE_OR, false, true><<<grid, block, smem, s>>>(a);
        else k_sweep_df<false, MODE_OR, false, true><<<grid, block, smem, s>>>(a);
    } else if (mode == MODE_SA) {
        if (coulomb) k_sweep_df<true, MODE_SA, false, true><<<grid, block, smem, s>>>(a);
        else k_sweep_df<false, MODE_SA, false, true><<<grid, block, smem, s>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <bool TRACKG>
static cudaError_t launch_df(const SweepArgs &a, int coulomb, int mode, int block, cudaStream_t s)
{
    if (mode != MODE_SA && block > kDfBlockMax) block = kDfBlockMax;
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
    if (mode == MODE_MAG) return cudaErrorInvalidValue;  // maximally Abelian gauge: native storage only
    // tracking E = g - 1 (a.ge set): the double-float accumulate kernel whatever tps says
    if (trackg && a.ge.base) return launch_df_e(a, coulomb, mode, block, s);
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
