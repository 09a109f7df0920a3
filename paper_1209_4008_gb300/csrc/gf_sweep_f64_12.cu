// Half-sweep kernels (overrelaxation and heatbath) for F64_12 link storage.
#include "gf_sweep.cuh"

namespace gf {

cudaError_t launch_sweep_f64_12(const SweepArgs &a, int tps, int coulomb, int mode, bool trackg, int block,
                              cudaStream_t s)
{
    return trackg ? dispatch_tps<F64_12, true>(a, tps, coulomb, mode, block, s)
                  : dispatch_tps<F64_12, false>(a, tps, coulomb, mode, block, s);
}

}  // namespace gf
