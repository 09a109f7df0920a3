// gf_internal.h -- declarations shared by the library's translation units
// (kernel launchers per storage format, codec/reduction launchers).  Not part
// of the public ABI (that is include/gf.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gf_device.cuh"

namespace gf {

// launch-configuration codes of the site update ("threads per site"):
// 1, 2, 4, 8 = per-subgroup form with that many threads per site; <= 0 =
// accumulate form, one thread per site, with a register budget of 255, 168 or
// 128 per thread (the last two for FP64 storage only)
constexpr int GF_ACC = 0, GF_ACC_R168 = -1, GF_ACC_R128 = -2;

// arguments of one half-sweep launch
struct SweepArgs {
    FieldRef f;       // resident field
    FieldRef gt;      // accumulated gauge transformation (F32_12 site field) or {0}
    FieldRef ge;      // double-float sweeps: E = g - 1 of the applied transformation (DF64_18 site field) or {0}
    Geom g;
    int parity;
    double omega;     // overrelaxation exponent
    int orv;          // reading of g -> g^omega: 0 rational 19-flop form, 1 first order, 2 exact power
    double T;         // heatbath temperature
    uint2 key;        // Philox key (seed)
    uint32_t sweep;   // Philox sweep counter
    int cap;          // heatbath rejection cap
    int sa_fp32;      // heatbath: 1 = the FP32 reading of the draw
    double prob;      // stochastic relaxation: probability of the microcanonical step
    int *status;      // [0]: heatbath draws that hit the cap
};

// half-sweep launchers, one per storage format (gf_sweep_*.cu)
cudaError_t launch_sweep_f64_18(const SweepArgs &a, int tps, int coulomb, int mode, bool trackg, int block,
                                cudaStream_t s);
cudaError_t launch_sweep_f64_12(const SweepArgs &a, int tps, int coulomb, int mode, bool trackg, int block,
                                cudaStream_t s);
cudaError_t launch_sweep_f32_18(const SweepArgs &a, int tps, int coulomb, int mode, bool trackg, int block,
                                cudaStream_t s);
cudaError_t launch_sweep_f32_12(const SweepArgs &a, int tps, int coulomb, int mode, bool trackg, int block,
                                cudaStream_t s);
cudaError_t launch_sweep_df64(const SweepArgs &a, int tps, int coulomb, int mode, bool trackg, int block,
                              cudaStream_t s);

inline cudaError_t launch_sweep(int fmt, const SweepArgs &a, int tps, int coulomb, int mode, bool trackg, int block,
                                cudaStream_t s)
{
    switch (fmt) {
    case F64_18: return launch_sweep_f64_18(a, tps, coulomb, mode, trackg, block, s);
    case F64_12: return launch_sweep_f64_12(a, tps, coulomb, mode, trackg, block, s);
    case F32_18: return launch_sweep_f32_18(a, tps, coulomb, mode, trackg, block, s);
    case F32_12: return launch_sweep_f32_12(a, tps, coulomb, mode, trackg, block, s);
    case DF64_18: return launch_sweep_df64(a, tps, coulomb, mode, trackg, block, s);
    default: return cudaErrorInvalidValue;
    }
}

inline int format_chunks(int fmt)
{
    switch (fmt) {
    case F64_18: return 9;
    case F64_12: return 6;
    case F32_18: return 5;
    case F32_12: return 3;
    case DF64_18: return 9;
    default: return 0;
    }
}

// bytes moved per site update by one half-sweep (8 links read + 8 written)
inline double format_link_bytes(int fmt)
{
    switch (fmt) {
    case F64_18: return 144.0;
    case F64_12: return 96.0;
    case F32_18: return 72.0;
    case F32_12: return 48.0;
    case DF64_18: return 144.0;
    default: return 0.0;
    }
}

// Where a caller's pointer lives, for entry points that take host or device
// memory: PTR_HOST (pageable or pinned host memory, or memory CUDA does not
// know), PTR_DEVICE (device memory of the current device, or managed memory),
// PTR_FOREIGN (device memory of another device: kernels launched on the
// current device must not dereference it).
enum PtrKind { PTR_HOST = 0, PTR_DEVICE = 1, PTR_FOREIGN = 2 };

inline PtrKind pointer_kind(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // this query's own error only
        return PTR_HOST;
    }
    if (a.type == cudaMemoryTypeManaged) return PTR_DEVICE;
    if (a.type != cudaMemoryTypeDevice) return PTR_HOST;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PTR_FOREIGN;
    }
    return a.device == dev ? PTR_DEVICE : PTR_FOREIGN;
}

// reductions write per-block partial sums (2 doubles per block)
constexpr int kReduceBlock = 256;

// codec, reductions and transforms (gf_field.cu)
cudaError_t launch_encode(int fmt, const double *aos, FieldRef f, const Geom &g, cudaStream_t s);
cudaError_t launch_decode(int fmt, FieldRef f, const Geom &g, double *aos, cudaStream_t s);
cudaError_t launch_reunitarize(int fmt, FieldRef f, const Geom &g, cudaStream_t s);
cudaError_t launch_widen(int src_fmt, FieldRef src, int dst_fmt, FieldRef dst, const Geom &g, cudaStream_t s);
// FP64-class field -> FP32 field (reunitarised in FP64, then rounded)
cudaError_t launch_narrow(int src_fmt, FieldRef src, int dst_fmt, FieldRef dst, const Geom &g, cudaStream_t s);
cudaError_t launch_gauge_identity(FieldRef gt, const Geom &g, cudaStream_t s);
cudaError_t launch_apply_tracked_gauge(const double *aos, FieldRef gt, int dst_fmt, FieldRef dst, const Geom &g,
                                       cudaStream_t s);
// F and theta of the resident field: nblocks partials, then the final sum
// Wilson-action update of the links U_mu(x), x of one parity (mode 0 heatbath, 1 overrelaxation;
// FP64 storage); heatbath draws that hit the cap are counted in *status
cudaError_t launch_wilson(int fmt, FieldRef f, const Geom &g, int mu, int parity, double beta, int mode, uint2 key,
                          uint32_t sweep, int cap, int *status, cudaStream_t s);

int measure_blocks(const Geom &g);
int slice_blocks(const Geom &g);  // blocks per timeslice of launch_measure_slices
// F_t, theta_t of every timeslice into slices[2 Lt]; out[0] = mean F_t, out[1] = max theta_t
cudaError_t launch_measure_slices(int fmt, FieldRef f, const Geom &g, int coulomb, double *partials,
                                  double *slices, double *out, cudaStream_t s);
cudaError_t launch_measure(int fmt, FieldRef f, const Geom &g, int coulomb, double *partials, double *out,
                           cudaStream_t s);
// F and theta of a canonical (AoS) field
int aos_blocks(const Geom &g);
cudaError_t launch_measure_aos(const double *aos, const Geom &g, int coulomb, double *partials, double *out,
                               cudaStream_t s);
cudaError_t launch_plaquette_aos(const double *aos, const Geom &g, double *partials, double *out, cudaStream_t s);

// learned warm start, field side (gf_learned.cu)
cudaError_t launch_features(int fmt, FieldRef f, const Geom &g, double inv_scale, void *out, cudaStream_t s);
cudaError_t launch_gauge_algebra(FieldRef gt, const Geom &g, double inv_scale, float *out, cudaStream_t s);
cudaError_t launch_expmap_to_gauge(const float *c, double scale, FieldRef gt, const Geom &g, cudaStream_t s);
cudaError_t launch_gauge_transform_resident(int fmt, FieldRef f, FieldRef gt, const Geom &g, cudaStream_t s);
cudaError_t launch_decode_gauge(FieldRef gt, const Geom &g, double *out, cudaStream_t s);
// FP64 field (F64_18 / F64_12) -> double-float working copy (DF64_18)
cudaError_t launch_to_df(int src_fmt, FieldRef src, FieldRef dst, const Geom &g, cudaStream_t s);
// FP64 field := g(x) U_mu(x) g(x+mu)^dagger with g = 1 + E (E a DF64_18 site
// field), reunitarised in FP64
cudaError_t launch_apply_gauge_e(int fmt, FieldRef f, FieldRef ge, const Geom &g, cudaStream_t s);

}  // namespace gf
