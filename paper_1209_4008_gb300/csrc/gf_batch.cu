// gf_batch.cu -- many independent lattices of uneven volume gauge-fixed in
// one persistent cooperative launch per precision phase.
//
// All configurations live in one arena (each in its own per-parity SoA
// block).  A configuration's half-sites are cut into tiles of
// (blockDim / threads-per-site) sites; the tiles of all configurations form
// one work list.  The persistent kernel walks that list with a grid stride and
// separates the phases of Alg. 1 with a grid-wide barrier:
//   [reunitarise (FP32)] -> measure tiles -> per-configuration F, theta and
//   convergence decision -> check_every x (RED, BLACK) half-sweeps -> ...
// so convergence is decided on the device and the whole solve of a phase is
// a single launch.  Converged configurations drop out of the work list.
// Every barrier wait is bounded by a %globaltimer limit; on expiry the kernel
// records GF_ETIMEOUT in a status word and every block returns.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "gf.h"
#include "gf_fieldops.cuh"
#include "gf_sweep.cuh"
#include "gf_sweep_df64.cuh"

using namespace gf;

namespace gf {

struct BatchConfig {
    Geom g;
    size_t off32, off64, offg;  // byte offsets of this configuration's fields in the arenas
    size_t offdf, offe;         // double-float working copy and its E = g - 1 site field
    int tile0;                  // first tile of this configuration (per parity)
    int ntiles;                 // tiles per parity
    int nk;                     // directions in F and theta
    int pad;
};

struct BatchArgs {
    const BatchConfig *cfg;
    const int *tile_cfg;  // tile -> configuration
    int ncfg;
    int ntiles;           // tiles per parity (all configurations)
    char *arena;          // field arena of the phase's precision
    char *garena;         // gauge-tracking arena (FP32-12 site fields)
    char *earena;         // double-float phase: E = g - 1 arena (DF64_18 site fields)
    int kind;             // arena offsets: 0 off32 (FP32), 1 off64 (FP64), 2 offdf (double-float copy)
    double omega;
    double target;
    int check_every;
    const int *max_iter;  // per configuration sweep budget of this phase
    int *conv;            // per configuration: 1 = done
    int *sweeps;          // per configuration sweeps done in this phase
    double *F;            // per configuration, last measurement
    double *theta;
    double *tile_partials;  // 2 doubles per (parity, tile)
    unsigned *bar;          // [0] arrival count, [1] generation
    int *status;
    long long timeout_ns;
    unsigned expected_blocks;  // blocks that must arrive at a barrier (gridDim.x)
    int reunit;                // reunitarise links (and g) at every check
};

__device__ __forceinline__ long long globaltimer_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with a bounded wait.  Returns false (in every thread of
// the block) once any block has recorded an error.
__device__ bool grid_barrier(const BatchArgs &b)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = b.bar + 1;
        unsigned gen = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(b.bar, 1u);
        if (arrived == b.expected_blocks - 1) {
            atomicExch(b.bar, 0u);
            __threadfence();
            atomicAdd(b.bar + 1, 1u);
        } else {
            long long t0 = globaltimer_ns();
            while (*vgen == gen) {
                if (globaltimer_ns() - t0 > b.timeout_ns) {
                    atomicCAS(b.status, 0, GF_ETIMEOUT);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        s_ok = (*(volatile int *)b.status == 0);
    }
    __syncthreads();
    return s_ok != 0;
}

template <int FMT>
__device__ __forceinline__ FieldRef field_of(const BatchArgs &b, const BatchConfig &c)
{
    return FieldRef{ b.arena + (b.kind == 2 ? c.offdf : (b.kind == 1 ? c.off64 : c.off32)), (size_t)c.g.plane * 16 };
}

__device__ __forceinline__ FieldRef gauge_of(const BatchArgs &b, const BatchConfig &c)
{
    return FieldRef{ b.garena + c.offg, (size_t)c.g.plane * 16 };
}

// TPS == 0: the accumulate form of the site update (one thread per site)
template <int FMT, int TPS, bool COULOMB, bool TRACKG>
__global__ void __launch_bounds__(256) k_batch_persistent(BatchArgs b)
{
    constexpr int TP = TPS == 0 ? 1 : TPS;
    const int spt = blockDim.x / TP;  // sites per tile
    const int j = threadIdx.x & (TP - 1);
    const int ls = threadIdx.x / TP;
    const unsigned gmask = site_group_mask<TP>();
    __shared__ double red[2];
    __shared__ int s_active;

    for (;;) {
        // 0. reunitarise the links (and g) of active configurations
        if (b.reunit) {
            for (int w = blockIdx.x; w < 2 * b.ntiles; w += gridDim.x) {
                int p = w >= b.ntiles ? 1 : 0, t = w - p * b.ntiles;
                const BatchConfig c = b.cfg[b.tile_cfg[t]];
                if (b.conv[b.tile_cfg[t]]) continue;
                int h = (t - c.tile0) * spt + ls;
                if (j != 0 || h >= c.g.Vh) continue;
                FieldRef f = field_of<FMT>(b, c);
                for (int mu = 0; mu < 4; ++mu) {
                    mat3<double> u = load_d<FMT>(f, (p * 4 + mu) * Store<FMT>::NCHUNK, h);
                    reunitarize3(u);
                    store_d<FMT>(f, (p * 4 + mu) * Store<FMT>::NCHUNK, h, u);
                }
                if (TRACKG) {
                    FieldRef gt = gauge_of(b, c);
                    mat3<double> u = load_d<F32_12>(gt, p * 3, h);
                    reunitarize3(u);
                    store_d<F32_12>(gt, p * 3, h, u);
                }
            }
            if (!grid_barrier(b)) return;
        }
        // 1. measure every tile (both parities) of active configurations
        for (int w = blockIdx.x; w < 2 * b.ntiles; w += gridDim.x) {
            int p = w >= b.ntiles ? 1 : 0, t = w - p * b.ntiles;
            int ci = b.tile_cfg[t];
            double fs = 0.0, ts = 0.0;
            if (!b.conv[ci]) {
                const BatchConfig c = b.cfg[ci];
                int h = (t - c.tile0) * spt + ls;
                if (j == 0 && h < c.g.Vh) {
                    if (c.nk == 3) measure_site<FMT, true>(field_of<FMT>(b, c), c.g, p, h, fs, ts);
                    else measure_site<FMT, false>(field_of<FMT>(b, c), c.g, p, h, fs, ts);
                }
            }
            block_sum2(fs, ts, red);
            __syncthreads();
            if (threadIdx.x == 0) {
                b.tile_partials[2 * w] = red[0];
                b.tile_partials[2 * w + 1] = red[1];
            }
            __syncthreads();
        }
        if (!grid_barrier(b)) return;
        // 2. per-configuration sums in a fixed order, convergence decision
        for (int ci = blockIdx.x; ci < b.ncfg; ci += gridDim.x) {
            if (b.conv[ci]) continue;  // uniform in the block
            const BatchConfig c = b.cfg[ci];
            double fs = 0.0, ts = 0.0;
            for (int k = threadIdx.x; k < 2 * c.ntiles; k += blockDim.x) {
                int p = k >= c.ntiles ? 1 : 0, t = c.tile0 + k - p * c.ntiles;
                int w = p * b.ntiles + t;
                fs += b.tile_partials[2 * w];
                ts += b.tile_partials[2 * w + 1];
            }
            block_sum2(fs, ts, red);
            __syncthreads();
            if (threadIdx.x == 0) {
                double V = 2.0 * c.g.Vh;
                double F = red[0] / (3.0 * c.nk * V), th = red[1] / (3.0 * V);
                b.F[ci] = F;
                b.theta[ci] = th;
                if (th < b.target || b.sweeps[ci] >= b.max_iter[ci] || !(th == th)) b.conv[ci] = 1;
            }
            __syncthreads();
        }
        if (!grid_barrier(b)) return;
        // 3. stop when every configuration is done
        if (threadIdx.x == 0) {
            int a = 0;
            for (int ci = 0; ci < b.ncfg; ++ci) a += b.conv[ci] ? 0 : 1;
            s_active = a;
        }
        __syncthreads();
        if (s_active == 0) return;
        // 4. check_every sweeps (each configuration limited by its budget)
        for (int s = 0; s < b.check_every; ++s) {
            for (int p = 0; p < 2; ++p) {
                for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
                    int ci = b.tile_cfg[t];
                    if (b.conv[ci] || b.sweeps[ci] + s >= b.max_iter[ci]) continue;
                    const BatchConfig c = b.cfg[ci];
                    int h = (t - c.tile0) * spt + ls;
                    if (h >= c.g.Vh) continue;
                    SweepArgs a;
                    memset(&a, 0, sizeof a);
                    a.f = field_of<FMT>(b, c);
                    a.gt = gauge_of(b, c);
                    a.g = c.g;
                    a.parity = p;
                    a.omega = b.omega;
                    a.orv = 0;  // the rational 19-flop form
                    a.T = 1.0;
                    a.key = make_uint2(0u, 0u);
                    a.sweep = 0;
                    a.cap = 1;
                    a.status = b.status;
                    if constexpr (FMT == DF64_18) {
                        // double-float copy of an FP64 field: the transformation is tracked as E = g - 1,
                        // prefetched into shared memory while the site update runs
                        extern __shared__ float4 epre[];
                        a.ge = FieldRef{ b.earena + c.offe, (size_t)c.g.plane * 16 };
                        prefetch_e_df(a, p, h, epre, threadIdx.x, blockDim.x);
                        if (c.nk == 3) sweep_site_df<true, MODE_OR, false, true>(a, h, epre, threadIdx.x, blockDim.x);
                        else sweep_site_df<false, MODE_OR, false, true>(a, h, epre, threadIdx.x, blockDim.x);
                    } else if (TPS == 0) {
                        if (c.nk == 3) sweep_site_acc<FMT, true, MODE_OR, TRACKG>(a, h);
                        else sweep_site_acc<FMT, false, MODE_OR, TRACKG>(a, h);
                    } else {
                        if (c.nk == 3) sweep_site<FMT, TP, true, MODE_OR, TRACKG>(a, h, j, gmask);
                        else sweep_site<FMT, TP, false, MODE_OR, TRACKG>(a, h, j, gmask);
                    }
                }
                if (!grid_barrier(b)) return;
            }
        }
        // 5. account the sweeps (read by step 2 only after the next barriers)
        if (blockIdx.x == 0) {
            for (int ci = threadIdx.x; ci < b.ncfg; ci += blockDim.x) {
                if (b.conv[ci]) continue;
                int n = b.max_iter[ci] - b.sweeps[ci];
                b.sweeps[ci] += n < b.check_every ? n : b.check_every;
            }
        }
    }
}

// Between the phases of the mixed policy: remember the FP32 sweeps, give each
// configuration the rest of its budget and clear the convergence flags.
__global__ void k_batch_next_phase(int n, int max_iter, int *conv, int *sweeps, int *maxit, int *sweeps32)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    sweeps32[i] = sweeps[i];
    maxit[i] = max_iter - sweeps[i];
    sweeps[i] = 0;
    conv[i] = 0;
}

// Between the double-float phase and the native FP64 one: remember the
// double-float sweeps, give each configuration the rest of its budget and
// clear the convergence flags.
__global__ void k_batch_after_df(int n, int *conv, int *sweeps, int *maxit, int *sweepsdf)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    sweepsdf[i] = sweeps[i];
    maxit[i] -= sweeps[i];
    sweeps[i] = 0;
    conv[i] = 0;
}

__global__ void k_batch_first_phase(int n, int max_iter, int *conv, int *sweeps, int *maxit, int *sweeps32,
                                    int *sweepsdf, int *status, unsigned *bar)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        maxit[i] = max_iter;
        sweeps[i] = 0;
        sweeps32[i] = 0;
        conv[i] = 0;
        sweepsdf[i] = 0;
    }
    if (i == 0) {
        *status = 0;
        bar[0] = 0;
        bar[1] = 0;
    }
}

// identity gauge fields / apply tracked gauge / encode / decode for one configuration
// reuse the single-lattice launchers (gf_internal.h).

}  // namespace gf

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

template <int FMT, int TPS, bool TRACKG>
void *persistent_kernel_ptr(bool coulomb)
{
    (void)coulomb;
    return (void *)k_batch_persistent<FMT, TPS, false, TRACKG>;
}

// Coulomb and Landau configurations share one kernel: the per-configuration
// nk selects the gauge inside (the COULOMB template argument of the kernel is
// unused; it is kept false).
void *kernel_for(int fmt, int tps, bool trackg)
{
#define GF_K(F, T)                                                                \
    if (fmt == F && tps == T) {                                                   \
        return trackg ? persistent_kernel_ptr<F, T, true>(false)                  \
                      : persistent_kernel_ptr<F, T, false>(false);                \
    }
    GF_K(F32_12, 0) GF_K(F32_12, 1) GF_K(F32_12, 2) GF_K(F32_12, 4) GF_K(F32_12, 8)
    GF_K(F32_18, 0) GF_K(F32_18, 1) GF_K(F32_18, 2) GF_K(F32_18, 4) GF_K(F32_18, 8)
#undef GF_K
    if (fmt == DF64_18 && tps == 0 && !trackg) return persistent_kernel_ptr<DF64_18, 0, false>(false);
#define GF_K64(F, T) \
    if (fmt == F && tps == T && !trackg) return persistent_kernel_ptr<F, T, false>(false);
    GF_K64(F64_18, 0) GF_K64(F64_18, 1) GF_K64(F64_18, 2) GF_K64(F64_18, 4) GF_K64(F64_18, 8)
    GF_K64(F64_12, 0) GF_K64(F64_12, 1) GF_K64(F64_12, 2) GF_K64(F64_12, 4) GF_K64(F64_12, 8)
#undef GF_K64
    return nullptr;
}

std::mutex g_batch_tune_mutex;
std::map<std::tuple<std::vector<int>, int, int>, std::pair<int, int>> g_batch_tune;  // (dims, fmt, gauge)

}  // namespace

struct gf_batch {
    int n = 0;
    int gauge = 0;
    std::vector<int> dims;  // 4n
    std::vector<Geom> geom;
    long total_sites = 0;
    // options
    int precision = GF_MIXED;
    int storage32 = 12, storage64 = 18;
    int check_every = 25;
    double theta_switch = 1e-6;
    int tps = 0, block = 0;
    int fp64_arith = 0;  // 1: FP64 phase as double-float sweeps on copies, E tracked, applied in FP64
    double timeout_ms = 2000.0;
    int extra_blocks = 0;  // test hook: a barrier that can never complete
    cudaStream_t stream = nullptr;
    // device memory
    char *a32 = nullptr, *a64 = nullptr, *ag = nullptr, *adf = nullptr, *ae = nullptr;
    size_t a32_bytes = 0, a64_bytes = 0, ag_bytes = 0, adf_bytes = 0, ae_bytes = 0;
    BatchConfig *dcfg = nullptr;
    int *dtile = nullptr;
    int tiles_spt = 0;  // sites per tile the tile table was built for
    int ntiles = 0;
    double *partials = nullptr;
    int *dint = nullptr;     // conv[n], sweeps[n], maxit[n], sweeps32[n], status, pad, bar[2], sweepsdf[n]
    double *ddbl = nullptr;  // F[n], theta[n]
    int *hint = nullptr;
    double *hdbl = nullptr;
    std::vector<BatchConfig> cfg;
    int use_graphs = 1;
    int skip_decode = 0;  // autotuning: leave the caller's fields untouched
    int tps64_override = 0, block64_override = 0;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev[3] = { nullptr, nullptr, nullptr };
    cudaGraphExec_t graph = nullptr;
    std::string graph_key;
    std::map<std::string, double> stats;
    std::string err;
};

static int bfail(gf_batch *b, int code, const std::string &m)
{
    b->err = m;
    return code;
}

static int bcuda(gf_batch *b, cudaError_t e, const char *what)
{
    cudaGetLastError();  // do not leave the error for the next runtime call to report
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return bfail(b, e == cudaErrorMemoryAllocation ? GF_ENOMEM : GF_ECUDA, buf);
}

#define BCK(call)                                              \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return bcuda(b, e_, #call);     \
    } while (0)

#define BRET(call)                  \
    do {                            \
        int r_ = (call);            \
        if (r_ != GF_OK) return r_; \
    } while (0)

static int bfmt32(const gf_batch *b) { return b->storage32 == 18 ? F32_18 : F32_12; }
static int bfmt64(const gf_batch *b) { return b->storage64 == 12 ? F64_12 : F64_18; }

static std::pair<int, int> batch_config(const gf_batch *b, int fmt)
{
    std::pair<int, int> cfg = fmt == F32_12 ? std::make_pair(1, 128) : std::make_pair(2, 128);
    {
        std::lock_guard<std::mutex> lk(g_batch_tune_mutex);
        auto it = g_batch_tune.find(std::make_tuple(b->dims, fmt, b->gauge));
        if (it != g_batch_tune.end()) cfg = it->second;
    }
    if (b->tps) cfg.first = b->tps == -1 ? 0 : b->tps;
    if (b->block) cfg.second = b->block;
    if ((fmt == F64_18 || fmt == F64_12) && b->block64_override) {  // override also for tps 0
        cfg.first = b->tps64_override;
        cfg.second = b->block64_override;
    }
    return cfg;
}

// (re)build the configuration table and tile list for a sites-per-tile size
static int build_tiles(gf_batch *b, int spt)
{
    if (b->tiles_spt == spt && b->dtile) return GF_OK;
    b->cfg.assign(b->n, BatchConfig{});
    std::vector<int> tiles;
    size_t o32 = 0, o64 = 0, og = 0, odf = 0, oe = 0;
    for (int i = 0; i < b->n; ++i) {
        BatchConfig &c = b->cfg[i];
        c.g = b->geom[i];
        size_t pb = (size_t)c.g.plane * 16;
        c.off32 = o32;
        c.off64 = o64;
        c.offg = og;
        c.offdf = odf;
        c.offe = oe;
        o32 += 8 * (size_t)format_chunks(bfmt32(b)) * pb;
        o64 += 8 * (size_t)format_chunks(bfmt64(b)) * pb;
        og += 6 * pb;
        odf += 8 * (size_t)format_chunks(DF64_18) * pb;
        oe += 2 * 9 * pb;
        c.tile0 = (int)tiles.size();
        c.ntiles = (c.g.Vh + spt - 1) / spt;
        c.nk = b->gauge == GF_COULOMB ? 3 : 4;
        for (int t = 0; t < c.ntiles; ++t) tiles.push_back(i);
    }
    if (b->a32_bytes < o32) {
        cudaFree(b->a32);
        b->a32 = nullptr;
        BCK(cudaMalloc(&b->a32, o32));
        b->a32_bytes = o32;
    }
    if (b->a64_bytes < o64) {
        cudaFree(b->a64);
        b->a64 = nullptr;
        BCK(cudaMalloc(&b->a64, o64));
        b->a64_bytes = o64;
    }
    if (b->ag_bytes < og) {
        cudaFree(b->ag);
        b->ag = nullptr;
        BCK(cudaMalloc(&b->ag, og));
        b->ag_bytes = og;
    }
    if (b->fp64_arith && b->adf_bytes < odf) {
        cudaFree(b->adf);
        b->adf = nullptr;
        BCK(cudaMalloc(&b->adf, odf));
        b->adf_bytes = odf;
    }
    if (b->fp64_arith && b->ae_bytes < oe) {
        cudaFree(b->ae);
        b->ae = nullptr;
        BCK(cudaMalloc(&b->ae, oe));
        b->ae_bytes = oe;
    }
    cudaFree(b->dcfg);
    cudaFree(b->dtile);
    cudaFree(b->partials);
    b->dcfg = nullptr;
    b->dtile = nullptr;
    b->partials = nullptr;
    BCK(cudaMalloc(&b->dcfg, sizeof(BatchConfig) * b->n));
    BCK(cudaMalloc(&b->dtile, sizeof(int) * tiles.size()));
    BCK(cudaMalloc(&b->partials, sizeof(double) * 4 * tiles.size()));
    BCK(cudaMemcpy(b->dcfg, b->cfg.data(), sizeof(BatchConfig) * b->n, cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->dtile, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice));
    b->ntiles = (int)tiles.size();
    b->tiles_spt = spt;
    return GF_OK;
}

// layout of the small integer block
// conv[n], sweeps[n], maxit[n], sweeps32[n], status, pad, bar[2]
static int *conv_of(gf_batch *b) { return b->dint; }
static int *sweeps_of(gf_batch *b) { return b->dint + b->n; }
static int *maxit_of(gf_batch *b) { return b->dint + 2 * b->n; }
static int *sweeps32_of(gf_batch *b) { return b->dint + 3 * b->n; }
static int *status_of(gf_batch *b) { return b->dint + 4 * b->n; }
static unsigned *bar_of(gf_batch *b) { return (unsigned *)(b->dint + 4 * b->n + 2); }
static int *sweepsdf_of(gf_batch *b) { return b->dint + 4 * b->n + 4; }
static size_t dint_count(const gf_batch *b) { return 5 * (size_t)b->n + 4; }

// An event recorded inside a stream capture must be an external record node
// to be recorded (and timeable) when the graph is replayed.
static cudaError_t record_event(gf_batch *b, cudaEvent_t ev)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(b->stream, &st);
    if (e != cudaSuccess) return e;
    return st == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, b->stream, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, b->stream);
}

// Issue one persistent phase (a cooperative launch) on the stream.
static int issue_phase(gf_batch *b, int fmt, bool trackg, double omega, double target)
{
    std::pair<int, int> lc = batch_config(b, fmt);
    int tps = lc.first, block = lc.second;
    if (fmt == DF64_18) {  // the double-float site update: one thread per site
        tps = 0;
        block = b->tiles_spt;
    }
    if (b->tiles_spt != block / (tps == 0 ? 1 : tps)) return bfail(b, GF_EINVAL, "both phases need the same sites per tile");
    void *fn = kernel_for(fmt, tps, trackg);
    if (!fn) return bfail(b, GF_EINVAL, "no batched kernel for this format / threads per site");
    int dev = 0, nsm = 0, per_sm = 0;
    const size_t smem = fmt == DF64_18 ? 9 * sizeof(float4) * (size_t)block : 0;  // prefetched E
    BCK(cudaGetDevice(&dev));
    BCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem));
    if (per_sm < 1) return bfail(b, GF_ECUDA, "batched kernel cannot be resident");
    int grid = nsm * per_sm;
    if (grid > 2 * b->ntiles) grid = 2 * b->ntiles;

    BatchArgs a;
    memset(&a, 0, sizeof a);
    a.cfg = b->dcfg;
    a.tile_cfg = b->dtile;
    a.ncfg = b->n;
    a.ntiles = b->ntiles;
    const bool fp64 = !(fmt == F32_12 || fmt == F32_18);
    a.kind = fmt == DF64_18 ? 2 : (fp64 ? 1 : 0);
    a.arena = a.kind == 2 ? b->adf : (fp64 ? b->a64 : b->a32);
    a.garena = b->ag;
    a.earena = b->ae;
    a.omega = omega;
    a.target = target;
    a.check_every = b->check_every;
    a.max_iter = maxit_of(b);
    a.conv = conv_of(b);
    a.sweeps = sweeps_of(b);
    a.F = b->ddbl;
    a.theta = b->ddbl + b->n;
    a.tile_partials = b->partials;
    a.bar = bar_of(b);
    a.status = status_of(b);
    a.timeout_ns = (long long)(b->timeout_ms * 1e6);
    a.expected_blocks = (unsigned)(grid + b->extra_blocks);
    a.reunit = fp64 ? 0 : 1;

    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = { &a };
    BCK(cudaLaunchKernelExC(&cfg, fn, args));
    b->stats[a.kind == 2 ? "grid_df64" : (fp64 ? "grid_fp64" : "grid_fp32")] = grid;
    b->stats["threads_per_site"] = tps;
    b->stats["block"] = block;
    return GF_OK;
}

// The whole solve of one call, stream ordered (capturable).
static int issue_solve(gf_batch *b, double *const *U, double omega, double theta_target, int max_iter)
{
    const bool mixed = b->precision == GF_MIXED;
    const bool fp32_first = b->precision != GF_FP64;
    const bool fp64_phase = !fp32_first || mixed;
    const int f32 = bfmt32(b), f64 = bfmt64(b);
    int nb = (b->n + 127) / 128;
    BCK(record_event(b, b->ev[0]));
    k_batch_first_phase<<<nb, 128, 0, b->stream>>>(b->n, max_iter, conv_of(b), sweeps_of(b), maxit_of(b),
                                                  sweeps32_of(b), sweepsdf_of(b), status_of(b), bar_of(b));
    BCK(cudaGetLastError());
    if (fp32_first) {
        for (int i = 0; i < b->n; ++i) {
            const BatchConfig &c = b->cfg[i];
            BCK(launch_encode(f32, U[i], FieldRef{ b->a32 + c.off32, (size_t)c.g.plane * 16 }, c.g, b->stream));
            if (mixed)
                BCK(launch_gauge_identity(FieldRef{ b->ag + c.offg, (size_t)c.g.plane * 16 }, c.g, b->stream));
        }
        BRET(issue_phase(b, f32, mixed, omega, mixed ? std::max(b->theta_switch, theta_target) : theta_target));
    }
    BCK(record_event(b, b->ev[1]));
    if (fp64_phase) {
        if (mixed) {
            k_batch_next_phase<<<nb, 128, 0, b->stream>>>(b->n, max_iter, conv_of(b), sweeps_of(b), maxit_of(b),
                                                         sweeps32_of(b));
            BCK(cudaGetLastError());
        }
        for (int i = 0; i < b->n; ++i) {
            const BatchConfig &c = b->cfg[i];
            FieldRef d64{ b->a64 + c.off64, (size_t)c.g.plane * 16 };
            if (mixed)
                BCK(launch_apply_tracked_gauge(U[i], FieldRef{ b->ag + c.offg, (size_t)c.g.plane * 16 }, f64, d64,
                                               c.g, b->stream));
            else
                BCK(launch_encode(f64, U[i], d64, c.g, b->stream));
            if (b->fp64_arith)
                BCK(launch_to_df(f64, d64, FieldRef{ b->adf + c.offdf, (size_t)c.g.plane * 16 }, c.g, b->stream));
        }
        if (b->fp64_arith) {
            // double-float sweeps on the copies, E = g - 1 tracked; g applied to the FP64 fields in
            // FP64; native FP64 sweeps then finish whatever lattice is not yet below the target
            BCK(cudaMemsetAsync(b->ae, 0, b->ae_bytes, b->stream));
            BRET(issue_phase(b, DF64_18, false, omega, theta_target));
            for (int i = 0; i < b->n; ++i) {
                const BatchConfig &c = b->cfg[i];
                BCK(launch_apply_gauge_e(f64, FieldRef{ b->a64 + c.off64, (size_t)c.g.plane * 16 },
                                         FieldRef{ b->ae + c.offe, (size_t)c.g.plane * 16 }, c.g, b->stream));
            }
            k_batch_after_df<<<nb, 128, 0, b->stream>>>(b->n, conv_of(b), sweeps_of(b), maxit_of(b), sweepsdf_of(b));
            BCK(cudaGetLastError());
        }
        BRET(issue_phase(b, f64, false, omega, theta_target));
    }
    BCK(record_event(b, b->ev[2]));
    int fmt_out = fp64_phase ? f64 : f32;
    for (int i = 0; i < b->n && !b->skip_decode; ++i) {
        const BatchConfig &c = b->cfg[i];
        FieldRef f{ (fp64_phase ? b->a64 + c.off64 : b->a32 + c.off32), (size_t)c.g.plane * 16 };
        if (!fp64_phase) BCK(launch_reunitarize(f32, f, c.g, b->stream));
        BCK(launch_decode(fmt_out, f, c.g, U[i], b->stream));
    }
    BCK(cudaMemcpyAsync(b->hint, b->dint, sizeof(int) * dint_count(b), cudaMemcpyDeviceToHost,
                        b->stream));
    BCK(cudaMemcpyAsync(b->hdbl, b->ddbl, sizeof(double) * 2 * b->n, cudaMemcpyDeviceToHost, b->stream));
    return GF_OK;
}

static void drop_graph(gf_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_key.clear();
}

static int ensure_small_buffers(gf_batch *b)
{
    if (!b->dint) BCK(cudaMalloc(&b->dint, sizeof(int) * dint_count(b)));
    if (!b->ddbl) BCK(cudaMalloc(&b->ddbl, sizeof(double) * 2 * (size_t)b->n));
    if (!b->hint) BCK(cudaMallocHost(&b->hint, sizeof(int) * dint_count(b)));
    if (!b->hdbl) BCK(cudaMallocHost(&b->hdbl, sizeof(double) * 2 * (size_t)b->n));
    for (int k = 0; k < 3; ++k)
        if (!b->ev[k]) BCK(cudaEventCreate(&b->ev[k]));
    if (!b->cap) BCK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    return GF_OK;
}

extern "C" {

int gf_batch_create(int n, const int *dims, int gauge, gf_batch **out)
{
    if (!out || !dims || n < 1) return GF_EINVAL;
    *out = nullptr;
    if (gauge != GF_LANDAU && gauge != GF_COULOMB) return GF_EINVAL;
    gf_batch *b = new (std::nothrow) gf_batch;
    if (!b) return GF_ENOMEM;
    b->n = n;
    b->gauge = gauge;
    b->dims.assign(dims, dims + 4 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        long V = 1;
        Geom g;
        for (int mu = 0; mu < 4; ++mu) {
            int L = dims[4 * i + mu];
            if (L < 2 || (L & 1)) {
                delete b;
                return GF_EINVAL;
            }
            g.L[mu] = L;
            V *= L;
        }
        if (V >= (1L << 31)) {
            delete b;
            return GF_EINVAL;
        }
        g.Lh0 = g.L[0] / 2;
        g.Vh = (int)(V / 2);
        g.plane = (int)((V / 2 + 63) / 64 * 64);
        b->geom.push_back(g);
        b->total_sites += V;
    }
    *out = b;
    return GF_OK;
}

int gf_batch_destroy(gf_batch *b)
{
    if (!b) return GF_OK;
    drop_graph(b);
    cudaFree(b->a32);
    cudaFree(b->a64);
    cudaFree(b->ag);
    cudaFree(b->adf);
    cudaFree(b->ae);
    cudaFree(b->dcfg);
    cudaFree(b->dtile);
    cudaFree(b->partials);
    cudaFree(b->dint);
    cudaFree(b->ddbl);
    if (b->hint) cudaFreeHost(b->hint);
    if (b->hdbl) cudaFreeHost(b->hdbl);
    for (int k = 0; k < 3; ++k)
        if (b->ev[k]) cudaEventDestroy(b->ev[k]);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return GF_OK;
}

const char *gf_batch_last_error(const gf_batch *b) { return b ? b->err.c_str() : "null batch"; }

int gf_batch_set_stream(gf_batch *b, void *stream)
{
    if (!b) return GF_EINVAL;
    b->stream = (cudaStream_t)stream;
    return GF_OK;
}

int gf_batch_set_option(gf_batch *b, const char *key, double v)
{
    if (!b || !key) return GF_EINVAL;
    std::string k(key);
    int iv = (int)v;
    if (k == "precision") {
        if (iv < GF_FP64 || iv > GF_FP32 || (double)iv != v) return bfail(b, GF_EINVAL, "precision");
        b->precision = iv;
    } else if (k == "storage32" || k == "storage64") {
        if (iv != 12 && iv != 18) return bfail(b, GF_EINVAL, k + ": 12 or 18");
        (k == "storage32" ? b->storage32 : b->storage64) = iv;
        b->tiles_spt = 0;
    } else if (k == "check_every") {
        if (iv < 1 || (double)iv != v) return bfail(b, GF_EINVAL, "check_every >= 1");
        b->check_every = iv;
    } else if (k == "theta_switch") {
        if (!(v > 0)) return bfail(b, GF_EINVAL, "theta_switch > 0");
        b->theta_switch = v;
    } else if (k == "threads_per_site") {
        // 1, 2, 4, 8; 0 = autotuned or default; -1 = the accumulate form (one thread per site)
        if (iv != -1 && iv != 0 && iv != 1 && iv != 2 && iv != 4 && iv != 8) return bfail(b, GF_EINVAL, "threads_per_site");
        b->tps = iv;
    } else if (k == "block") {
        if (iv < 0 || iv > 256 || iv % 32) return bfail(b, GF_EINVAL, "block: 0 or 32..256 step 32");
        b->block = iv;
    } else if (k == "barrier_timeout_ms") {
        if (!(v > 0) || v > 60000) return bfail(b, GF_EINVAL, "barrier_timeout_ms in (0, 60000]");
        b->timeout_ms = v;
    } else if (k == "barrier_extra_blocks") {
        if (iv < 0 || iv > 1) return bfail(b, GF_EINVAL, "barrier_extra_blocks: 0 or 1");
        b->extra_blocks = iv;
    } else if (k == "use_graphs") {
        b->use_graphs = v != 0.0;
    } else if (k == "fp64_arith") {
        if (iv != 0 && iv != 1) return bfail(b, GF_EINVAL, "fp64_arith: 0 (native) or 1 (double-float)");
        b->fp64_arith = iv;
        b->tiles_spt = 0;  // the arenas of the double-float phase are sized with the tiles
    } else {
        return bfail(b, GF_EINVAL, "unknown option " + k);
    }
    drop_graph(b);
    return GF_OK;
}

int gf_batch_get_stat(const gf_batch *b, const char *key, double *v)
{
    if (!b || !key || !v) return GF_EINVAL;
    auto it = b->stats.find(key);
    if (it == b->stats.end()) return GF_EINVAL;
    *v = it->second;
    return GF_OK;
}

int gf_batch_overrelax(gf_batch *b, double *const *U, double omega, double theta_target, int max_iter,
                       int *iters, double *F, double *theta)
{
    if (!b) return GF_EINVAL;
    if (!U) return bfail(b, GF_EINVAL, "U is NULL");
    if (!(omega > 0.0 && omega < 2.0)) return bfail(b, GF_EINVAL, "omega must lie in (0, 2)");
    if (!(theta_target >= 0.0) || !std::isfinite(theta_target) || max_iter < 0)
        return bfail(b, GF_EINVAL, "theta_target >= 0, max_iter >= 0");
    for (int i = 0; i < b->n; ++i) {
        if (!U[i] || (uintptr_t)U[i] % 16 || pointer_kind(U[i]) != PTR_DEVICE)
            return bfail(b, GF_EINVAL, "every field must be a 16-byte aligned pointer to memory of the current device");
    }
    BRET(ensure_small_buffers(b));
    const bool fp32_first = b->precision != GF_FP64;
    const int f32 = bfmt32(b), f64 = bfmt64(b);
    std::pair<int, int> l32 = batch_config(b, f32), l64 = batch_config(b, f64);
    auto spt_of = [](std::pair<int, int> l) { return l.second / (l.first == 0 ? 1 : l.first); };
    int spt = fp32_first ? spt_of(l32) : spt_of(l64);
    if (b->precision == GF_MIXED && spt_of(l64) != spt) {
        // both phases walk one tile table: keep the FP64 phase on the FP32 tile size
        int tps64 = l64.first;
        if (spt * (tps64 == 0 ? 1 : tps64) > 256) tps64 = 0;
        b->tps64_override = tps64;
        b->block64_override = spt * (tps64 == 0 ? 1 : tps64);
    } else {
        b->tps64_override = 0;
        b->block64_override = 0;
    }
    BRET(build_tiles(b, spt));

    // graph key: every input of the captured sequence
    std::string key(reinterpret_cast<const char *>(U), sizeof(double *) * b->n);
    double params[3] = { omega, theta_target, (double)max_iter };
    key.append(reinterpret_cast<const char *>(params), sizeof params);
    key.append(reinterpret_cast<const char *>(&b->stream), sizeof b->stream);

    if (b->use_graphs) {
        if (!b->graph || b->graph_key != key) {
            drop_graph(b);
            cudaStream_t user = b->stream;
            b->stream = b->cap;
            cudaGraph_t g;
            BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            int rc = issue_solve(b, U, omega, theta_target, max_iter);
            cudaError_t e = cudaStreamEndCapture(b->cap, &g);
            b->stream = user;
            if (rc != GF_OK) {
                if (e == cudaSuccess) cudaGraphDestroy(g);
                return rc;
            }
            BCK(e);
            cudaError_t e2 = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            BCK(e2);
            b->graph_key = key;
        }
        BCK(cudaGraphLaunch(b->graph, b->stream));
    } else {
        BRET(issue_solve(b, U, omega, theta_target, max_iter));
    }
    BCK(cudaStreamSynchronize(b->stream));
    float ms32 = 0, ms64 = 0;
    BCK(cudaEventElapsedTime(&ms32, b->ev[0], b->ev[1]));
    BCK(cudaEventElapsedTime(&ms64, b->ev[1], b->ev[2]));
    int status = b->hint[4 * b->n];
    if (status) return bfail(b, status, "a grid barrier wait expired in the persistent batched kernel");
    const bool fp64_phase = !fp32_first || b->precision == GF_MIXED;
    bool all = true;
    double total = 0;
    for (int i = 0; i < b->n; ++i) {
        int s_last = b->hint[b->n + i];
        int s32 = b->precision == GF_MIXED ? b->hint[3 * b->n + i] : (fp32_first ? s_last : 0);
        int sdf = fp64_phase && b->fp64_arith ? b->hint[4 * b->n + 4 + i] : 0;
        int it = b->precision == GF_MIXED ? s32 + sdf + s_last : sdf + s_last;
        double th = b->hdbl[b->n + i];
        if (iters) iters[i] = it;
        if (F) F[i] = b->hdbl[i];
        if (theta) theta[i] = th;
        if (!(th < theta_target)) all = false;
        total += (double)it * 2.0 * b->geom[i].Vh;
    }
    (void)fp64_phase;
    b->stats["site_updates"] = total;
    b->stats["ms_fp32"] = ms32;
    b->stats["ms_fp64"] = ms64;
    b->stats["ms_total"] = ms32 + ms64;
    b->stats["tiles"] = b->ntiles;
    return all ? GF_OK : GF_ENOTCONVERGED;
}

int gf_batch_autotune(gf_batch *b, double *const *U, int *threads_per_site, int *block)
{
    if (!b) return GF_EINVAL;
    const int saved_prec = b->precision, saved_tps = b->tps, saved_block = b->block, saved_graphs = b->use_graphs;
    const int fmts[2] = { bfmt32(b), bfmt64(b) };
    const int precs[2] = { GF_FP32, GF_FP64 };
    const int tps_c[5] = { 0, 1, 2, 4, 8 }, blk_c[3] = { 64, 128, 256 };
    int rc = GF_OK;
    b->skip_decode = 1;
    b->use_graphs = 0;
    for (int f = 0; f < 2 && rc == GF_OK; ++f) {
        double best = 1e300;
        std::pair<int, int> pick{ 1, 128 };
        b->precision = precs[f];
        for (int i = 0; i < 5 && rc == GF_OK; ++i)
            for (int k = 0; k < 3 && rc == GF_OK; ++k) {
                b->tps = tps_c[i] == 0 ? -1 : tps_c[i];
                b->block = blk_c[k];
                // fixed work: theta_target 0 never converges, 2 checks' worth of sweeps
                int r = gf_batch_overrelax(b, U, 1.7, 0.0, 2 * b->check_every, nullptr, nullptr, nullptr);
                if (r != GF_ENOTCONVERGED && r != GF_OK) {
                    rc = r;
                    break;
                }
                double ms = b->stats["ms_total"];
                if (ms < best) {
                    best = ms;
                    pick = { tps_c[i], blk_c[k] };
                }
            }
        if (rc == GF_OK) {
            std::lock_guard<std::mutex> lk(g_batch_tune_mutex);
            g_batch_tune[std::make_tuple(b->dims, fmts[f], b->gauge)] = pick;
            if (f == 0) {
                if (threads_per_site) *threads_per_site = pick.first;
                if (block) *block = pick.second;
            }
        }
    }
    b->skip_decode = 0;
    b->precision = saved_prec;
    b->tps = saved_tps;
    b->block = saved_block;
    b->use_graphs = saved_graphs;
    b->tiles_spt = 0;
    drop_graph(b);
    return rc;
}

// One call for the common case: a batch with the default options, used once.
int gf_overrelax_batched(int n, const int (*dims)[4], double **U, double omega, double theta_target, int max_iter,
                         int *iters, double *F, double *theta)
{
    if (n < 1 || !dims || !U) return GF_EINVAL;
    gf_batch *b = nullptr;
    int rc = gf_batch_create(n, &dims[0][0], GF_LANDAU, &b);
    if (rc != GF_OK) return rc;
    b->use_graphs = 0;  // used once: capturing a graph would not pay
    rc = gf_batch_overrelax(b, U, omega, theta_target, max_iter, iters, F, theta);
    gf_batch_destroy(b);
    return rc;
}

}  // extern "C"
