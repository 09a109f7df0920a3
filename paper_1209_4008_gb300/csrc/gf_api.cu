// gf_api.cu -- the C ABI of libgf.so (declared in include/gf.h): contexts,
// options, the resident field, the convergence loop of Alg. 1 (theta checked
// every N sweeps, Sec. 4.1) replayed from CUDA graphs, the mixed FP32 -> FP64
// driver, simulated annealing and the threads-per-site autotuner.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "gf.h"
#include "gf_internal.h"

using namespace gf;

namespace {

struct GraphKey {
    int fmt, tps, block, n, trackg, measure, reunit, ktime, orv, slices;
    double omega;
    const void *field, *gt, *ge;
    bool operator<(const GraphKey &o) const
    {
        return std::tie(fmt, tps, block, n, trackg, measure, reunit, ktime, orv, slices, omega, field, gt, ge) <
               std::tie(o.fmt, o.tps, o.block, o.n, o.trackg, o.measure, o.reunit, o.ktime, o.orv, o.slices,
                        o.omega, o.field, o.gt, o.ge);
    }
};

// resident state of gf_overrelax's double-float stages: the working copy
// (fdf, DF64_18) of the exact FP64 field (f64); never visible between calls
constexpr int kResDfWork = 3;

std::mutex g_tune_mutex;
// autotuner cache: (Lx, Ly, Lz, Lt, format, gauge, mode) -> (threads per site, block);
// mode 0: overrelaxation (and stochastic relaxation), 1: heatbath
std::map<std::tuple<int, int, int, int, int, int, int>, std::pair<int, int>> g_tune_cache;

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct gf_ctx {
    int dims[4];
    int gauge;
    Geom geom;
    long V;
    // options
    int precision = GF_FP64;
    int storage64 = 18;
    int storage32 = 12;
    int check_every = 100;
    double theta_switch = 1e-6;
    int track_gauge = 1;
    int reunit_every = 1;
    int tps = 0;
    int block = 0;
    int fp64_arith = 0;  // FP64 phase: 0 native FP64, 1 double-float on the FP32 pipe (DF64_18)
    bool exact_run = false;  // inside gf_overrelax with double-float stages on a copy of an FP64 field
    int variant = 0;  // 0 auto, 1 per-subgroup rotations of the held links, 2 accumulate form
    int acc_regs = 0;  // accumulate form, FP64 storage: register budget 255, 168 or 128 (0 = autotuned)
    int or_variant = 0;  // g -> g^omega: 0 rational 19-flop form, 1 first order, 2 exact power
    int learned_repeat = 0;       // further applications of the learned warm start in the FP64 phase
    double learned_factor = 1e-2;  // ... each after theta has fallen by this factor
    int fp32_restarts = 0;  // GF_MIXED: FP32 stages after the first, each from the FP64 field with g reset
    int slice_theta = 0;  // 1: convergence judged on the largest theta of the timeslices
    double *dslices = nullptr;  // F_t, theta_t of the last per-timeslice measurement
    int use_graphs = 1;
    int kernel_timing = 0;     // events around the sweep kernels of every check chunk
    cudaEvent_t kev[2] = { nullptr, nullptr };
    double kms[2] = { 0.0, 0.0 };  // sweep-kernel milliseconds of the last call: [FP32 storage, FP64 class]
    long kn[2] = { 0, 0 };         // half-sweep launches those milliseconds cover
    int autotune = 0;
    int sa_cap = 64;
    int sa_draw = 0;           // heatbath draw: 0 the FP64 definition, 1 its FP32 reading
    uint32_t sa_sweep_offset = 0;
    int track = 0;             // resident sweeps also rotate the tracked g
    double sr_p = 0.0;         // > 0: gf_overrelax uses stochastic relaxation with this probability
    uint64_t sr_seed = 1;      // Philox key of the stochastic relaxation draws
    uint32_t sr_sweep = 0;     // Philox sweep counter, advanced by every stochastic sweep
    gf_net *net = nullptr;     // learned warm start applied at the FP32 -> FP64 switch
    void *feat = nullptr;      // BF16 network inputs [V][80]
    float *cbuf = nullptr;     // network outputs [V][8]
    // streams
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    // device buffers
    char *f64 = nullptr;
    size_t f64_bytes = 0;
    char *f32 = nullptr;
    size_t f32_bytes = 0;
    char *gt = nullptr;
    char *fdf = nullptr;  // double-float working copy of the FP64 field (gf_overrelax, fp64_arith 1)
    char *ge = nullptr;   // E = g - 1 tracked by the double-float sweeps (DF64_18 site field)
    double *staging = nullptr;
    double *partials = nullptr;
    double *dres = nullptr;
    double *hres = nullptr;
    int *dstatus = nullptr;
    int resident = -1;
    int resident_fmt = -1;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::map<std::string, double> stats;
    std::string err;
};

// ---------------------------------------------------------------------------
// error helpers
// ---------------------------------------------------------------------------
static int fail(gf_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

static int cuda_fail(gf_ctx *c, cudaError_t e, const char *what)
{
    cudaGetLastError();  // do not leave the error for the next runtime call to report
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return fail(c, e == cudaErrorMemoryAllocation ? GF_ENOMEM : GF_ECUDA, buf);
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

#define RET(call)                   \
    do {                            \
        int r_ = (call);            \
        if (r_ != GF_OK) return r_; \
    } while (0)

// ---------------------------------------------------------------------------
// buffers
// ---------------------------------------------------------------------------
static int fmt64(const gf_ctx *c)
{
    if (c->fp64_arith == 1 && !c->exact_run) return DF64_18;
    return c->storage64 == 12 ? F64_12 : F64_18;
}
static int fmt32(const gf_ctx *c) { return c->storage32 == 18 ? F32_18 : F32_12; }
// the Coulomb flag and the overrelaxation mode of the sweep kernels for the context's gauge
static int coulomb_of(const gf_ctx *c) { return c->gauge == GF_COULOMB ? 1 : 0; }
static int or_mode(const gf_ctx *c) { return c->gauge == GF_MAG ? 3 : 0; }  // MODE_MAG : MODE_OR
static bool twelve_real(int fmt) { return fmt == F64_12 || fmt == F32_12; }

static size_t plane_bytes(const gf_ctx *c) { return (size_t)c->geom.plane * 16; }
static size_t field_bytes(const gf_ctx *c, int fmt) { return 8 * (size_t)format_chunks(fmt) * plane_bytes(c); }

static FieldRef ref(const gf_ctx *c, char *base) { return FieldRef{ base, plane_bytes(c) }; }

static void drop_graphs(gf_ctx *c)
{
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
}

static int ensure_common(gf_ctx *ctx)
{
    if (!ctx->partials) {
        size_t n = (size_t)measure_blocks(ctx->geom);
        size_t m = (size_t)aos_blocks(ctx->geom);
        size_t k = (size_t)slice_blocks(ctx->geom) * (size_t)ctx->geom.L[3];
        CK(cudaMalloc(&ctx->partials, sizeof(double) * 2 * std::max(n, std::max(m, k))));
    }
    if (!ctx->dslices) CK(cudaMalloc(&ctx->dslices, sizeof(double) * 2 * (size_t)ctx->geom.L[3]));
    if (!ctx->dres) CK(cudaMalloc(&ctx->dres, sizeof(double) * 4));
    if (!ctx->hres) CK(cudaMallocHost(&ctx->hres, sizeof(double) * 4));
    if (!ctx->dstatus) CK(cudaMalloc(&ctx->dstatus, sizeof(int) * 4));
    if (!ctx->cap) CK(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
    return GF_OK;
}

static int ensure_field(gf_ctx *ctx, int prec)
{
    RET(ensure_common(ctx));
    if (prec == GF_FP64) {
        size_t need = field_bytes(ctx, fmt64(ctx));
        if (ctx->f64_bytes < need) {
            drop_graphs(ctx);
            if (ctx->f64) cudaFree(ctx->f64);
            ctx->f64 = nullptr;
            ctx->f64_bytes = 0;
            CK(cudaMalloc(&ctx->f64, need));
            ctx->f64_bytes = need;
        }
    } else {
        size_t need = field_bytes(ctx, fmt32(ctx));
        if (ctx->f32_bytes < need) {
            drop_graphs(ctx);
            if (ctx->f32) cudaFree(ctx->f32);
            ctx->f32 = nullptr;
            ctx->f32_bytes = 0;
            CK(cudaMalloc(&ctx->f32, need));
            ctx->f32_bytes = need;
        }
    }
    return GF_OK;
}

static int ensure_gauge_field(gf_ctx *ctx)
{
    if (!ctx->gt) {
        drop_graphs(ctx);
        CK(cudaMalloc(&ctx->gt, 2 * 3 * plane_bytes(ctx)));
    }
    return GF_OK;
}

// the double-float working field and the E field of gf_overrelax's double-float stages
static int ensure_df_work(gf_ctx *ctx)
{
    if (!ctx->fdf) {
        drop_graphs(ctx);
        CK(cudaMalloc(&ctx->fdf, field_bytes(ctx, DF64_18)));
    }
    if (!ctx->ge) {
        drop_graphs(ctx);
        CK(cudaMalloc(&ctx->ge, 2 * 9 * plane_bytes(ctx)));
    }
    return GF_OK;
}

static int ensure_staging(gf_ctx *ctx)
{
    if (!ctx->staging) CK(cudaMalloc(&ctx->staging, sizeof(double) * 72 * (size_t)ctx->V));
    return GF_OK;
}

// device view of a caller field: the pointer itself, or the staging copy
static int device_view(gf_ctx *ctx, const double *U, const double **view, bool *host)
{
    if (!U) return fail(ctx, GF_EINVAL, "field pointer is NULL");
    if ((uintptr_t)U % 16) return fail(ctx, GF_EINVAL, "field pointer must be 16-byte aligned");
    const PtrKind k = pointer_kind(U);
    if (k == PTR_FOREIGN) return fail(ctx, GF_EINVAL, "field is device memory of another device");
    *host = k == PTR_HOST;
    if (*host) {
        RET(ensure_staging(ctx));
        CK(cudaMemcpyAsync(ctx->staging, U, sizeof(double) * 72 * (size_t)ctx->V, cudaMemcpyHostToDevice,
                           ctx->stream));
        *view = ctx->staging;
    } else {
        *view = U;
    }
    return GF_OK;
}

static char *resident_base(gf_ctx *ctx)
{
    if (ctx->resident == kResDfWork) return ctx->fdf;
    return ctx->resident == GF_FP64 ? ctx->f64 : ctx->f32;
}

// ---------------------------------------------------------------------------
// launch configuration
// ---------------------------------------------------------------------------
static std::pair<int, int> default_config(int fmt)
{
    switch (fmt) {
    case F32_12: return { GF_ACC, 64 };
    case F32_18: return { 2, 128 };
    case F64_12: return { GF_ACC, 64 };
    case DF64_18: return { GF_ACC, 128 };
    default: return { GF_ACC, 64 };  // F64_18
    }
}

static std::tuple<int, int, int, int, int, int, int> tune_key(const gf_ctx *c, int fmt, int mode)
{
    return std::make_tuple(c->dims[0], c->dims[1], c->dims[2], c->dims[3], fmt, c->gauge, mode == 1 ? 1 : 0);
}

static std::pair<int, int> launch_config(const gf_ctx *c, int fmt, int mode = 0)
{
    std::pair<int, int> cfg = default_config(fmt);
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_cache.find(tune_key(c, fmt, mode));
        if (it == g_tune_cache.end() && mode == 1) it = g_tune_cache.find(tune_key(c, fmt, 0));
        if (it != g_tune_cache.end()) cfg = it->second;
    }
    if (c->tps) cfg.first = c->tps;
    if (c->variant == 2 && cfg.first > 0) cfg.first = GF_ACC;  // accumulate form: one thread per site
    if (c->variant == 1 && cfg.first <= 0) cfg.first = c->tps ? c->tps : 2;
    if (cfg.first <= 0 && c->acc_regs) {  // explicit register budget of the accumulate form
        cfg.first = c->acc_regs == 168 ? GF_ACC_R168 : (c->acc_regs == 128 ? GF_ACC_R128 : GF_ACC);
        if (fmt != F64_18 && fmt != F64_12) cfg.first = GF_ACC;
    }
    if (cfg.first == GF_ACC_R168 && cfg.second > 128) cfg.second = 128;
    if (c->gauge == GF_MAG && cfg.first <= 0) cfg.first = c->tps > 0 ? c->tps : 2;  // per-subgroup form only
    if (c->block) cfg.second = c->block;
    return cfg;
}

static SweepArgs sweep_args(gf_ctx *ctx, char *field, int parity, double omega)
{
    SweepArgs a;
    memset(&a, 0, sizeof a);
    a.f = ref(ctx, field);
    a.gt = ref(ctx, ctx->gt);
    if (ctx->resident == kResDfWork && field == ctx->fdf) a.ge = ref(ctx, ctx->ge);
    a.g = ctx->geom;
    a.parity = parity;
    a.omega = omega;
    a.orv = ctx->or_variant;
    a.T = 1.0;
    a.cap = ctx->sa_cap;
    a.sa_fp32 = ctx->sa_draw;
    a.status = ctx->dstatus;
    return a;
}

static cudaError_t issue_sweeps(gf_ctx *ctx, int fmt, char *field, double omega, int n, bool trackg,
                                std::pair<int, int> cfg, cudaStream_t s)
{
    for (int k = 0; k < n; ++k)
        for (int p = 0; p < 2; ++p) {
            SweepArgs a = sweep_args(ctx, field, p, omega);
            cudaError_t e = launch_sweep(fmt, a, cfg.first, coulomb_of(ctx), or_mode(ctx), trackg, cfg.second, s);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

// F and theta (or, per timeslice, mean F_t and max theta_t) of a resident field into dres
static cudaError_t launch_check(gf_ctx *ctx, int fmt, FieldRef f, cudaStream_t s)
{
    if (ctx->slice_theta)
        return launch_measure_slices(fmt, f, ctx->geom, ctx->gauge, ctx->partials, ctx->dslices, ctx->dres, s);
    return launch_measure(fmt, f, ctx->geom, ctx->gauge, ctx->partials, ctx->dres, s);
}

// n sweeps of the resident field [+ reunitarisation] [+ F/theta into hres]
static int run_chunk(gf_ctx *ctx, int fmt, char *field, double omega, int n, bool trackg, bool measure,
                     bool reunit)
{
    std::pair<int, int> cfg = launch_config(ctx, fmt);
    FieldRef f = ref(ctx, field);
    const bool kt = ctx->kernel_timing && n > 0;
    if (ctx->sr_p > 0.0) {  // stochastic relaxation: fresh Philox counters every sweep, no graph replay
        if (kt) CK(cudaEventRecord(ctx->kev[0], ctx->stream));
        for (int k = 0; k < n; ++k, ++ctx->sr_sweep)
            for (int p = 0; p < 2; ++p) {
                SweepArgs a = sweep_args(ctx, field, p, omega);
                a.prob = ctx->sr_p;
                a.key = make_uint2((uint32_t)ctx->sr_seed, (uint32_t)(ctx->sr_seed >> 32));
                a.sweep = ctx->sr_sweep;
                CK(launch_sweep(fmt, a, cfg.first, coulomb_of(ctx), 2, false, cfg.second, ctx->stream));
            }
        if (kt) CK(cudaEventRecord(ctx->kev[1], ctx->stream));
        if (reunit) CK(launch_reunitarize(fmt, f, ctx->geom, ctx->stream));
        if (measure) {
            CK(launch_check(ctx, fmt, f, ctx->stream));
            CK(cudaMemcpyAsync(ctx->hres, ctx->dres, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        }
        return GF_OK;
    }
    if (ctx->use_graphs && n > 0) {
        GraphKey key{ fmt,    cfg.first,       cfg.second,       n,     trackg, measure, reunit, kt ? 1 : 0,
                      ctx->or_variant, ctx->slice_theta, omega, field, ctx->gt,
                      ctx->resident == kResDfWork ? ctx->ge : nullptr };
        auto it = ctx->graphs.find(key);
        if (it == ctx->graphs.end()) {
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            if (kt) e = cudaEventRecordWithFlags(ctx->kev[0], ctx->cap, cudaEventRecordExternal);
            if (e == cudaSuccess) e = issue_sweeps(ctx, fmt, field, omega, n, trackg, cfg, ctx->cap);
            if (e == cudaSuccess && kt) e = cudaEventRecordWithFlags(ctx->kev[1], ctx->cap, cudaEventRecordExternal);
            if (e == cudaSuccess && reunit) e = launch_reunitarize(fmt, f, ctx->geom, ctx->cap);
            if (e == cudaSuccess && measure)
                e = launch_check(ctx, fmt, f, ctx->cap);
            if (e == cudaSuccess && measure)
                e = cudaMemcpyAsync(ctx->hres, ctx->dres, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->cap);
            cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &graph);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "capturing the sweep graph");
            CK(e2);
            cudaGraphExec_t exec;
            cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            CK(e3);
            it = ctx->graphs.emplace(key, exec).first;
        }
        CK(cudaGraphLaunch(it->second, ctx->stream));
        return GF_OK;
    }
    if (kt) CK(cudaEventRecord(ctx->kev[0], ctx->stream));
    CK(issue_sweeps(ctx, fmt, field, omega, n, trackg, cfg, ctx->stream));
    if (kt) CK(cudaEventRecord(ctx->kev[1], ctx->stream));
    if (reunit) CK(launch_reunitarize(fmt, f, ctx->geom, ctx->stream));
    if (measure) {
        CK(launch_check(ctx, fmt, f, ctx->stream));
        CK(cudaMemcpyAsync(ctx->hres, ctx->dres, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    return GF_OK;
}

static int measure_resident(gf_ctx *ctx, double *F, double *theta)
{
    if (ctx->resident < 0) return fail(ctx, GF_ESTATE, "no resident field");
    CK(launch_check(ctx, ctx->resident_fmt, ref(ctx, resident_base(ctx)), ctx->stream));
    CK(cudaMemcpyAsync(ctx->hres, ctx->dres, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (F) *F = ctx->hres[0];
    if (theta) *theta = ctx->hres[1];
    return GF_OK;
}

// below this theta a check may declare the FP32 rounding floor reached (stall)
constexpr double kStallTheta = 1e-8;

// Alg. 1 WHILE loop on the resident field: theta known on entry; sweep in
// chunks of check_every until theta < target or budget sweeps are spent.
// stall: also stop once theta (below kStallTheta) has fallen by less than 10 %
// over the last 100 sweeps -- the rounding floor of an FP32 field.
static int converge(gf_ctx *ctx, double omega, double target, int budget, bool trackg, bool reunit, int *used,
                    double *F, double *theta, bool stall = false)
{
    int fmt = ctx->resident_fmt;
    char *field = resident_base(ctx);
    int it = 0, checks = 0;
    const int window = std::max(1, (100 + ctx->check_every - 1) / ctx->check_every);
    std::vector<double> hist;
    while (!(*theta < target) && it < budget) {
        int n = ctx->check_every;
        if (n > budget - it) n = budget - it;
        RET(run_chunk(ctx, fmt, field, omega, n, trackg, true, reunit));
        CK(cudaStreamSynchronize(ctx->stream));
        if (ctx->kernel_timing && n > 0) {
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, ctx->kev[0], ctx->kev[1]));
            const int w = (fmt == F32_12 || fmt == F32_18) ? 0 : 1;
            ctx->kms[w] += ms;
            ctx->kn[w] += 2L * n;
        }
        *F = ctx->hres[0];
        *theta = ctx->hres[1];
        it += n;
        ++checks;
        if (!std::isfinite(*theta)) return fail(ctx, GF_EINVAL, "theta became non-finite (input not in SU(3)?)");
        if (stall) {
            hist.push_back(*theta);
            const size_t m = hist.size();
            if (*theta < kStallTheta && m > (size_t)window && *theta > 0.9 * hist[m - 1 - window]) break;
        }
    }
    *used = it;
    ctx->stats["checks"] += checks;
    return GF_OK;
}

static int upload(gf_ctx *ctx, const double *view, int prec)
{
    RET(ensure_field(ctx, prec));
    int fmt = prec == GF_FP64 ? fmt64(ctx) : fmt32(ctx);
    char *base = prec == GF_FP64 ? ctx->f64 : ctx->f32;
    CK(launch_encode(fmt, view, ref(ctx, base), ctx->geom, ctx->stream));
    ctx->resident = prec;
    ctx->resident_fmt = fmt;
    return GF_OK;
}

static int download(gf_ctx *ctx, double *U, bool host)
{
    if (ctx->resident < 0) return fail(ctx, GF_ESTATE, "no resident field");
    double *dst = U;
    if (host) {
        RET(ensure_staging(ctx));
        dst = ctx->staging;
    }
    CK(launch_decode(ctx->resident_fmt, ref(ctx, resident_base(ctx)), ctx->geom, dst, ctx->stream));
    if (host) {
        CK(cudaMemcpyAsync(U, ctx->staging, sizeof(double) * 72 * (size_t)ctx->V, cudaMemcpyDeviceToHost,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return GF_OK;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
// heatbath half-sweeps of a scratch field for the autotuner (T = 1, fixed key)
static cudaError_t issue_sa_sweeps(gf_ctx *ctx, int fmt, char *field, int n, std::pair<int, int> cfg, cudaStream_t s)
{
    for (int k = 0; k < n; ++k)
        for (int p = 0; p < 2; ++p) {
            SweepArgs a = sweep_args(ctx, field, p, 1.0);
            a.T = 1.0;
            a.key = make_uint2(0x9e3779b9u, 0u);
            a.sweep = (uint32_t)k;
            cudaError_t e = launch_sweep(fmt, a, cfg.first, coulomb_of(ctx), 1, false, cfg.second, s);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

// mode 0: time overrelaxation sweeps; 1: heatbath sweeps
static int autotune_format(gf_ctx *ctx, int fmt, char *field, int *tps_out, int *block_out, int mode = 0)
{
    size_t bytes = field_bytes(ctx, fmt);
    char *scratch = nullptr;
    CK(cudaMalloc(&scratch, bytes));
    cudaError_t e = cudaMemcpyAsync(scratch, field, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // accumulate form (with the smaller register budgets for FP64 storage), then 1-8 threads per site
    const int tps_c[7] = { GF_ACC, 1, 2, 4, 8, GF_ACC_R168, GF_ACC_R128 };
    const int ntps = (fmt == F64_18 || fmt == F64_12) ? 7 : 5;
    const int blk_c[3] = { 64, 128, 256 };
    float best = 1e30f;
    std::pair<int, int> pick = default_config(fmt);
    if (ctx->gauge == GF_MAG) pick.first = 2;
    for (int i = 0; i < ntps && e == cudaSuccess; ++i)
        for (int b = 0; b < 3 && e == cudaSuccess; ++b) {
            if (tps_c[i] == GF_ACC_R168 && blk_c[b] > 128) continue;
            // the double-float overrelaxation kernel runs blocks of at most 128 threads
            if (fmt == DF64_18 && tps_c[i] == GF_ACC && mode == 0 && blk_c[b] > 128) continue;
            if (ctx->gauge == GF_MAG && tps_c[i] <= 0) continue;  // the MAG step uses the per-subgroup form
            std::pair<int, int> cfg{ tps_c[i], blk_c[b] };
            e = mode == 1 ? issue_sa_sweeps(ctx, fmt, scratch, 1, cfg, ctx->stream)
                          : issue_sweeps(ctx, fmt, scratch, 1.7, 1, false, cfg, ctx->stream);  // warm up
            if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
            if (e == cudaSuccess)
                e = mode == 1 ? issue_sa_sweeps(ctx, fmt, scratch, 2, cfg, ctx->stream)
                              : issue_sweeps(ctx, fmt, scratch, 1.7, 3, false, cfg, ctx->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            // a smaller register budget of the accumulate form (more sites in flight per SM)
            // replaces a larger one only if it is more than 1 % faster: with fewer sites in
            // flight the second read of each site's links still finds them in L2, so the
            // larger budget moves fewer DRAM bytes at the same FP64-bound time
            const bool more_in_flight = tps_c[i] < 0 && pick.first <= 0 && tps_c[i] < pick.first;
            if (e == cudaSuccess && ms < (more_in_flight ? 0.99f : 1.0f) * best) {
                best = ms;
                pick = cfg;
            }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(scratch);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_cache[tune_key(ctx, fmt, mode)] = pick;
    }
    if (tps_out) *tps_out = pick.first;
    if (block_out) *block_out = pick.second;
    return GF_OK;
}

static bool tuned(const gf_ctx *c, int fmt, int mode = 0)
{
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    return g_tune_cache.count(tune_key(c, fmt, mode)) > 0;
}

// One double-float stage of gf_overrelax's FP64 phase ("fp64_arith" 1).  The
// resident FP64 field (the exact field) is copied into the double-float
// working field, whose sweeps run on the FP32 pipe while the transformation
// they apply is tracked as E = g - 1 in double-float; at the end g = 1 + E,
// reunitarised in FP64, is applied to the exact field in FP64.  The exact
// field therefore stays a gauge transform of the input to FP64 rounding,
// whatever the double-float rounding of the working copy.  On entry F and
// theta are those of the exact field; on return, too.
static int df_stage(gf_ctx *ctx, double omega, double target, int budget, int *used, double *F, double *theta)
{
    *used = 0;
    if (*theta < target || budget <= 0) return GF_OK;
    const int xfmt = ctx->resident_fmt;
    RET(ensure_df_work(ctx));
    CK(launch_to_df(xfmt, ref(ctx, ctx->f64), ref(ctx, ctx->fdf), ctx->geom, ctx->stream));
    CK(cudaMemsetAsync(ctx->ge, 0, 2 * 9 * plane_bytes(ctx), ctx->stream));
    ctx->resident = kResDfWork;
    ctx->resident_fmt = DF64_18;
    if (ctx->autotune && !tuned(ctx, DF64_18)) {
        const int rc = autotune_format(ctx, DF64_18, ctx->fdf, nullptr, nullptr);
        if (rc != GF_OK) {
            ctx->resident = GF_FP64;
            ctx->resident_fmt = xfmt;
            return rc;
        }
    }
    double Fw = *F, thw = *theta;
    int u = 0;
    const int rc = converge(ctx, omega, target, budget, true, false, &u, &Fw, &thw);
    ctx->resident = GF_FP64;  // back to the exact field, whatever happened
    ctx->resident_fmt = xfmt;
    RET(rc);
    CK(launch_apply_gauge_e(xfmt, ref(ctx, ctx->f64), ref(ctx, ctx->ge), ctx->geom, ctx->stream));
    RET(measure_resident(ctx, F, theta));
    *used = u;
    ctx->stats["sweeps_df64"] += u;
    return GF_OK;
}

// FP64-class convergence of the resident FP64 field: double-float stages
// (exact_run), then native FP64 sweeps for whatever target is left; else
// native FP64 sweeps (12-real storage reunitarised at every check)
static int converge64(gf_ctx *ctx, double omega, double target, int budget, int *used, double *F, double *theta)
{
    *used = 0;
    if (ctx->exact_run) {
        RET(df_stage(ctx, omega, target, budget, used, F, theta));
        budget -= *used;
    }
    int u = 0;
    RET(converge(ctx, omega, target, budget, false, twelve_real(ctx->resident_fmt), &u, F, theta));
    *used += u;
    return GF_OK;
}

// ---------------------------------------------------------------------------
// learned warm start (resident FP64 field)
// ---------------------------------------------------------------------------
static int ensure_learned_buffers(gf_ctx *ctx)
{
    if (!ctx->feat) CK(cudaMalloc(&ctx->feat, 2 * (size_t)GF_NET_CIN * ctx->V));
    if (!ctx->cbuf) CK(cudaMalloc(&ctx->cbuf, sizeof(float) * GF_NET_COUT * ctx->V));
    return GF_OK;
}

// network inputs -> network -> g = exp(i s c.lambda/2) -> resident field g U g^+
static int learned_correction(gf_ctx *ctx, double theta)
{
    if (ctx->resident != GF_FP64) return fail(ctx, GF_ESTATE, "learned correction needs the FP64 field");
    RET(ensure_learned_buffers(ctx));
    RET(ensure_gauge_field(ctx));
    double s = sqrt(theta);
    CK(launch_features(ctx->resident_fmt, ref(ctx, ctx->f64), ctx->geom, 1.0 / s, ctx->feat, ctx->stream));
    gf_net_set_stream(ctx->net, ctx->stream);
    int r = gf_net_forward(ctx->net, ctx->feat, ctx->cbuf);
    if (r != GF_OK) return fail(ctx, r, std::string("network: ") + gf_net_last_error(ctx->net));
    CK(launch_expmap_to_gauge(ctx->cbuf, s, ref(ctx, ctx->gt), ctx->geom, ctx->stream));
    CK(launch_gauge_transform_resident(ctx->resident_fmt, ref(ctx, ctx->f64), ref(ctx, ctx->gt), ctx->geom,
                                       ctx->stream));
    return GF_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *gf_error_string(int code)
{
    switch (code) {
    case GF_OK: return "GF_OK";
    case GF_EINVAL: return "GF_EINVAL";
    case GF_ECUDA: return "GF_ECUDA";
    case GF_ETIMEOUT: return "GF_ETIMEOUT";
    case GF_ENOTCONVERGED: return "GF_ENOTCONVERGED";
    case GF_ENOMEM: return "GF_ENOMEM";
    case GF_EREJECT: return "GF_EREJECT";
    case GF_ESTATE: return "GF_ESTATE";
    default: return "GF_UNKNOWN";
    }
}

int gf_create(const int dims[4], int gauge, gf_ctx **out)
{
    if (!dims || !out) return GF_EINVAL;
    *out = nullptr;
    if (gauge != GF_LANDAU && gauge != GF_COULOMB && gauge != GF_MAG) return GF_EINVAL;
    long V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2 || (dims[mu] & 1)) return GF_EINVAL;
        V *= dims[mu];
        if (V >= (1L << 31)) return GF_EINVAL;
    }
    gf_ctx *c = new (std::nothrow) gf_ctx;
    if (!c) return GF_ENOMEM;
    for (int mu = 0; mu < 4; ++mu) {
        c->dims[mu] = dims[mu];
        c->geom.L[mu] = dims[mu];
    }
    c->gauge = gauge;
    c->V = V;
    c->geom.Lh0 = dims[0] / 2;
    c->geom.Vh = (int)(V / 2);
    c->geom.plane = (int)((V / 2 + 63) / 64 * 64);
    *out = c;
    return GF_OK;
}

int gf_destroy(gf_ctx *ctx)
{
    if (!ctx) return GF_OK;
    drop_graphs(ctx);
    cudaFree(ctx->f64);
    cudaFree(ctx->f32);
    cudaFree(ctx->gt);
    cudaFree(ctx->fdf);
    cudaFree(ctx->ge);
    cudaFree(ctx->staging);
    cudaFree(ctx->feat);
    cudaFree(ctx->cbuf);
    cudaFree(ctx->partials);
    cudaFree(ctx->dslices);
    cudaFree(ctx->dres);
    cudaFree(ctx->dstatus);
    if (ctx->hres) cudaFreeHost(ctx->hres);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    for (int i = 0; i < 2; ++i)
        if (ctx->kev[i]) cudaEventDestroy(ctx->kev[i]);
    delete ctx;
    return GF_OK;
}

const char *gf_last_error(const gf_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int gf_set_stream(gf_ctx *ctx, void *stream)
{
    if (!ctx) return GF_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    return GF_OK;
}

int gf_set_option(gf_ctx *ctx, const char *key, double v)
{
    if (!ctx || !key) return GF_EINVAL;
    std::string k(key);
    int iv = (int)v;
    bool integral = (double)iv == v;
    if (k == "precision") {
        if (!integral || iv < GF_FP64 || iv > GF_FP32) return fail(ctx, GF_EINVAL, "precision: 0, 1 or 2");
        ctx->precision = iv;
    } else if (k == "storage64") {
        if (iv != 18 && iv != 12) return fail(ctx, GF_EINVAL, "storage64: 18 or 12");
        if (ctx->resident == GF_FP64 && iv != ctx->storage64) ctx->resident = -1;
        ctx->storage64 = iv;
    } else if (k == "storage32") {
        if (iv != 18 && iv != 12) return fail(ctx, GF_EINVAL, "storage32: 18 or 12");
        if (ctx->resident == GF_FP32 && iv != ctx->storage32) ctx->resident = -1;
        ctx->storage32 = iv;
    } else if (k == "check_every") {
        if (!integral || iv < 1) return fail(ctx, GF_EINVAL, "check_every >= 1");
        ctx->check_every = iv;
    } else if (k == "theta_switch") {
        if (!(v > 0.0)) return fail(ctx, GF_EINVAL, "theta_switch > 0");
        ctx->theta_switch = v;
    } else if (k == "track_gauge") {
        ctx->track_gauge = v != 0.0;
    } else if (k == "reunitarize_every") {
        if (!integral || iv < 0) return fail(ctx, GF_EINVAL, "reunitarize_every >= 0");
        ctx->reunit_every = iv;
    } else if (k == "threads_per_site") {
        if (iv != 0 && iv != 1 && iv != 2 && iv != 4 && iv != 8) return fail(ctx, GF_EINVAL, "threads_per_site");
        ctx->tps = iv;
    } else if (k == "block") {
        if (!integral || iv < 0 || iv > 256 || (iv % 32)) return fail(ctx, GF_EINVAL, "block: 0 or 32..256 step 32");
        ctx->block = iv;
    } else if (k == "fp64_arith") {
        if (iv != 0 && iv != 1) return fail(ctx, GF_EINVAL, "fp64_arith: 0 (native) or 1 (double-float)");
        if (iv == 1 && ctx->gauge == GF_MAG) return fail(ctx, GF_EINVAL, "fp64_arith: not in the maximally Abelian gauge");
        if (ctx->resident == GF_FP64 && iv != ctx->fp64_arith) ctx->resident = -1;
        ctx->fp64_arith = iv;
    } else if (k == "variant") {
        if (!integral || iv < 0 || iv > 2) return fail(ctx, GF_EINVAL, "variant: 0, 1 or 2");
        ctx->variant = iv;
    } else if (k == "learned_repeat") {
        if (!integral || iv < 0 || iv > 64) return fail(ctx, GF_EINVAL, "learned_repeat: 0..64");
        ctx->learned_repeat = iv;
    } else if (k == "learned_factor") {
        if (!(v > 0.0 && v < 1.0)) return fail(ctx, GF_EINVAL, "learned_factor in (0, 1)");
        ctx->learned_factor = v;
    } else if (k == "fp32_restarts") {
        if (!integral || iv < 0 || iv > 16) return fail(ctx, GF_EINVAL, "fp32_restarts: 0..16");
        ctx->fp32_restarts = iv;
    } else if (k == "theta_per_timeslice") {
        if (v != 0.0 && ctx->gauge == GF_MAG) return fail(ctx, GF_EINVAL, "theta_per_timeslice: not in the maximally Abelian gauge");
        ctx->slice_theta = v != 0.0;
    } else if (k == "or_variant") {
        if (!integral || iv < 0 || iv > 2) return fail(ctx, GF_EINVAL, "or_variant: 0, 1 or 2");
        ctx->or_variant = iv;
    } else if (k == "acc_registers") {
        if (iv != 0 && iv != 255 && iv != 168 && iv != 128) return fail(ctx, GF_EINVAL, "acc_registers: 0, 255, 168 or 128");
        ctx->acc_regs = iv;
    } else if (k == "use_graphs") {
        ctx->use_graphs = v != 0.0;
    } else if (k == "kernel_timing") {
        if (v != 0.0) {
            for (int i = 0; i < 2; ++i)
                if (!ctx->kev[i]) CK(cudaEventCreate(&ctx->kev[i]));
        }
        ctx->kernel_timing = v != 0.0;
    } else if (k == "autotune") {
        ctx->autotune = v != 0.0;
    } else if (k == "track") {
        ctx->track = v != 0.0;
    } else if (k == "stochastic_p") {
        if (!(v >= 0.0 && v <= 1.0)) return fail(ctx, GF_EINVAL, "stochastic_p in [0, 1]");
        if (v > 0.0 && ctx->gauge == GF_MAG) return fail(ctx, GF_EINVAL, "stochastic_p: not in the maximally Abelian gauge");
        ctx->sr_p = v;
    } else if (k == "sr_seed") {
        if (!(v >= 0.0) || v > 18446744073709551615.0) return fail(ctx, GF_EINVAL, "sr_seed");
        ctx->sr_seed = (uint64_t)v;
        ctx->sr_sweep = 0;
    } else if (k == "sa_draw") {
        if (iv != 0 && iv != 1) return fail(ctx, GF_EINVAL, "sa_draw: 0 (FP64 draw) or 1 (FP32 reading)");
        ctx->sa_draw = iv;
    } else if (k == "sa_cap") {
        if (!integral || iv < 1 || iv > 255) return fail(ctx, GF_EINVAL, "sa_cap: 1..255");
        ctx->sa_cap = iv;
    } else if (k == "sa_sweep_offset") {
        if (!(v >= 0.0) || v > 4294967295.0) return fail(ctx, GF_EINVAL, "sa_sweep_offset");
        ctx->sa_sweep_offset = (uint32_t)v;
    } else {
        return fail(ctx, GF_EINVAL, "unknown option " + k);
    }
    return GF_OK;
}

int gf_get_option(const gf_ctx *ctx, const char *key, double *v)
{
    if (!ctx || !key || !v) return GF_EINVAL;
    std::string k(key);
    if (k == "precision") *v = ctx->precision;
    else if (k == "storage64") *v = ctx->storage64;
    else if (k == "storage32") *v = ctx->storage32;
    else if (k == "check_every") *v = ctx->check_every;
    else if (k == "theta_switch") *v = ctx->theta_switch;
    else if (k == "track_gauge") *v = ctx->track_gauge;
    else if (k == "reunitarize_every") *v = ctx->reunit_every;
    else if (k == "threads_per_site") *v = ctx->tps;
    else if (k == "block") *v = ctx->block;
    else if (k == "variant") *v = ctx->variant;
    else if (k == "fp64_arith") *v = ctx->fp64_arith;
    else if (k == "use_graphs") *v = ctx->use_graphs;
    else if (k == "acc_registers") *v = ctx->acc_regs;
    else if (k == "or_variant") *v = ctx->or_variant;
    else if (k == "learned_repeat") *v = ctx->learned_repeat;
    else if (k == "learned_factor") *v = ctx->learned_factor;
    else if (k == "fp32_restarts") *v = ctx->fp32_restarts;
    else if (k == "theta_per_timeslice") *v = ctx->slice_theta;
    else if (k == "kernel_timing") *v = ctx->kernel_timing;
    else if (k == "autotune") *v = ctx->autotune;
    else if (k == "sa_cap") *v = ctx->sa_cap;
    else if (k == "sa_draw") *v = ctx->sa_draw;
    else if (k == "track") *v = ctx->track;
    else if (k == "stochastic_p") *v = ctx->sr_p;
    else if (k == "sr_seed") *v = (double)ctx->sr_seed;
    else if (k == "sa_sweep_offset") *v = ctx->sa_sweep_offset;
    else return GF_EINVAL;
    return GF_OK;
}

int gf_get_stat(const gf_ctx *ctx, const char *key, double *v)
{
    if (!ctx || !key || !v) return GF_EINVAL;
    auto it = ctx->stats.find(key);
    if (it == ctx->stats.end()) return GF_EINVAL;
    *v = it->second;
    return GF_OK;
}

int gf_upload(gf_ctx *ctx, const double *U, int precision)
{
    if (!ctx) return GF_EINVAL;
    if (precision != GF_FP64 && precision != GF_FP32) return fail(ctx, GF_EINVAL, "precision: GF_FP64 or GF_FP32");
    RET(ensure_common(ctx));
    const double *view;
    bool host;
    RET(device_view(ctx, U, &view, &host));
    RET(upload(ctx, view, precision));
    if (host) CK(cudaStreamSynchronize(ctx->stream));
    return GF_OK;
}

int gf_download(gf_ctx *ctx, double *U)
{
    if (!ctx) return GF_EINVAL;
    if (!U || (uintptr_t)U % 16) return fail(ctx, GF_EINVAL, "field pointer NULL or not 16-byte aligned");
    const PtrKind k = pointer_kind(U);
    if (k == PTR_FOREIGN) return fail(ctx, GF_EINVAL, "field is device memory of another device");
    return download(ctx, U, k == PTR_HOST);
}

int gf_or_half_sweep(gf_ctx *ctx, int parity, double omega)
{
    if (!ctx) return GF_EINVAL;
    if (ctx->resident < 0) return fail(ctx, GF_ESTATE, "no resident field");
    if ((parity & ~1) || !(omega > 0.0 && omega < 2.0)) return fail(ctx, GF_EINVAL, "parity 0/1, omega in (0,2)");
    if (ctx->track && !ctx->gt) return fail(ctx, GF_ESTATE, "track is set but no gauge field (gf_gauge_reset)");
    std::pair<int, int> cfg = launch_config(ctx, ctx->resident_fmt);
    SweepArgs a = sweep_args(ctx, resident_base(ctx), parity, omega);
    CK(launch_sweep(ctx->resident_fmt, a, cfg.first, coulomb_of(ctx), or_mode(ctx), ctx->track != 0, cfg.second,
                    ctx->stream));
    return GF_OK;
}

int gf_or_sweeps(gf_ctx *ctx, double omega, int nsweeps)
{
    if (!ctx) return GF_EINVAL;
    if (ctx->resident < 0) return fail(ctx, GF_ESTATE, "no resident field");
    if (nsweeps < 0 || !(omega > 0.0 && omega < 2.0)) return fail(ctx, GF_EINVAL, "nsweeps >= 0, omega in (0,2)");
    if (nsweeps == 0) return GF_OK;
    if (ctx->track && !ctx->gt) return fail(ctx, GF_ESTATE, "track is set but no gauge field (gf_gauge_reset)");
    return run_chunk(ctx, ctx->resident_fmt, resident_base(ctx), omega, nsweeps, ctx->track != 0, false, false);
}

static int mag_unsupported(gf_ctx *ctx, const char *what)
{
    return fail(ctx, GF_EINVAL, std::string(what) + " is not available in the maximally Abelian gauge");
}

int gf_sa_half_sweep(gf_ctx *ctx, int parity, double T, uint64_t seed, uint32_t sweep)
{
    if (!ctx) return GF_EINVAL;
    if (ctx->gauge == GF_MAG) return mag_unsupported(ctx, "annealing");
    if (ctx->resident < 0) return fail(ctx, GF_ESTATE, "no resident field");
    if ((parity & ~1) || !(T > 0.0) || !std::isfinite(T)) return fail(ctx, GF_EINVAL, "parity 0/1, T > 0");
    std::pair<int, int> cfg = launch_config(ctx, ctx->resident_fmt, 1);
    SweepArgs a = sweep_args(ctx, resident_base(ctx), parity, 1.0);
    a.T = T;
    a.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    a.sweep = sweep;
    CK(launch_sweep(ctx->resident_fmt, a, cfg.first, coulomb_of(ctx), 1, false, cfg.second, ctx->stream));
    return GF_OK;
}

int gf_sr_half_sweep(gf_ctx *ctx, int parity, double p, uint64_t seed, uint32_t sweep)
{
    if (!ctx) return GF_EINVAL;
    if (ctx->gauge == GF_MAG) return mag_unsupported(ctx, "stochastic relaxation");
    if (ctx->resident < 0) return fail(ctx, GF_ESTATE, "no resident field");
    if ((parity & ~1) || !(p >= 0.0 && p <= 1.0)) return fail(ctx, GF_EINVAL, "parity 0/1, p in [0, 1]");
    std::pair<int, int> cfg = launch_config(ctx, ctx->resident_fmt);
    SweepArgs a = sweep_args(ctx, resident_base(ctx), parity, 1.0);
    a.prob = p;
    a.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    a.sweep = sweep;
    CK(launch_sweep(ctx->resident_fmt, a, cfg.first, coulomb_of(ctx), 2, false, cfg.second, ctx->stream));
    return GF_OK;
}

int gf_measure_timeslices(gf_ctx *ctx, double *F_t, double *theta_t)
{
    if (!ctx) return GF_EINVAL;
    if (ctx->gauge == GF_MAG) return mag_unsupported(ctx, "per-timeslice measurement");
    if (ctx->resident < 0) return fail(ctx, GF_ESTATE, "no resident field");
    RET(ensure_common(ctx));
    const int Lt = ctx->geom.L[3];
    CK(launch_measure_slices(ctx->resident_fmt, ref(ctx, resident_base(ctx)), ctx->geom, ctx->gauge, ctx->partials,
                             ctx->dslices, ctx->dres, ctx->stream));
    std::vector<double> h(2 * (size_t)Lt);
    CK(cudaMemcpyAsync(h.data(), ctx->dslices, sizeof(double) * 2 * Lt, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    std::vector<double> a(Lt), b(Lt);
    for (int t = 0; t < Lt; ++t) {
        a[t] = h[2 * t];
        b[t] = h[2 * t + 1];
    }
    if (F_t) CK(cudaMemcpy(F_t, a.data(), sizeof(double) * Lt, cudaMemcpyDefault));
    if (theta_t) CK(cudaMemcpy(theta_t, b.data(), sizeof(double) * Lt, cudaMemcpyDefault));
    return GF_OK;
}

int gf_measure(gf_ctx *ctx, double *F_out, double *theta_out)
{
    if (!ctx) return GF_EINVAL;
    return measure_resident(ctx, F_out, theta_out);
}

int gf_reunitarize(gf_ctx *ctx)
{
    if (!ctx) return GF_EINVAL;
    if (ctx->resident < 0) return fail(ctx, GF_ESTATE, "no resident field");
    CK(launch_reunitarize(ctx->resident_fmt, ref(ctx, resident_base(ctx)), ctx->geom, ctx->stream));
    return GF_OK;
}

int gf_autotune(gf_ctx *ctx, int *threads_per_site, int *block)
{
    if (!ctx) return GF_EINVAL;
    if (ctx->resident < 0) return fail(ctx, GF_ESTATE, "no resident field");
    return autotune_format(ctx, ctx->resident_fmt, resident_base(ctx), threads_per_site, block);
}

static int aos_reduce(gf_ctx *ctx, const double *U, int which, double *out)
{
    if (!ctx) return GF_EINVAL;
    if (!out) return fail(ctx, GF_EINVAL, "output pointer is NULL");
    RET(ensure_common(ctx));
    const double *view;
    bool host;
    RET(device_view(ctx, U, &view, &host));
    if (which == 2) CK(launch_plaquette_aos(view, ctx->geom, ctx->partials, ctx->dres, ctx->stream));
    else CK(launch_measure_aos(view, ctx->geom, ctx->gauge, ctx->partials, ctx->dres, ctx->stream));
    CK(cudaMemcpyAsync(ctx->hres, ctx->dres, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *out = which == 1 ? ctx->hres[1] : ctx->hres[0];
    return GF_OK;
}

int gf_functional(gf_ctx *ctx, const double *U, double *F_out) { return aos_reduce(ctx, U, 0, F_out); }
int gf_theta(gf_ctx *ctx, const double *U, double *theta_out) { return aos_reduce(ctx, U, 1, theta_out); }
int gf_plaquette(gf_ctx *ctx, const double *U, double *P_out) { return aos_reduce(ctx, U, 2, P_out); }

int gf_overrelax(gf_ctx *ctx, double *U, double omega, double theta_target, int max_iter, int *iters_out,
                 double *F_out, double *theta_out)
{
    if (!ctx) return GF_EINVAL;
    if (!U) return fail(ctx, GF_EINVAL, "field pointer is NULL");
    if (!(omega > 0.0 && omega < 2.0)) return fail(ctx, GF_EINVAL, "omega must lie in (0, 2)");
    if (!(theta_target >= 0.0) || !std::isfinite(theta_target)) return fail(ctx, GF_EINVAL, "theta_target");
    if (max_iter < 0) return fail(ctx, GF_EINVAL, "max_iter < 0");
    if (ctx->precision == GF_MIXED && ctx->fp32_restarts > 0 && !(ctx->track_gauge && ctx->reunit_every == 1))
        return fail(ctx, GF_EINVAL, "fp32_restarts needs track_gauge 1 and reunitarize_every 1");
    ctx->stats.clear();
    ctx->kms[0] = ctx->kms[1] = 0.0;
    ctx->kn[0] = ctx->kn[1] = 0;
    double t0 = now_ms();
    RET(ensure_common(ctx));
    const double *view;
    bool host;
    RET(device_view(ctx, U, &view, &host));
    // double-float FP64 phase: stages on a working copy of an FP64 field (not
    // with stochastic relaxation, whose sweeps do not track the transformation)
    struct ExactRun {
        gf_ctx *c;
        ~ExactRun() { c->exact_run = false; }
    } exact_guard{ ctx };
    ctx->exact_run = ctx->fp64_arith == 1 && ctx->sr_p == 0.0;

    int used32 = 0, used64 = 0;
    double F = 0.0, theta = 0.0, ms32 = 0.0, ms64 = 0.0;
    if (ctx->precision == GF_FP64) {
        RET(upload(ctx, view, GF_FP64));
        if (ctx->autotune && !tuned(ctx, ctx->resident_fmt))
            RET(autotune_format(ctx, ctx->resident_fmt, ctx->f64, nullptr, nullptr));
        RET(measure_resident(ctx, &F, &theta));
        double t1 = now_ms();
        // 12-real storage: reunitarised at every check (row 2 is rebuilt on every load)
        RET(converge64(ctx, omega, theta_target, max_iter, &used64, &F, &theta));
        ms64 = now_ms() - t1;
    } else {
        bool track = ctx->precision == GF_MIXED && ctx->track_gauge;
        // FP32 restarts: every FP32 stage, the first included, also ends at the FP32 rounding floor
        const bool refine = ctx->precision == GF_MIXED && ctx->fp32_restarts > 0;
        double target32 = ctx->precision == GF_MIXED ? ctx->theta_switch : theta_target;
        if (theta_target > target32) target32 = theta_target;
        RET(upload(ctx, view, GF_FP32));
        if (track) {
            RET(ensure_gauge_field(ctx));
            CK(launch_gauge_identity(ref(ctx, ctx->gt), ctx->geom, ctx->stream));
        }
        if (ctx->autotune && !tuned(ctx, ctx->resident_fmt))
            RET(autotune_format(ctx, ctx->resident_fmt, ctx->f32, nullptr, nullptr));
        RET(measure_resident(ctx, &F, &theta));
        double t1 = now_ms();
        // reunitarise at every check when reunitarize_every == 1 (graph-fused); else every n-th check below
        bool fused = ctx->reunit_every == 1;
        if (fused || ctx->reunit_every == 0) {
            RET(converge(ctx, omega, target32, max_iter, track, fused, &used32, &F, &theta, refine));
        } else {
            int budget = max_iter;
            while (!(theta < target32) && used32 < budget) {
                int chunk_budget = ctx->check_every * ctx->reunit_every;
                if (chunk_budget > budget - used32) chunk_budget = budget - used32;
                int u = 0;
                RET(converge(ctx, omega, target32, chunk_budget, track, false, &u, &F, &theta));
                used32 += u;
                CK(launch_reunitarize(ctx->resident_fmt, ref(ctx, ctx->f32), ctx->geom, ctx->stream));
                if (u == 0) break;
            }
        }
        CK(cudaStreamSynchronize(ctx->stream));
        ms32 = now_ms() - t1;
        if (ctx->precision == GF_MIXED) {
            double t2 = now_ms();
            RET(ensure_field(ctx, GF_FP64));
            if (track) {
                CK(launch_apply_tracked_gauge(view, ref(ctx, ctx->gt), fmt64(ctx), ref(ctx, ctx->f64), ctx->geom,
                                              ctx->stream));
            } else {
                CK(launch_widen(ctx->resident_fmt, ref(ctx, ctx->f32), fmt64(ctx), ref(ctx, ctx->f64), ctx->geom,
                                ctx->stream));
            }
            ctx->resident = GF_FP64;
            ctx->resident_fmt = fmt64(ctx);
            if (ctx->autotune && !tuned(ctx, ctx->resident_fmt))
                RET(autotune_format(ctx, ctx->resident_fmt, ctx->f64, nullptr, nullptr));
            RET(measure_resident(ctx, &F, &theta));
            ctx->stats["theta_switch_measured"] = theta;
            // "fp32_restarts" n > 0: n times, the FP32 field is re-encoded from the FP64 field, g is
            // reset to the identity, the FP32 sweeps run to their rounding floor, and g is applied
            // to the FP64 field in FP64.  Each stage starts g afresh, so the rounding g gathered in
            // the stage before is not carried; the FP64 field stays a gauge transform of the input.
            for (int r = 0; refine && r < ctx->fp32_restarts && theta > 0.0 && !(theta < theta_target); ++r) {
                const double t3 = now_ms();
                const int f32fmt = fmt32(ctx);
                CK(launch_narrow(ctx->resident_fmt, ref(ctx, ctx->f64), f32fmt, ref(ctx, ctx->f32), ctx->geom,
                                 ctx->stream));
                CK(launch_gauge_identity(ref(ctx, ctx->gt), ctx->geom, ctx->stream));
                ctx->resident = GF_FP32;
                ctx->resident_fmt = f32fmt;
                double F32 = 0.0, theta32 = 0.0;
                RET(measure_resident(ctx, &F32, &theta32));
                int u = 0;
                RET(converge(ctx, omega, theta_target, max_iter - used32 - used64, true, true, &u, &F32, &theta32,
                             true));
                used32 += u;
                ctx->resident = GF_FP64;
                ctx->resident_fmt = fmt64(ctx);
                CK(launch_gauge_transform_resident(ctx->resident_fmt, ref(ctx, ctx->f64), ref(ctx, ctx->gt),
                                                   ctx->geom, ctx->stream));
                RET(measure_resident(ctx, &F, &theta));
                ctx->stats["fp32_restarts_done"] += 1;
                ctx->stats["theta_after_restarts"] = theta;
                ctx->stats["ms_restarts"] += now_ms() - t3;
            }
            if (ctx->net && theta > 0.0 && !(theta < theta_target)) {
                double t3 = now_ms();
                RET(learned_correction(ctx, theta));
                RET(measure_resident(ctx, &F, &theta));
                ctx->stats["ms_learned"] = now_ms() - t3;
                ctx->stats["theta_before_learned"] = ctx->stats["theta_switch_measured"];
                ctx->stats["theta_after_learned"] = theta;
            }
            // with "learned_repeat" n > 0 the prediction is applied again each time theta has
            // fallen by a factor learned_factor (at most n more times) before the final stretch
            int repeats = ctx->net ? ctx->learned_repeat : 0;
            while (repeats > 0 && theta > 0.0 && !(theta < theta_target)) {
                const double stage = std::max(theta_target, theta * ctx->learned_factor);
                int u = 0;
                RET(converge64(ctx, omega, stage, max_iter - used32 - used64, &u, &F, &theta));
                used64 += u;
                if (!(theta < stage) || theta < theta_target) break;  // budget spent, or done
                double t3 = now_ms();
                RET(learned_correction(ctx, theta));
                RET(measure_resident(ctx, &F, &theta));
                ctx->stats["ms_learned"] += now_ms() - t3;
                ctx->stats["learned_applications"] += 1;
                --repeats;
            }
            int u = 0;
            RET(converge64(ctx, omega, theta_target, max_iter - used32 - used64, &u, &F, &theta));
            used64 += u;
            ms64 = now_ms() - t2;
        } else {
            CK(launch_reunitarize(ctx->resident_fmt, ref(ctx, ctx->f32), ctx->geom, ctx->stream));
            RET(measure_resident(ctx, &F, &theta));
        }
    }
    RET(download(ctx, U, host));
    CK(cudaStreamSynchronize(ctx->stream));
    std::pair<int, int> cfg = launch_config(ctx, ctx->resident_fmt);
    ctx->stats["sweeps"] = used32 + used64;
    ctx->stats["sweeps_fp32"] = used32;
    ctx->stats["sweeps_fp64"] = used64;
    ctx->stats["ms_fp32"] = ms32;
    ctx->stats["ms_fp64"] = ms64;
    if (ctx->kernel_timing) {
        ctx->stats["ms_sweep_kernels_fp32"] = ctx->kms[0];
        ctx->stats["sweep_launches_fp32"] = (double)ctx->kn[0];
        ctx->stats["ms_sweep_kernels_fp64"] = ctx->kms[1];
        ctx->stats["sweep_launches_fp64"] = (double)ctx->kn[1];
    }
    ctx->stats["ms_total"] = now_ms() - t0;
    ctx->stats["threads_per_site"] = cfg.first > 0 ? cfg.first : 1;
    ctx->stats["accumulate_form"] = cfg.first <= 0;
    ctx->stats["acc_registers"] = cfg.first == GF_ACC_R168 ? 168 : (cfg.first == GF_ACC_R128 ? 128 : 255);
    ctx->stats["block"] = cfg.second;
    if (iters_out) *iters_out = used32 + used64;
    if (F_out) *F_out = F;
    if (theta_out) *theta_out = theta;
    return theta < theta_target ? GF_OK : GF_ENOTCONVERGED;
}

int gf_gauge_reset(gf_ctx *ctx)
{
    if (!ctx) return GF_EINVAL;
    RET(ensure_common(ctx));
    RET(ensure_gauge_field(ctx));
    CK(launch_gauge_identity(ref(ctx, ctx->gt), ctx->geom, ctx->stream));
    return GF_OK;
}

int gf_get_gauge(gf_ctx *ctx, double *g)
{
    if (!ctx || !g) return GF_EINVAL;
    if (!ctx->gt) return fail(ctx, GF_ESTATE, "no tracked gauge field");
    const PtrKind k = pointer_kind(g);
    if (k == PTR_FOREIGN) return fail(ctx, GF_EINVAL, "output is device memory of another device");
    bool host = k == PTR_HOST;
    double *dst = g;
    if (host) {
        RET(ensure_staging(ctx));
        dst = ctx->staging;
    }
    CK(launch_decode_gauge(ref(ctx, ctx->gt), ctx->geom, dst, ctx->stream));
    if (host) CK(cudaMemcpyAsync(g, dst, sizeof(double) * 18 * (size_t)ctx->V, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return GF_OK;
}

int gf_converge(gf_ctx *ctx, double omega, double theta_target, int max_iter, int *iters_out, double *F_out,
                double *theta_out)
{
    if (!ctx) return GF_EINVAL;
    if (ctx->resident < 0) return fail(ctx, GF_ESTATE, "no resident field");
    if (!(omega > 0.0 && omega < 2.0) || !(theta_target >= 0.0) || max_iter < 0)
        return fail(ctx, GF_EINVAL, "omega in (0,2), theta_target >= 0, max_iter >= 0");
    if (ctx->track && !ctx->gt) return fail(ctx, GF_ESTATE, "track is set but no gauge field (gf_gauge_reset)");
    double F = 0.0, theta = 0.0;
    int used = 0;
    RET(measure_resident(ctx, &F, &theta));
    bool reunit = ctx->resident == GF_FP32 && ctx->reunit_every > 0;
    RET(converge(ctx, omega, theta_target, max_iter, ctx->track != 0, reunit, &used, &F, &theta));
    if (iters_out) *iters_out = used;
    if (F_out) *F_out = F;
    if (theta_out) *theta_out = theta;
    return theta < theta_target ? GF_OK : GF_ENOTCONVERGED;
}

int gf_apply_tracked_gauge(gf_ctx *ctx, const double *U)
{
    if (!ctx) return GF_EINVAL;
    if (!ctx->gt) return fail(ctx, GF_ESTATE, "no tracked gauge field");
    const double *view;
    bool host;
    RET(device_view(ctx, U, &view, &host));
    RET(ensure_field(ctx, GF_FP64));
    CK(launch_apply_tracked_gauge(view, ref(ctx, ctx->gt), fmt64(ctx), ref(ctx, ctx->f64), ctx->geom, ctx->stream));
    ctx->resident = GF_FP64;
    ctx->resident_fmt = fmt64(ctx);
    CK(cudaStreamSynchronize(ctx->stream));
    return GF_OK;
}

int gf_features(gf_ctx *ctx, double scale, void *features)
{
    if (!ctx || !features || !(scale > 0.0)) return GF_EINVAL;
    if (ctx->resident != GF_FP64) return fail(ctx, GF_ESTATE, "features need a resident FP64 field");
    if (pointer_kind(features) != PTR_DEVICE) return fail(ctx, GF_EINVAL, "features must be device memory of the current device");
    CK(launch_features(ctx->resident_fmt, ref(ctx, ctx->f64), ctx->geom, 1.0 / scale, features, ctx->stream));
    return GF_OK;
}

int gf_gauge_algebra(gf_ctx *ctx, double scale, float *c)
{
    if (!ctx || !c || !(scale > 0.0)) return GF_EINVAL;
    if (!ctx->gt) return fail(ctx, GF_ESTATE, "no tracked gauge field");
    if (pointer_kind(c) != PTR_DEVICE) return fail(ctx, GF_EINVAL, "output must be device memory of the current device");
    CK(launch_gauge_algebra(ref(ctx, ctx->gt), ctx->geom, 1.0 / scale, c, ctx->stream));
    return GF_OK;
}

int gf_apply_algebra(gf_ctx *ctx, const float *c, double scale)
{
    if (!ctx || !c || !(scale > 0.0)) return GF_EINVAL;
    if (ctx->resident != GF_FP64) return fail(ctx, GF_ESTATE, "needs a resident FP64 field");
    if (pointer_kind(c) != PTR_DEVICE) return fail(ctx, GF_EINVAL, "coefficients must be device memory of the current device");
    RET(ensure_gauge_field(ctx));
    CK(launch_expmap_to_gauge(c, scale, ref(ctx, ctx->gt), ctx->geom, ctx->stream));
    CK(launch_gauge_transform_resident(ctx->resident_fmt, ref(ctx, ctx->f64), ref(ctx, ctx->gt), ctx->geom,
                                       ctx->stream));
    return GF_OK;
}

int gf_set_net(gf_ctx *ctx, gf_net *net)
{
    if (!ctx) return GF_EINVAL;
    if (ctx->gauge != GF_LANDAU && net)
        return fail(ctx, GF_EINVAL, "the learned warm start is defined for Landau gauge (its inputs use the Landau violation)");
    ctx->net = net;
    return GF_OK;
}

int gf_anneal(gf_ctx *ctx, double *U, double T0, double T1, int steps, uint64_t seed)
{
    if (!ctx) return GF_EINVAL;
    if (!U) return fail(ctx, GF_EINVAL, "field pointer is NULL");
    if (ctx->gauge == GF_MAG) return mag_unsupported(ctx, "annealing");
    if (!(T0 > 0.0) || !(T1 > 0.0) || !std::isfinite(T0) || !std::isfinite(T1) || steps < 0)
        return fail(ctx, GF_EINVAL, "temperatures must be positive and finite, steps >= 0");
    ctx->stats.clear();
    double t0 = now_ms();
    RET(ensure_common(ctx));
    const double *view;
    bool host;
    RET(device_view(ctx, U, &view, &host));
    int prec = ctx->precision == GF_FP32 ? GF_FP32 : GF_FP64;
    // fp64_arith 1: the heatbath sweeps run on a double-float copy of the FP64 field with the
    // transformation tracked as E = g - 1 and applied to the FP64 field in FP64 at the end, so the
    // annealed field stays a gauge transform of the input to FP64 rounding
    const bool exact = ctx->fp64_arith == 1 && prec == GF_FP64;
    struct ExactRun {
        gf_ctx *c;
        int xfmt;
        ~ExactRun()
        {
            c->exact_run = false;
            if (c->resident == kResDfWork) {  // an error left the working copy resident
                c->resident = GF_FP64;
                c->resident_fmt = xfmt;
            }
        }
    } exact_guard{ ctx, F64_18 };
    ctx->exact_run = exact;
    RET(upload(ctx, view, prec));
    if (exact) {
        exact_guard.xfmt = ctx->resident_fmt;
        RET(ensure_df_work(ctx));
        CK(launch_to_df(ctx->resident_fmt, ref(ctx, ctx->f64), ref(ctx, ctx->fdf), ctx->geom, ctx->stream));
        CK(cudaMemsetAsync(ctx->ge, 0, 2 * 9 * plane_bytes(ctx), ctx->stream));
        ctx->resident = kResDfWork;
        ctx->resident_fmt = DF64_18;
    }
    if (ctx->autotune && !tuned(ctx, ctx->resident_fmt, 1))
        RET(autotune_format(ctx, ctx->resident_fmt, resident_base(ctx), nullptr, nullptr, 1));
    CK(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int) * 4, ctx->stream));
    std::pair<int, int> cfg = launch_config(ctx, ctx->resident_fmt, 1);
    // 12-real storage rebuilds row 2 from rows 0, 1 on every load; under the
    // large rotations of annealing that feeds unitarity errors back with gain
    // up to 2 per update, so those fields are reunitarised every 4 sweeps
    const bool reunit = twelve_real(ctx->resident_fmt);
    for (int k = 0; k < steps; ++k) {
        double T = steps > 1 ? T0 + (T1 - T0) * (double)k / (double)(steps - 1) : T0;
        for (int p = 0; p < 2; ++p) {
            SweepArgs a = sweep_args(ctx, resident_base(ctx), p, 1.0);
            a.T = T;
            a.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
            a.sweep = ctx->sa_sweep_offset + (uint32_t)k;
            CK(launch_sweep(ctx->resident_fmt, a, cfg.first, coulomb_of(ctx), 1, exact, cfg.second, ctx->stream));
        }
        if (reunit && (k % 4 == 3 || k == steps - 1))
            CK(launch_reunitarize(ctx->resident_fmt, ref(ctx, resident_base(ctx)), ctx->geom, ctx->stream));
    }
    if (exact) {
        ctx->resident = GF_FP64;
        ctx->resident_fmt = exact_guard.xfmt;
        CK(launch_apply_gauge_e(ctx->resident_fmt, ref(ctx, ctx->f64), ref(ctx, ctx->ge), ctx->geom, ctx->stream));
    }
    int rejects = 0;
    CK(cudaMemcpyAsync(ctx->hres + 2, ctx->dstatus, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    RET(download(ctx, U, host));
    CK(cudaStreamSynchronize(ctx->stream));
    memcpy(&rejects, ctx->hres + 2, sizeof(int));
    ctx->stats["sweeps"] = steps;
    ctx->stats["sa_rejects"] = rejects;
    ctx->stats["ms_total"] = now_ms() - t0;
    ctx->stats["threads_per_site"] = cfg.first > 0 ? cfg.first : 1;
    ctx->stats["accumulate_form"] = cfg.first <= 0;
    ctx->stats["acc_registers"] = cfg.first == GF_ACC_R168 ? 168 : (cfg.first == GF_ACC_R128 ? 128 : 255);
    ctx->stats["block"] = cfg.second;
    if (rejects) return fail(ctx, GF_EREJECT, "heatbath rejection cap reached in some draws");
    return GF_OK;
}


// ---------------------------------------------------------------------------
// Wilson-action gauge-field generation (thermalised inputs)
// ---------------------------------------------------------------------------
int gf_wilson_update(gf_ctx *ctx, int mu, int parity, double beta, int mode, uint64_t seed, uint32_t sweep)
{
    if (!ctx) return GF_EINVAL;
    if (ctx->resident != GF_FP64 || ctx->resident_fmt == DF64_18)
        return fail(ctx, GF_ESTATE, "needs a resident FP64 field (storage 18 or 12)");
    if (mu < 0 || mu > 3 || (parity & ~1) || !(beta > 0.0) || !std::isfinite(beta) || (mode != 0 && mode != 1))
        return fail(ctx, GF_EINVAL, "mu 0..3, parity 0/1, beta > 0, mode 0 (heatbath) or 1 (overrelaxation)");
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    CK(launch_wilson(ctx->resident_fmt, ref(ctx, ctx->f64), ctx->geom, mu, parity, beta, mode, key, sweep, ctx->sa_cap,
                     ctx->dstatus, ctx->stream));
    return GF_OK;
}

int gf_generate(gf_ctx *ctx, double *U, double beta, int n_sweeps, int n_or, uint64_t seed, uint32_t sweep0)
{
    if (!ctx) return GF_EINVAL;
    if (!U) return fail(ctx, GF_EINVAL, "field pointer is NULL");
    if (!(beta > 0.0) || !std::isfinite(beta) || n_sweeps < 0 || n_or < 0)
        return fail(ctx, GF_EINVAL, "beta > 0, n_sweeps >= 0, n_or >= 0");
    if (ctx->fp64_arith == 1) return fail(ctx, GF_EINVAL, "generation runs on FP64 storage (fp64_arith 0)");
    ctx->stats.clear();
    double t0 = now_ms();
    RET(ensure_common(ctx));
    const double *view;
    bool host;
    RET(device_view(ctx, U, &view, &host));
    RET(upload(ctx, view, GF_FP64));
    CK(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int) * 4, ctx->stream));
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    FieldRef f = ref(ctx, ctx->f64);
    const bool reunit = twelve_real(ctx->resident_fmt);  // row 2 rebuilt on load: keep rows 0, 1 unitary
    for (int k = 0; k < n_sweeps; ++k) {
        for (int mu = 0; mu < 4; ++mu)
            for (int p = 0; p < 2; ++p)
                CK(launch_wilson(ctx->resident_fmt, f, ctx->geom, mu, p, beta, 0, key, sweep0 + (uint32_t)k,
                                 ctx->sa_cap, ctx->dstatus, ctx->stream));
        for (int o = 0; o < n_or; ++o)
            for (int mu = 0; mu < 4; ++mu)
                for (int p = 0; p < 2; ++p)
                    CK(launch_wilson(ctx->resident_fmt, f, ctx->geom, mu, p, beta, 1, key, 0, ctx->sa_cap,
                                     ctx->dstatus, ctx->stream));
        if (reunit && (k % 4 == 3 || k == n_sweeps - 1))
            CK(launch_reunitarize(ctx->resident_fmt, f, ctx->geom, ctx->stream));
    }
    int rejects = 0;
    CK(cudaMemcpyAsync(ctx->hres + 2, ctx->dstatus, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    RET(download(ctx, U, host));
    CK(cudaStreamSynchronize(ctx->stream));
    memcpy(&rejects, ctx->hres + 2, sizeof(int));
    ctx->stats["sweeps"] = n_sweeps;
    ctx->stats["or_sweeps"] = (double)n_sweeps * n_or;
    ctx->stats["sa_rejects"] = rejects;
    ctx->stats["ms_total"] = now_ms() - t0;
    if (rejects) return fail(ctx, GF_EREJECT, "heatbath rejection cap reached in some draws");
    return GF_OK;
}

}  // extern "C"
