// gf_noalloc.cu -- gf_measure_noalloc: F and theta of a canonical device
// field without any device allocation.
//
// Who needs it: callers that must not call cudaMalloc -- code running while a
// CUDA graph is being captured elsewhere in the process, callers inside a
// framework that owns all device memory through its own pool, and
// memory-budgeted services that forbid allocation after start-up.  The
// context-based gf_functional / gf_theta allocate their reduction scratch on
// first use; this entry point instead keeps its scratch in a fixed
// file-scope device array that every GPU loading the library holds until the
// process exits.
//
// Limits and sharing: the array holds per-block partial sums for at most
// kNoallocMaxBlocks blocks of kNoallocBlock sites, i.e. lattices of up to
// GF_NOALLOC_MAX_SITES sites; larger volumes are rejected with GF_EINVAL.
// Every call on a device uses the same array and leaves its partial sums in
// it; each call overwrites every entry it later reads, so nothing needs
// clearing, but calls whose kernels overlap on the GPU (different streams
// without ordering) race on the array and must be serialised by the caller.
#include <mutex>

#include "gf.h"
#include "gf_device.cuh"
#include "gf_internal.h"

namespace {

using namespace gf;

constexpr int kNoallocBlock = 256;
constexpr int kNoallocMaxBlocks = GF_NOALLOC_MAX_SITES / kNoallocBlock;

// two partial sums (F, theta) per block
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoallocMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices];  // device address of the array, per device

__device__ __forceinline__ void site_of_lex(const Geom &g, int i, int c[4])
{
    int r = i / g.L[0];
    c[0] = i - r * g.L[0];
    int r2 = r / g.L[1];
    c[1] = r - r2 * g.L[1];
    c[3] = r2 / g.L[2];
    c[2] = r2 - c[3] * g.L[2];
}

// D += s (U - U^dagger)/(2i) on the upper triangle of the Hermitian D
__device__ __forceinline__ void accumulate_divergence(const double *u, double s, double dre[3][3],
                                                      double dim[3][3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dre[a][a] += s * u[2 * (4 * a) + 1];
#pragma unroll
        for (int b = a + 1; b < 3; ++b) {
            const double *uab = u + 2 * (3 * a + b), *uba = u + 2 * (3 * b + a);
            dre[a][b] += s * 0.5 * (uab[1] + uba[1]);
            dim[a][b] -= s * 0.5 * (uab[0] - uba[0]);
        }
    }
}

// Per-block partial sums of Re tr U_mu(x) (mu < nk) and of tr[D D^dagger] for
// the traceless part of D(x) = sum_mu [A_mu(x) - A_mu(x - mu)], one site per
// thread, canonical layout.
__global__ void __launch_bounds__(kNoallocBlock) k_measure_noalloc(const double *__restrict__ U, Geom g, int nk,
                                                                   double *partials)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double fsum = 0.0, tsum = 0.0;
    if (i < 2 * g.Vh) {
        int c[4];
        site_of_lex(g, i, c);
        double dre[3][3] = { { 0 } }, dim[3][3] = { { 0 } };
        for (int mu = 0; mu < nk; ++mu) {
            const double *uf = U + (4L * i + mu) * 18;
            fsum += uf[0] + uf[8] + uf[16];
            accumulate_divergence(uf, 1.0, dre, dim);
            int st = lex_stride(g, mu);
            int j = coord_of(c, mu) == 0 ? i + (extent_of(g, mu) - 1) * st : i - st;
            accumulate_divergence(U + (4L * j + mu) * 18, -1.0, dre, dim);
        }
        double tr = (dre[0][0] + dre[1][1] + dre[2][2]) * (1.0 / 3.0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double d = dre[a][a] - tr;
            tsum += d * d;
#pragma unroll
            for (int b = a + 1; b < 3; ++b) tsum += 2.0 * (dre[a][b] * dre[a][b] + dim[a][b] * dim[a][b]);
        }
    }
    __shared__ double sf[kNoallocBlock / 32], st[kNoallocBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fsum += __shfl_down_sync(0xffffffffu, fsum, o);
        tsum += __shfl_down_sync(0xffffffffu, tsum, o);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sf[w] = fsum;
        st[w] = tsum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < kNoallocBlock / 32; ++k) {
            a += sf[k];
            b += st[k];
        }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

// one block: fixed-order sum of the partials, normalised, into out[0..1]
__global__ void __launch_bounds__(kNoallocBlock) k_finish_noalloc(const double *__restrict__ partials, int n,
                                                                  double sF, double sT, double *out)
{
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        a += partials[2 * k];
        b += partials[2 * k + 1];
    }
    __shared__ double ra[kNoallocBlock], rb[kNoallocBlock];
    ra[threadIdx.x] = a;
    rb[threadIdx.x] = b;
    __syncthreads();
    for (int s = kNoallocBlock / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            ra[threadIdx.x] += ra[threadIdx.x + s];
            rb[threadIdx.x] += rb[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = ra[0] * sF;
        out[1] = rb[0] * sT;
    }
}

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the array's name as a device pointer).
int scratch_for_current_device(double **ptr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GF_ECUDA;
    std::lock_guard<std::mutex> lk(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return GF_ECUDA;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *ptr = g_scratch_ptr[dev];
    return GF_OK;
}

}  // namespace

extern "C" int gf_measure_noalloc(const int dims[4], int gauge, const double *U, double *out, void *stream)
{
    if (!dims || !U || !out) return GF_EINVAL;
    if (gauge != GF_LANDAU && gauge != GF_COULOMB) return GF_EINVAL;
    if ((uintptr_t)U % 16 || (uintptr_t)out % 8) return GF_EINVAL;
    long V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2 || (dims[mu] & 1)) return GF_EINVAL;
        V *= dims[mu];
        if (V > GF_NOALLOC_MAX_SITES) return GF_EINVAL;
    }
    // an error left pending by the caller's own earlier work stays theirs: report it, do not clear it
    if (cudaPeekAtLastError() != cudaSuccess) return GF_ECUDA;
    // both must be memory of the current device: the kernels below run there
    if (pointer_kind(U) != PTR_DEVICE || pointer_kind(out) != PTR_DEVICE) return GF_EINVAL;

    double *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != GF_OK) return rc;

    Geom g;
    for (int mu = 0; mu < 4; ++mu) g.L[mu] = dims[mu];
    g.Lh0 = dims[0] / 2;
    g.Vh = (int)(V / 2);
    g.plane = 0;
    int nk = gauge == GF_COULOMB ? 3 : 4;
    int nblocks = (int)((V + kNoallocBlock - 1) / kNoallocBlock);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_measure_noalloc<<<nblocks, kNoallocBlock, 0, s>>>(U, g, nk, scratch);
    if (cudaGetLastError() != cudaSuccess) return GF_ECUDA;
    k_finish_noalloc<<<1, kNoallocBlock, 0, s>>>(scratch, nblocks, 1.0 / (3.0 * nk * (double)V),
                                                 1.0 / (3.0 * (double)V), out);
    return cudaGetLastError() == cudaSuccess ? GF_OK : GF_ECUDA;
}
