// gf_net.cu -- the learned warm-start network: four periodic 4D convolutions
// with 3^4 taps (channels 80 -> 32 -> 32 -> 32 -> 8), ReLU between layers,
// BF16 weights and activations, FP32 accumulation; forward, backward (data
// and weights), mean-squared-error loss and Adam, all on the GPU.
//
// Conventions (as in the oracle): activations X[site][C] with site = x +
// Lx (y + Ly (z + Lz t)); tap k = (dx+1) + 3 (dy+1) + 9 (dz+1) + 27 (dt+1);
// W[k][co][ci]; Y[s][co] = b[co] + sum_k sum_ci W[k][co][ci] X[s + d(k)][ci].
#include <cuda.h>  // CUtensorMap and its enums (the encoder is looked up at run time)
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>

#include "gf.h"
#include "gf_conv_tc.cuh"
#include "gf_device.cuh"
#include "gf_internal.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kC[5] = { GF_NET_CIN, 32, 32, 32, GF_NET_COUT };

struct Lat {
    int L[4];
    int V;
};

__device__ __forceinline__ int shift_site(const Lat &g, int s, int k, int sign)
{
    int c0 = s % g.L[0];
    int r = s / g.L[0];
    int c1 = r % g.L[1];
    r /= g.L[1];
    int c2 = r % g.L[2];
    int c3 = r / g.L[2];
    int d0 = k % 3 - 1, d1 = (k / 3) % 3 - 1, d2 = (k / 9) % 3 - 1, d3 = k / 27 - 1;
    c0 += sign * d0;
    c1 += sign * d1;
    c2 += sign * d2;
    c3 += sign * d3;
    c0 = c0 < 0 ? c0 + g.L[0] : (c0 >= g.L[0] ? c0 - g.L[0] : c0);
    c1 = c1 < 0 ? c1 + g.L[1] : (c1 >= g.L[1] ? c1 - g.L[1] : c1);
    c2 = c2 < 0 ? c2 + g.L[2] : (c2 >= g.L[2] ? c2 - g.L[2] : c2);
    c3 = c3 < 0 ? c3 + g.L[3] : (c3 >= g.L[3] ? c3 - g.L[3] : c3);
    return c0 + g.L[0] * (c1 + g.L[1] * (c2 + g.L[2] * c3));
}

// Set-up of a kernel that needs more than 48 KiB of dynamic shared memory: the attribute is set
// once on each device (bit dev of done), and *nsm gets that device's SM count when asked for.
static cudaError_t kernel_setup(const void *fn, int smem, std::atomic<unsigned long long> &done, int *nsm = nullptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!((done.load() >> dev) & 1ull)) {
        if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
        done.fetch_or(1ull << dev);
    }
    return nsm ? cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, dev) : cudaSuccess;
}

// two floats rounded to BF16, packed low | high
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// ---------------------------------------------------------------------------
// convolution on CUDA cores: Y[s][o] = b[o] + sum_k sum_i Wk[k][o][i] X[s + sign d(k)][i]
// 256 threads: SITES sites x (O / 8) output groups of 8 outputs each.
// Optional epilogue: ReLU, or multiplication by (mask[s][o] > 0).
// ---------------------------------------------------------------------------
template <int I, int O>
__global__ void __launch_bounds__(256) k_conv_cc(const bf16 *__restrict__ X, const bf16 *__restrict__ W,
                                                 const float *__restrict__ bias, Lat g, int sign, int relu,
                                                 const bf16 *__restrict__ mask, bf16 *__restrict__ Yb,
                                                 float *__restrict__ Yf)
{
    constexpr int G = O / 8;             // output groups
    constexpr int SITES = 256 / G;       // sites per block
    __shared__ float xs[SITES][I + 1];
    __shared__ __align__(16) float ws[I][O];
    __shared__ int nbr[SITES];
    const int sl = threadIdx.x % SITES, og = threadIdx.x / SITES;
    const int s0 = blockIdx.x * SITES;
    float acc[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) acc[o] = bias ? bias[og * 8 + o] : 0.0f;
    for (int k = 0; k < 81; ++k) {
        __syncthreads();
        for (int r = threadIdx.x; r < SITES; r += 256) nbr[r] = s0 + r < g.V ? shift_site(g, s0 + r, k, sign) : -1;
        __syncthreads();
        for (int e = threadIdx.x; e < SITES * I; e += 256) {
            int r = e / I, i = e - r * I;
            int nb = nbr[r];
            xs[r][i] = nb >= 0 ? __bfloat162float(X[(long)nb * I + i]) : 0.0f;
        }
        for (int e = threadIdx.x; e < I * O; e += 256) {
            int o = e / I, i = e - o * I;
            ws[i][o] = __bfloat162float(W[((long)k * O + o) * I + i]);
        }
        __syncthreads();
#pragma unroll 4
        for (int i = 0; i < I; ++i) {
            float x = xs[sl][i];
            float4 w0 = *reinterpret_cast<const float4 *>(&ws[i][og * 8]);
            float4 w1 = *reinterpret_cast<const float4 *>(&ws[i][og * 8 + 4]);
            acc[0] += w0.x * x;
            acc[1] += w0.y * x;
            acc[2] += w0.z * x;
            acc[3] += w0.w * x;
            acc[4] += w1.x * x;
            acc[5] += w1.y * x;
            acc[6] += w1.z * x;
            acc[7] += w1.w * x;
        }
    }
    int s = s0 + sl;
    if (s >= g.V) return;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        int oc = og * 8 + o;
        float v = acc[o];
        if (relu) v = v > 0.0f ? v : 0.0f;
        if (mask && !(__bfloat162float(mask[(long)s * O + oc]) > 0.0f)) v = 0.0f;
        if (Yb) Yb[(long)s * O + oc] = __float2bfloat16(v);
        if (Yf) Yf[(long)s * O + oc] = v;
    }
}

// dW[k][o][i] += sum over a chunk of sites of dY[s][o] X[s + d(k)][i];
// db[o] += sum_s dY[s][o] (tap 13 blocks only).  Block = (tap, chunk).
template <int I, int O>
__global__ void __launch_bounds__(256) k_conv_dw(const bf16 *__restrict__ dY, const bf16 *__restrict__ X, Lat g,
                                                 float *__restrict__ dW, float *__restrict__ db)
{
    constexpr int CH = 64;
    constexpr int PER = (I * O + 255) / 256;
    __shared__ float ys[CH][O + 1];
    __shared__ float xs[CH][I + 1];
    __shared__ int nbr[CH];
    const int k = blockIdx.y;
    const int s0 = blockIdx.x * CH;
    if (threadIdx.x < CH) nbr[threadIdx.x] = s0 + threadIdx.x < g.V ? shift_site(g, s0 + threadIdx.x, k, 1) : -1;
    __syncthreads();
    for (int e = threadIdx.x; e < CH * O; e += 256) {
        int r = e / O, o = e - r * O;
        int s = s0 + r;
        ys[r][o] = s < g.V ? __bfloat162float(dY[(long)s * O + o]) : 0.0f;
    }
    for (int e = threadIdx.x; e < CH * I; e += 256) {
        int r = e / I, i = e - r * I;
        xs[r][i] = nbr[r] >= 0 ? __bfloat162float(X[(long)nbr[r] * I + i]) : 0.0f;
    }
    __syncthreads();
    float acc[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) acc[j] = 0.0f;
    for (int r = 0; r < CH; ++r) {
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            int e = threadIdx.x + j * 256;
            if (e < I * O) {
                int o = e / I, i = e - o * I;
                acc[j] += ys[r][o] * xs[r][i];
            }
        }
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        int e = threadIdx.x + j * 256;
        if (e < I * O) atomicAdd(&dW[(long)k * I * O + e], acc[j]);
    }
    if (k == 13 && db && threadIdx.x < O) {
        float a = 0.0f;
        for (int r = 0; r < CH; ++r) a += ys[r][threadIdx.x];
        atomicAdd(&db[threadIdx.x], a);
    }
}

// one warp, fixed order: lane l sums partials l, l + 32, ..., then a shuffle tree
__global__ void k_sum_partials(const double *p, int n, double scale, double *out)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) s += p[i];
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if (threadIdx.x == 0) *out = s * scale;
}

// BF16 copies of the weights W [81][O][I]: W[k][o][i] and Wt[k][i][o] for the
// gather kernels, and the same two blocked by 8 input channels for the halo kernels' TMA
// boxes: Wh[i / 8][k][o][i % 8] and Wth[o / 8][k][i][o % 8] (I, O multiples of 8)
// Row block of tap k = jx + 3 jy + 9 jz + 27 jt in the blocked weight copies used with the
// given sign of the shift: within each dt slab (27 rows) the order is (jy, z block, jx) with z
// block 2 - jz for sign +1 and jz for sign -1.  Then, for one jy, the rows that two adjacent z
// planes of the x-line kernel need from one halo view are adjacent (see k_conv_line_ptc).
__host__ __device__ constexpr int slab_row(int k, int sign)
{
    return 27 * (k / 27) + (k % 3) + 3 * (sign > 0 ? 2 - (k / 9) % 3 : (k / 9) % 3) + 9 * ((k / 3) % 3);
}

// weight e of W [81][O][I] (FP32 value w) into its four BF16 copies
__device__ __forceinline__ void cast_weight(long e, float wf, int I, int O, bf16 *__restrict__ Wb,
                                            bf16 *__restrict__ Wt, bf16 *__restrict__ Wh, bf16 *__restrict__ Wth)
{
    int k = (int)(e / ((long)I * O));
    int r = (int)(e - (long)k * I * O);
    int o = r / I, i = r - o * I;
    bf16 w = __float2bfloat16(wf);
    Wb[e] = w;
    Wt[((long)k * I + i) * O + o] = w;
    Wh[(((long)(i >> 3) * 81 + slab_row(k, 1)) * O + o) * 8 + (i & 7)] = w;
    Wth[(((long)(o >> 3) * 81 + slab_row(k, -1)) * I + i) * 8 + (o & 7)] = w;
}

__global__ void k_cast_weights(const float *__restrict__ W, int I, int O, bf16 *__restrict__ Wb,
                               bf16 *__restrict__ Wt, bf16 *__restrict__ Wh, bf16 *__restrict__ Wth)
{
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long n = 81L * I * O;
    if (e >= n) return;
    cast_weight(e, W[e], I, O, Wb, Wt, Wh, Wth);
}

// the four layers' weight copies, for the Adam kernel
struct WeightCopies {
    long woff[4];
    int I[4], O[4];
    bf16 *Wb[4], *Wt[4], *Wh[4], *Wth[4];
};

// Adam on the FP32 master parameters; an updated weight goes into its BF16 copies at once
// (W[k][o][i], Wt[k][i][o] and the blocked Wh, Wth), as k_cast_weights would write them
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ gr, float *__restrict__ m,
                       float *__restrict__ v, long n, float lr, float b1, float b2, float eps, float c1, float c2,
                       WeightCopies wc)
{
    long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float gi = gr[e];
    float mi = b1 * m[e] + (1.0f - b1) * gi;
    float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    const float pi = p[e] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    p[e] = pi;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const int I = wc.I[l], O = wc.O[l];
        const long r = e - wc.woff[l];
        if (r >= 0 && r < 81L * I * O) cast_weight(r, pi, I, O, wc.Wb[l], wc.Wt[l], wc.Wh[l], wc.Wth[l]);
    }
}


// ---------------------------------------------------------------------------
// convolution on the tensor cores (tcgen05): see gf_conv_tc.cuh
// IP: input channels padded to a multiple of 16; N: output channels padded
// (16 or 32).  X rows have I channels, W is [81][O][I].
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap_coord(int c, int L) { return c < 0 ? c + L : (c >= L ? c - L : c); }

// v[j] for j in {0, 1, 2} without dynamic indexing (stays in registers)
__device__ __forceinline__ int sel3(const int v[3], int j) { return j == 0 ? v[0] : (j == 1 ? v[1] : v[2]); }

template <int IP, int N>
struct TcLayout {
    static constexpr int A_BYTES = gf::tc::kM * IP * 2;
    static constexpr int B_BYTES = N * IP * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int BAR_OFF = gf::tc::kStages * STAGE + gf::tc::kGuardBytes;
    static constexpr int SMEM = BAR_OFF + (gf::tc::kStages + 1) * 8 + 16;
};

template <int IP, int N>
__global__ void __launch_bounds__(128) k_conv_tc(const bf16 *__restrict__ X, int I, const bf16 *__restrict__ W, int O,
                                                 const float *__restrict__ bias, Lat g, int sign, int relu,
                                                 const bf16 *__restrict__ mask, bf16 *__restrict__ Yb,
                                                 float *__restrict__ Yf, int *__restrict__ err)
{
    using namespace gf::tc;
    typedef TcLayout<IP, N> LY;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + LY::BAR_OFF);  // kStages + 1 (final)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + LY::BAR_OFF + (kStages + 1) * 8);
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int s0 = blockIdx.x * kM;
    constexpr uint32_t idesc = instr_desc(kM, N);

    if (tid == 0) {
        for (int st = 0; st <= kStages; ++st) mbar_init(&bar[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    const int site = s0 + tid;
    // neighbour of this row's site for tap k = (d0+1) + 3 (d1+1) + 9 (d2+1) +
    // 27 (d3+1): the sum over dimensions of the wrapped coordinate c + sign d
    // times its stride, the 12 terms formed once
    int o0[3], o1[3], o2[3], o3[3];
    {
        int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
        if (site < g.V) {
            c0 = site % g.L[0];
            int r = site / g.L[0];
            c1 = r % g.L[1];
            r /= g.L[1];
            c2 = r % g.L[2];
            c3 = r / g.L[2];
        }
        const int st1 = g.L[0], st2 = g.L[0] * g.L[1], st3 = st2 * g.L[2];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int d = sign * (j - 1);
            o0[j] = wrap_coord(c0 + d, g.L[0]);
            o1[j] = wrap_coord(c1 + d, g.L[1]) * st1;
            o2[j] = wrap_coord(c2 + d, g.L[2]) * st2;
            o3[j] = wrap_coord(c3 + d, g.L[3]) * st3;
        }
    }
    constexpr int AC = IP / 8;                                  // 16-byte chunks of one A row
    constexpr int WPT = (N * (IP / 8) + kThreads - 1) / kThreads;  // weight chunks per thread
    uint4 cur[AC], nxt[AC], wcur[WPT], wnxt[WPT];
    // global loads of tap k's A row and B chunks into registers
    auto fetch = [&](int k, uint4 *a, uint4 *w) {
        const int nbs = site < g.V ? sel3(o0, k % 3) + sel3(o1, (k / 3) % 3) + sel3(o2, (k / 9) % 3) + sel3(o3, k / 27)
                                   : -1;
#pragma unroll
        for (int c = 0; c < AC; ++c) {
            a[c] = make_uint4(0, 0, 0, 0);
            if (nbs >= 0 && 8 * c < I) a[c] = *reinterpret_cast<const uint4 *>(X + (long)nbs * I + 8 * c);
        }
#pragma unroll
        for (int q = 0; q < WPT; ++q) {
            const int e = tid + q * kThreads;
            const int o = e / (IP / 8), c = e - o * (IP / 8);
            w[q] = make_uint4(0, 0, 0, 0);
            if (e < N * (IP / 8) && o < O && 8 * c < I)
                w[q] = *reinterpret_cast<const uint4 *>(W + ((long)k * O + o) * I + 8 * c);
        }
    };
    fetch(0, cur, wcur);
    bool fail = false;
    for (int k = 0; k < 81; ++k) {
        const int st = k % kStages;
        if (k + 1 < 81) fetch(k + 1, nxt, wnxt);  // in flight while tap k is staged
        if (k >= kStages) {
            if (!mbar_wait(&bar[st], (uint32_t)((k / kStages - 1) & 1))) fail = true;
        }
        if (__syncthreads_or(fail)) {
            fail = true;
            break;
        }
        uint8_t *A = smem + st * LY::STAGE;
        uint8_t *B = A + LY::A_BYTES;
        // A: this thread's neighbour row, K-major core matrices (8 rows x 16 B):
        // core (mr, kc) at (kc * 16 + mr) * 128  -> SBO 128, LBO 2048
#pragma unroll
        for (int c = 0; c < AC; ++c) *reinterpret_cast<uint4 *>(A + (c * 16 + (tid >> 3)) * 128 + (tid & 7) * 16) = cur[c];
        // B: weights of tap k, core (mr, kc) at (kc * (N/8) + mr) * 128 -> SBO 128, LBO N*16
#pragma unroll
        for (int q = 0; q < WPT; ++q) {
            const int e = tid + q * kThreads;
            if (e < N * (IP / 8)) {
                const int o = e / (IP / 8), c = e - o * (IP / 8);
                *reinterpret_cast<uint4 *>(B + (c * (N / 8) + (o >> 3)) * 128 + (o & 7) * 16) = wcur[q];
            }
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < IP / 16; ++kk) {
                uint64_t ad = smem_desc(smem_u32(A + kk * 2 * 2048), 2048, 128);
                uint64_t bd = smem_desc(smem_u32(B + kk * 2 * (N / 8) * 128), (N / 8) * 128, 128);
                mma_bf16(tmem, ad, bd, idesc, (k | kk) != 0);
            }
            mma_commit(&bar[st]);
        }
#pragma unroll
        for (int c = 0; c < AC; ++c) cur[c] = nxt[c];
#pragma unroll
        for (int q = 0; q < WPT; ++q) wcur[q] = wnxt[q];
    }
    // all MMAs issued by thread 0 are complete once the final commit arrives
    if (tid == 0) mma_commit(&bar[kStages]);
    if (!mbar_wait(&bar[kStages], 0)) fail = true;
    fail = __syncthreads_or(fail);
    if (!fail) {
        fence_after_sync();
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        if (N == 32) {
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
        } else {
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
                " [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (site < g.V) {
#pragma unroll
            for (int o = 0; o < N; ++o) {
                if (o >= O) break;
                float v = __uint_as_float(r[o]) + (bias ? bias[o] : 0.0f);
                if (relu) v = v > 0.0f ? v : 0.0f;
                if (mask && !(__bfloat162float(mask[(long)site * O + o]) > 0.0f)) v = 0.0f;
                if (Yb) Yb[(long)site * O + o] = __float2bfloat16(v);
                if (Yf) Yf[(long)site * O + o] = v;
            }
        }
    } else if (tid == 0) {
        atomicExch(err, GF_ETIMEOUT);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
    }
}

template <int IP, int N>
cudaError_t conv_tc(const bf16 *X, int I, const bf16 *W, int O, const float *b, const Lat &g, int sign, int relu,
                    const bf16 *mask, bf16 *Yb, float *Yf, int *err, cudaStream_t s)
{
    typedef TcLayout<IP, N> LY;
    static std::atomic<unsigned long long> configured{ 0 };
    cudaError_t e = kernel_setup((const void *)k_conv_tc<IP, N>, LY::SMEM, configured);
    if (e != cudaSuccess) return e;
    k_conv_tc<IP, N><<<(g.V + gf::tc::kM - 1) / gf::tc::kM, gf::tc::kThreads, LY::SMEM, s>>>(X, I, W, O, b, g, sign,
                                                                                          relu, mask, Yb, Yf, err);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// halo-tile convolution on the tensor cores (net option "conv_halo"): a CTA
// computes an 8 (x) x 16 (y) x 2 (z) tile of one t, two accumulators of
// M = 128 rows (row r = x + 8 y, one per z plane).  A phase is one 16-channel
// chunk of the input and one slab of 27 taps (fixed dt); those taps read only
// one t-plane of the tile's periodic halo (18 x 4 lines of 10 sites), which the
// phase stages in shared memory K-major without swizzle: the 8 consecutive x
// positions of a y line form one core matrix (8 rows x 16 B), consecutive y
// lines are 160 B apart (SBO) and the two 8-channel core columns one plane half
// apart (LBO).  The A operand of tap d and plane z is then the same array from
// another start address, so nothing is gathered per tap; the slab's weights
// serve both planes.  (Aligned x-shifted copies double the MMA rate but triple
// the halo bytes or need a copy pass; measured, both were slower than this
// layout, which keeps shared memory small enough for two CTAs per SM.)
// Staging is TMA (cp.async.bulk.tensor): the input is first copied into a
// buffer with one periodic ghost site on each side of every dimension
// (k_pad_periodic), so every halo plane is one in-range 5D box {8 channels,
// 10 x, 18 y, 4 z, 1 t} and the slab's weights one 3D box {8 channels, N
// outputs, 27 taps} per 8-channel half; channels past the input's and rows past the
// outputs' are filled with zeros by the TMA unit.  One thread drives the
// pipeline: the boxes of phase n + 1 land in the other buffers (mbarrier with
// expected bytes) while the MMAs of phase n run, and a buffer is refilled once
// the MMAs that read it have completed (tcgen05.commit).  Every wait is
// bounded.  Needs Lx % 8 == 0, Ly % 16 == 0 and Lz % 2 == 0; other lattices use
// k_conv_tc.
// ---------------------------------------------------------------------------
namespace halo {
constexpr int TX = 8, TY = 16, TZ = 2;
constexpr int HY = TY + 2, HZ = TZ + 2;
constexpr int HX = TX + 2;             // sites of one halo line
constexpr int NL = HY * HZ;            // lines (y, z) of one t-plane of the halo
constexpr int RAW = NL * HX * 16;      // one 8-channel half of a halo t-plane (one TMA box)
constexpr int LBO_A = RAW;             // between the two 8-channel core columns
constexpr int SBO_A = HX * 16;         // between consecutive y lines (8-row groups)
constexpr int A_BYTES = 2 * RAW;       // one phase: a halo t-plane
constexpr int THREADS = 256;           // warps w and w + 4 read one TMEM lane quarter (two planes)
}  // namespace halo

template <int N>
struct HaloLayout {
    static constexpr int W_HALF = 27 * N * 16;        // one 8-channel half of a slab: [tap][o][8 channels]
    static constexpr int W_BYTES = 2 * W_HALF;
    static constexpr int B_OFF = 2 * halo::A_BYTES;
    // bar[0..1]: boxes of even / odd phases landed; bar[2..3]: MMAs of even / odd phases done; bar[4]: drain
    static constexpr int BAR_OFF = B_OFF + 2 * W_BYTES;
    static constexpr int SMEM = BAR_OFF + 5 * 8 + 8 + 16;
    static constexpr int TMEM_COLS = halo::TZ * N < 32 ? 32 : halo::TZ * N;
    static constexpr uint32_t TX_BYTES = halo::A_BYTES + W_BYTES;  // bytes the boxes of one phase deliver
};

static bool halo_ok(const Lat &g)
{
    return g.L[0] % halo::TX == 0 && g.L[1] % halo::TY == 0 && g.L[2] % halo::TZ == 0;
}

// sites of the ghost-padded lattice: (Lx + 2 gx)(Ly + 2)(Lz + 2)(Lt + 2), gx = 1
// with ghosts in x, 0 without
static long padded_sites(const Lat &g, int gx = 1)
{
    return (long)(g.L[0] + 2 * gx) * (g.L[1] + 2) * (g.L[2] + 2) * (g.L[3] + 2);
}

// Xp = X with one periodic ghost site on each side of y, z, t (and of x when
// gx = 1), blocked by 8 channels so that a TMA box row is a contiguous run:
// Xp[c][pt][pz][py][px][8] holds channels 8 c .. 8 c + 7 of site
// ((px - gx) mod Lx, (py - 1) mod Ly, (pz - 1) mod Lz, (pt - 1) mod Lt).  One
// thread per padded site: it reads the site's I channels (contiguous) and
// writes one 16-byte piece per group, consecutive threads side by side.
__global__ void k_pad_periodic(const bf16 *__restrict__ X, int I, Lat g, int gx, bf16 *__restrict__ Xp)
{
    const int G = I / 8;
    const int Px = g.L[0] + 2 * gx, Py = g.L[1] + 2, Pz = g.L[2] + 2;
    const long P = (long)Px * Py * Pz * (g.L[3] + 2);
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (long)gridDim.x * blockDim.x) {
        long p = e;
        const int px = (int)(p % Px);
        p /= Px;
        const int py = (int)(p % Py);
        p /= Py;
        const int pz = (int)(p % Pz);
        const int pt = (int)(p / Pz);
        const long zt = wrap_coord(pz - 1, g.L[2]) + (long)g.L[2] * wrap_coord(pt - 1, g.L[3]);
        const long s = wrap_coord(px - gx, g.L[0]) + (long)g.L[0] * (wrap_coord(py - 1, g.L[1]) + (long)g.L[1] * zt);
        const uint4 *src = reinterpret_cast<const uint4 *>(X + s * I);
        uint4 *dst = reinterpret_cast<uint4 *>(Xp) + e;
        for (int c = 0; c < G; ++c) dst[(long)c * P] = src[c];
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(gf::tc::smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(gf::tc::smem_u32(bar)) : "memory");
}

// untiled bulk copy of bytes (a multiple of 16) from global to shared memory, completing on bar
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     gf::tc::smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(gf::tc::smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            gf::tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(gf::tc::smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(gf::tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(gf::tc::smem_u32(bar))
        : "memory");
}

// bounded wait for a barrier phase with a pause between polls (threads that
// only wait for the end do not take issue slots from the one that works)
__device__ __forceinline__ bool mbar_wait_idle(uint64_t *bar, uint32_t parity)
{
    const long long t0 = gf::tc::now_ns();
    while (!gf::tc::mbar_try_wait(bar, parity)) {
        if (gf::tc::now_ns() - t0 > gf::tc::kWaitNs) return false;
        __nanosleep(500);
    }
    return true;
}

// 32 (N = 32) or 16 (N = 16) accumulator columns of this warp's lane quarter, as floats
template <int N>
__device__ __forceinline__ void tmem_load_cols(uint32_t taddr, float *v)
{
    uint32_t r[N];
    if (N == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
            " [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int o = 0; o < N; ++o) v[o] = __uint_as_float(r[o]);
}

// coordinate c on an axis of extent L >= 3 with gh ghost sites on each side (padded index p
// holds (p - gh) mod L) sits at padded index c + gh and, when gh = 1 and c is on a face, at
// the ghost on the far side: image 1 is that ghost's index, or -1
__device__ __forceinline__ int padded_image(int i, int c, int L, int gh)
{
    if (i == 0) return c + gh;
    return !gh ? -1 : c == L - 1 ? 0 : c == 0 ? L + 1 : -1;
}

// One row of a convolution's output (site (x, y, z, t), O channels in acc) into
// the ghost-padded copy that the next convolution reads, blocked by 8
// channels: Yp[c][pt][pz][py][px][8] with gx ghost sites in x and one in y, z
// and t (the layout k_pad_periodic writes).  The row goes to every padded
// position holding the site, so no copy pass is needed.  Lanes with
// consecutive x write consecutive 16-byte pieces.
template <int N>
__device__ __forceinline__ void store_padded_row(const float (&acc)[N], int O, bf16 *__restrict__ Yp, int gx,
                                                 const Lat &g, int x, int y, int z, int t)
{
    const int Px = g.L[0] + 2 * gx, Py = g.L[1] + 2, Pz = g.L[2] + 2;
    const long P = (long)Px * Py * Pz * (g.L[3] + 2);
    uint4 u[N / 8];
#pragma unroll
    for (int c = 0; c < N / 8; ++c) {
        u[c].x = pack_bf16x2(acc[8 * c + 0], acc[8 * c + 1]);
        u[c].y = pack_bf16x2(acc[8 * c + 2], acc[8 * c + 3]);
        u[c].z = pack_bf16x2(acc[8 * c + 4], acc[8 * c + 5]);
        u[c].w = pack_bf16x2(acc[8 * c + 6], acc[8 * c + 7]);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(Yp);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int pt = padded_image(it, t, g.L[3], 1);
        if (pt < 0) continue;
#pragma unroll
        for (int iz = 0; iz < 2; ++iz) {
            const int pz = padded_image(iz, z, g.L[2], 1);
            if (pz < 0) continue;
#pragma unroll
            for (int iy = 0; iy < 2; ++iy) {
                const int py = padded_image(iy, y, g.L[1], 1);
                if (py < 0) continue;
                const long line = (((long)pt * Pz + pz) * Py + py) * Px;
#pragma unroll
                for (int ix = 0; ix < 2; ++ix) {
                    const int px = padded_image(ix, x, g.L[0], gx);
                    if (px < 0) continue;
#pragma unroll
                    for (int c = 0; c < N / 8; ++c)
                        if (c < O / 8) dst[(long)c * P + line + px] = u[c];
                }
            }
        }
    }
}

// Knuth's two-sum: s + e == a + b exactly (round to nearest, no reassociation)
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// The loss partials and dY of the last layer, one site (8 outputs) per step:
// d = out - target in FP32, dY = 2 d / n in BF16, and sum d^2 into partial[block].
// Each square is an exact pair p + e (p = d d rounded, e = fma(d, d, -p)); a
// site's 8 pairs are summed in FP32 with two-sum (the rounding errors collected
// in a second word), and the two words enter the thread's FP64 accumulator:
// four operations of the slow FP64 pipe per site instead of 16.  Exact where the
// sums fit in the two words; else the site sum is off by a few units of 2^-48 of it.
// PADDED: dY goes into the ghost-padded copy with x ghosts, one channel group
// (the layout k_pad_periodic writes), at every padded position of the site.
template <bool PADDED>
__global__ void k_mse(const float *__restrict__ out, const float *__restrict__ t, Lat g, float inv_n,
                      bf16 *__restrict__ dout, double *__restrict__ partial)
{
    double acc = 0.0;
    for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += (long)gridDim.x * blockDim.x) {
        const float4 *o4 = reinterpret_cast<const float4 *>(out) + 2 * s;
        const float4 *y4 = reinterpret_cast<const float4 *>(t) + 2 * s;
        const float4 oa = o4[0], ob = o4[1], ya = y4[0], yb = y4[1];
        float d[8] = { oa.x - ya.x, oa.y - ya.y, oa.z - ya.z, oa.w - ya.w,
                       ob.x - yb.x, ob.y - yb.y, ob.z - yb.z, ob.w - yb.w };
        float hi = 0.0f, lo = 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float p = __fmul_rn(d[j], d[j]);
            const float e = __fmaf_rn(d[j], d[j], -p);
            float r;
            two_sum_f(hi, p, hi, r);
            lo = __fadd_rn(lo, __fadd_rn(r, e));
        }
        acc += (double)hi;
        acc += (double)lo;
        float gr[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) gr[j] = 2.0f * d[j] * inv_n;
        if (PADDED) {
            const int x = (int)(s % g.L[0]);
            long r = s / g.L[0];
            const int y = (int)(r % g.L[1]);
            r /= g.L[1];
            store_padded_row<8>(gr, 8, dout, 1, g, x, y, (int)(r % g.L[2]), (int)(r / g.L[2]));
        } else {
            uint4 u;
            u.x = pack_bf16x2(gr[0], gr[1]);
            u.y = pack_bf16x2(gr[2], gr[3]);
            u.z = pack_bf16x2(gr[4], gr[5]);
            u.w = pack_bf16x2(gr[6], gr[7]);
            reinterpret_cast<uint4 *>(dout)[s] = u;
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// The epilogue of one warp's 32 accumulator rows (row r of the warp is the
// site site_of(r); this thread holds row lane in acc): bias, ReLU, the mask,
// then BF16 (Yb) or FP32 (Yf) rows of O channels.  Mask and output rows pass
// through the warp's staging area in shared memory (32 rows of at most 128 B),
// so global memory is read and written in 16-byte pieces at consecutive
// addresses: one 2-byte access per channel made an L2 request per element.
template <int N, typename SiteOf>
__device__ __forceinline__ void epilogue_rows(float (&acc)[N], int O, const float *__restrict__ bias, int relu,
                                              const bf16 *__restrict__ mask, bf16 *__restrict__ Yb,
                                              float *__restrict__ Yf, uint4 *stage, int lane, SiteOf site_of)
{
#pragma unroll
    for (int o = 0; o < N; ++o) {
        float v = acc[o] + (bias && o < O ? bias[o] : 0.0f);
        acc[o] = relu && !(v > 0.0f) ? 0.0f : v;
    }
    if (mask) {
        const int cpr = O / 8;  // 16-byte pieces of a BF16 row
        for (int c = lane; c < 32 * cpr; c += 32)
            stage[c] = reinterpret_cast<const uint4 *>(mask + site_of(c / cpr) * O)[c % cpr];
        __syncwarp();
        const bf16 *m = reinterpret_cast<const bf16 *>(stage + lane * cpr);
#pragma unroll
        for (int o = 0; o < N; ++o)
            if (o < O && !(__bfloat162float(m[o]) > 0.0f)) acc[o] = 0.0f;
        __syncwarp();
    }
    if (Yb) {
        const int cpr = O / 8;
#pragma unroll
        for (int c = 0; c < N / 8; ++c) {
            if (c < cpr) {
                uint4 u;
                u.x = pack_bf16x2(acc[8 * c + 0], acc[8 * c + 1]);
                u.y = pack_bf16x2(acc[8 * c + 2], acc[8 * c + 3]);
                u.z = pack_bf16x2(acc[8 * c + 4], acc[8 * c + 5]);
                u.w = pack_bf16x2(acc[8 * c + 6], acc[8 * c + 7]);
                stage[lane * cpr + c] = u;
            }
        }
        __syncwarp();
        for (int c = lane; c < 32 * cpr; c += 32)
            reinterpret_cast<uint4 *>(Yb + site_of(c / cpr) * O)[c % cpr] = stage[c];
        __syncwarp();
    }
    if (Yf) {
        const int cpr = O / 4;  // 16-byte pieces of an FP32 row
#pragma unroll
        for (int c = 0; c < N / 4; ++c)
            if (c < cpr)
                stage[lane * cpr + c] = make_uint4(__float_as_uint(acc[4 * c + 0]), __float_as_uint(acc[4 * c + 1]),
                                                   __float_as_uint(acc[4 * c + 2]), __float_as_uint(acc[4 * c + 3]));
        __syncwarp();
        for (int c = lane; c < 32 * cpr; c += 32)
            reinterpret_cast<uint4 *>(Yf + site_of(c / cpr) * O)[c % cpr] = stage[c];
        __syncwarp();
    }
}

template <int IP, int N>
__global__ void __launch_bounds__(halo::THREADS) k_conv_halo_tc(const __grid_constant__ CUtensorMap tx,
                                                                const __grid_constant__ CUtensorMap tw, int O,
                                                                const float *__restrict__ bias, Lat g, int sign,
                                                                int relu, const bf16 *__restrict__ mask,
                                                                bf16 *__restrict__ Yb, float *__restrict__ Yf,
                                                                int *__restrict__ err)
{
    using namespace gf::tc;
    using namespace halo;
    typedef HaloLayout<N> LY;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + LY::BAR_OFF);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + LY::BAR_OFF + 40);
    const int tid = threadIdx.x, warp = tid >> 5;
    constexpr uint32_t idesc = instr_desc(kM, N);
    constexpr int NPHASE = (IP / 16) * 3;  // (16-channel chunk, dt slab)

    int b = blockIdx.x;
    const int nbx = g.L[0] / TX, nby = g.L[1] / TY, nbz = g.L[2] / TZ;
    const int x0 = (b % nbx) * TX;
    b /= nbx;
    const int y0 = (b % nby) * TY;
    b /= nby;
    const int z0 = (b % nbz) * TZ;
    const int t0 = b / nbz;

    if (tid == 0) {
        for (int k = 0; k < 5; ++k) mbar_init(&bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(LY::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    bool fail = false;
    if (tid == 0) {
        // the boxes of phase ph into buffer ph & 1: the halo t-plane read by the slab's taps
        // (dt = sign (slab - 1)) in padded coordinates (halo x0 - 1 is padded x0; the plane of
        // channel group c at t is c Pt + t), one box per 8-channel half, then the slab's weights
        auto issue = [&](int ph) {
            const int buf = ph & 1, ch0 = 16 * (ph / 3), slab = ph % 3;
            const int ht = sign > 0 ? slab : 2 - slab;
            uint64_t *full = &bar[buf];
            mbar_expect_tx(full, LY::TX_BYTES);
            uint8_t *A = smem + buf * A_BYTES;
#pragma unroll
            for (int kc = 0; kc < 2; ++kc)
                tma_load_4d(A + kc * LBO_A, &tx, 8 * x0, y0, z0, (ch0 / 8 + kc) * (g.L[3] + 2) + t0 + ht, full);
            uint8_t *B = smem + LY::B_OFF + buf * LY::W_BYTES;
#pragma unroll
            for (int kc = 0; kc < 2; ++kc) tma_load_3d(B + kc * LY::W_HALF, &tw, 0, 27 * slab, ch0 / 8 + kc, full);
        };
        int issued = 0, landed = 0;
        issue(0);
        issued = 1;
        for (int ph = 0; ph < NPHASE; ++ph) {
            const int nx = ph + 1;
            if (nx < NPHASE) {
                // the buffers of phase nx were last read by the MMAs of phase ph - 1
                if (ph > 0 && !mbar_wait(&bar[2 + ((ph - 1) & 1)], (uint32_t)(((ph - 1) >> 1) & 1))) {
                    fail = true;
                    break;
                }
                issue(nx);
                issued = nx + 1;
            }
            if (!mbar_wait(&bar[ph & 1], (uint32_t)((ph >> 1) & 1))) {  // the boxes of phase ph have landed
                fail = true;
                break;
            }
            landed = ph + 1;
            fence_after_sync();
            const uint8_t *A = smem + (ph & 1) * A_BYTES;
            const uint8_t *B = smem + LY::B_OFF + (ph & 1) * LY::W_BYTES;
            for (int j = 0; j < 27; ++j) {
                const int dx = sign * (j % 3 - 1), dy = sign * ((j / 3) % 3 - 1), dz = sign * (j / 9 - 1);
                const uint64_t bd = smem_desc(smem_u32(B + slab_row(j, sign) * N * 16), LY::W_HALF, 128);
#pragma unroll
                for (int zz = 0; zz < TZ; ++zz) {
                    // first halo line of the shifted tile of plane zz; x offset dx + 1 within the line
                    const int l0 = (dy + 1) + HY * (zz + dz + 1);
                    const uint64_t ad = smem_desc(smem_u32(A + (l0 * HX + dx + 1) * 16), LBO_A, SBO_A);
                    mma_bf16(tmem + (uint32_t)(zz * N), ad, bd, idesc, (ph | j) != 0);
                }
            }
            mma_commit(&bar[2 + (ph & 1)]);
        }
        // boxes issued but not consumed must land before the CTA ends (bounded)
        for (int q = landed; q < issued; ++q)
            if (!mbar_wait(&bar[q & 1], (uint32_t)((q >> 1) & 1))) fail = true;
        mma_commit(&bar[4]);  // arrives once every MMA issued above is complete
    }
    // everyone: all MMAs complete (bounded wait), then the epilogue
    const bool drained = mbar_wait_idle(&bar[4], 0);
    fail = __syncthreads_or(fail || !drained);
    if (!fail) {
        fence_after_sync();
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 of plane w / 4; accumulator row = x + 8 y
        const int zz = warp >> 2, q = warp & 3;
        float acc[N];
        tmem_load_cols<N>(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(zz * N), acc);
        const long plane = (long)g.L[1] * ((z0 + zz) + (long)g.L[2] * t0);
        auto site_of = [&](int r) {
            const int row = q * 32 + r;
            return (long)(x0 + (row & 7)) + (long)g.L[0] * ((y0 + (row >> 3)) + plane);
        };
        // the A buffers are free once every MMA has completed
        epilogue_rows<N>(acc, O, bias, relu, mask, Yb, Yf, reinterpret_cast<uint4 *>(smem) + warp * 256,
                         tid & 31, site_of);
    } else if (tid == 0) {
        atomicExch(err, GF_ETIMEOUT);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(LY::TMEM_COLS)
                     : "memory");
    }
}

// the tensor-map encoder of the driver, looked up once through the runtime (no link to the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// Pads X [V][I] (I a multiple of 8) into xpad (blocked by 8 channels, x ghosts
// when gx = 1; skipped when padded is set because xpad already holds it) and
// encodes the tensor maps of the halo kernels.  A line of x
// and its 8 channels are contiguous in xpad, and so are the rows o of a tap and
// their 8 channels in the blocked weights, so each is one inner dimension and
// a box row is a contiguous run (a TMA request per 16-byte row would bind the
// L2): tx over xpad as {8 Px, Py, Pz, (I / 8) Pt} with box {8 bx, by, bz, 1},
// tw over Wblk[I / 8][81][O][8] as {8 O, 81, I / 8} with box {8 N, 27, 1}.
// Channel groups past I / 8 and rows past O are outside the maps: the TMA unit
// fills them with zeros.
static cudaError_t halo_prepare(const bf16 *X, int I, const bf16 *Wblk, int O, int N, const Lat &g, int gx, int bx,
                                int by, int bz, bf16 *xpad, cudaStream_t s, CUtensorMap *tx, CUtensorMap *tw,
                                bool padded = false)
{
    const EncodeTiledFn enc = encode_tiled();
    if (!enc || !xpad) return cudaErrorNotSupported;
    if (!padded) {  // padded: xpad already holds X so padded
        const long P = padded_sites(g, gx);
        const int pblocks = (int)std::min<long>((P + 255) / 256, 152L * 32);
        k_pad_periodic<<<pblocks, 256, 0, s>>>(X, I, g, gx, xpad);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const cuuint64_t es = sizeof(bf16);
    const cuuint64_t Px = g.L[0] + 2 * gx, Py = g.L[1] + 2, Pz = g.L[2] + 2, Pt = g.L[3] + 2;
    const cuuint64_t xdim[4] = { 8 * Px, Py, Pz, (cuuint64_t)(I / 8) * Pt };
    const cuuint64_t xstr[3] = { 8 * es * Px, 8 * es * Px * Py, 8 * es * Px * Py * Pz };
    const cuuint32_t xbox[4] = { (cuuint32_t)(8 * bx), (cuuint32_t)by, (cuuint32_t)bz, 1 };
    const cuuint32_t ones[4] = { 1, 1, 1, 1 };
    const cuuint64_t wdim[3] = { 8 * (cuuint64_t)O, 81, (cuuint64_t)(I / 8) };
    const cuuint64_t wstr[2] = { 8 * es * O, 8 * es * O * 81 };
    const cuuint32_t wbox[3] = { (cuuint32_t)(8 * N), 27, 1 };
    if (enc(tx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, xpad, xdim, xstr, xbox, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS ||
        enc(tw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16 *>(Wblk), wdim, wstr, wbox, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

// X [V][I] through the padded copy into the halo-tile kernel; Wblk = the weights blocked by 8 input channels
template <int IP, int N>
cudaError_t conv_halo_tc(const bf16 *X, int I, const bf16 *Wblk, int O, const float *b, const Lat &g, int sign,
                         int relu, const bf16 *mask, bf16 *Yb, float *Yf, int *err, bf16 *xpad, cudaStream_t s)
{
    typedef HaloLayout<N> LY;
    static std::atomic<unsigned long long> configured{ 0 };
    cudaError_t e = kernel_setup((const void *)k_conv_halo_tc<IP, N>, LY::SMEM, configured);
    if (e != cudaSuccess) return e;
    CUtensorMap tx, tw;
    e = halo_prepare(X, I, Wblk, O, N, g, 1, halo::HX, halo::HY, halo::HZ, xpad, s, &tx, &tw);
    if (e != cudaSuccess) return e;
    const int blocks = (g.L[0] / halo::TX) * (g.L[1] / halo::TY) * (g.L[2] / halo::TZ) * g.L[3];
    k_conv_halo_tc<IP, N><<<blocks, halo::THREADS, LY::SMEM, s>>>(tx, tw, O, b, g, sign, relu, mask, Yb, Yf, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// x-line convolution on the tensor cores (the default where Lx is 8, 16 or 32):
// a tile is whole periodic x lines, 128 / Lx lines of y (M = 128 rows,
// row r = x + Lx y) in each of two z planes, at one t.  The x shift of a tap is
// taken out of the A operand and applied to the accumulator: for the lines of
// one (dy, dz) a single MMA multiplies the unshifted rows by the weights of the
// three taps dx = -1, 0, +1 side by side (N = 3 x 32 columns), and the epilogue
// adds the three column blocks with their rows moved by -dx, a lane shuffle
// within each line that wraps around the period.  So every A view starts on a
// whole line (a multiple of 128 bytes), the halo has no x ghosts, and a phase
// issues 18 (dy, dz, plane) products instead of the tile kernel's 54 x-shifted
// ones; adjacent z planes share their halo views, so those 18 products are 12
// MMAs (k_conv_line_ptc below).  A phase is one 16-channel chunk and one dt
// slab as above; its halo t-plane, 4 z x (128 / Lx + 2) y lines of Lx sites,
// is one TMA box per 8-channel half from the ghost-padded copy, and its
// weights the same boxes as above.  Needs Lx in {8, 16, 32},
// Ly % (128 / Lx) == 0, Lz % 2 == 0.
// ---------------------------------------------------------------------------
namespace xline {
constexpr int TZ = 2, HZ = TZ + 2;
constexpr int RAW_MAX = HZ * 16 * (128 + 2 * 32);  // one 8-channel half of a halo t-plane, Lx = 32
constexpr int A_BYTES = 2 * RAW_MAX;
}  // namespace xline

static bool line_ok(const Lat &g)
{
    const int Lx = g.L[0];
    return (Lx == 8 || Lx == 16 || Lx == 32) && g.L[1] % (128 / Lx) == 0 && g.L[2] % xline::TZ == 0;
}

// ---------------------------------------------------------------------------
// The kernel is persistent: one CTA per SM walks the tiles b, b + gridDim.x,
// ...  Warp 8 issues the boxes of every (tile, phase) into a ring of STAGES
// buffers; warp 9 issues the MMAs into one of two accumulator sets in tensor
// memory (tile parity); warps 0-7 read the other set and run the epilogue
// (warps w and w + 4 read one TMEM lane quarter of the two planes), so a
// tile's epilogue overlaps the next tile's MMAs.  (One CTA per tile, two per
// SM, left the tensor pipe idle during each tile's epilogue: 156 against 135
// us for a 32 -> 32 layer at 32^4.)  Every wait is bounded.
// ---------------------------------------------------------------------------
namespace xlp {
constexpr int EPI_WARPS = 8;                    // two planes x four TMEM lane quarters
constexpr int THREADS = (EPI_WARPS + 2) * 32;   // + a TMA warp and an MMA warp
constexpr int EPI_STAGE = 2048;                 // per epilogue warp: 32 rows of at most 64 bytes
constexpr int SMEM_MAX = 232448;                // opt-in shared memory per block
}  // namespace xlp

// MB: mask buffers (0 = no ReLU mask)
template <int N, int MB>
struct LinePLayout {
    static constexpr bool MASKED = MB > 0;
    static constexpr int W_HALF = 27 * N * 16;
    static constexpr int W_BYTES = 2 * W_HALF;
    static constexpr int STAGE = xline::A_BYTES + W_BYTES;
    // MASKED: the output goes into a padded copy (no staging area) and MB buffers hold the ReLU
    // mask of a tile each (two planes x up to 4 channel groups x 128 sites x 16 bytes)
    static constexpr int EPI_BYTES = MASKED ? 0 : xlp::EPI_WARPS * xlp::EPI_STAGE;
    static constexpr int MASK_GROUP = 128 * 16;
    static constexpr int MASK_PLANE = 4 * MASK_GROUP;
    static constexpr int MASK_TILE = 2 * MASK_PLANE;
    static constexpr int MASK_BYTES = MB * MASK_TILE;
    static constexpr int FIXED = EPI_BYTES + MASK_BYTES + 1024;  // staging, masks, barriers and slack
    static constexpr int STAGES = (xlp::SMEM_MAX - FIXED) / STAGE < 4 ? (xlp::SMEM_MAX - FIXED) / STAGE : 4;
    static_assert(STAGES >= 2, "two buffers at least");
    static constexpr int MASK_OFF = STAGES * STAGE;
    static constexpr int EPI_OFF = MASK_OFF + MASK_BYTES;
    static constexpr int BAR_OFF = EPI_OFF + EPI_BYTES;
    // bar[0..S-1] boxes landed, bar[S..2S-1] buffer free, bar[2S..2S+1] accumulator set full,
    // bar[2S+2..2S+3] accumulator set read, bar[2S+4] drain; MASKED: bar[2S+5..2S+4+MB] mask
    // landed, bar[2S+5+MB..2S+4+2MB] mask read
    static constexpr int NBAR = 2 * STAGES + 5 + 2 * MB;
    static constexpr int SMEM = BAR_OFF + NBAR * 8 + 16;
    static constexpr int NM = 3 * N;
    static constexpr int PS = NM;                   // TMEM columns between the two planes (adjacent)
    static constexpr int ACC_COLS = 2 * PS;         // one tile's accumulators
    static constexpr int TMEM_COLS = 2 * ACC_COLS <= 256 ? 256 : 512;  // two tiles in flight
};

// (mask buffers of the masked variant: two where a tile has only three phases (IP = 16), so the
// TMA warp can run a tile ahead; one elsewhere, which leaves room for four stages)
template <int IP, bool MASKED>
constexpr int line_mask_bufs()
{
    return MASKED ? (IP <= 16 ? 2 : 1) : 0;
}

template <int IP, int N, bool MASKED>
__global__ void __launch_bounds__(xlp::THREADS, 1) k_conv_line_ptc(const __grid_constant__ CUtensorMap tx,
                                                                   const __grid_constant__ CUtensorMap tw, int O,
                                                                   const float *__restrict__ bias, Lat g, int sign,
                                                                   int relu, const bf16 *__restrict__ mask,
                                                                   bf16 *__restrict__ Yb, float *__restrict__ Yf,
                                                                   bf16 *__restrict__ Yp, int ygx,
                                                                   int *__restrict__ err, int x0)
{
    using namespace gf::tc;
    using namespace xline;
    constexpr int MB = line_mask_bufs<IP, MASKED>();
    constexpr int MBD = MB > 0 ? MB : 1;  // (divisor in code that runs only when MASKED)
    typedef LinePLayout<N, MB> LY;
    constexpr int S = LY::STAGES;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + LY::BAR_OFF);
    uint64_t *full = bar, *empty = bar + S, *acc_full = bar + 2 * S, *acc_empty = bar + 2 * S + 2;
    uint64_t *drain = bar + 2 * S + 4, *mask_full = bar + 2 * S + 5, *mask_empty = bar + 2 * S + 5 + MB;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + LY::BAR_OFF + LY::NBAR * 8);
    int *consumed_sh = reinterpret_cast<int *>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr uint32_t idesc1 = instr_desc(kM, LY::NM);      // one plane: taps dx = -1, 0, +1
    constexpr uint32_t idesc2 = instr_desc(kM, 2 * LY::NM);  // both planes from one halo view
    constexpr int NPHASE = (IP / 16) * 3;  // (16-channel chunk, dt slab)

    const int Lx = g.L[0], TYL = 128 / Lx, HY = TYL + 2;
    const uint32_t line = (uint32_t)Lx * 16;
    const uint32_t raw = (uint32_t)(HZ * HY) * line;
    const int nby = g.L[1] / TYL, nbz = g.L[2] / TZ;
    const int ntiles = nby * nbz * g.L[3];
    const int nt = (int)blockIdx.x < ntiles ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    auto tile_of = [&](int k, int &y0, int &z0, int &t0) {
        int b = (int)blockIdx.x + k * (int)gridDim.x;
        y0 = (b % nby) * TYL;
        b /= nby;
        z0 = (b % nbz) * TZ;
        t0 = b / nbz;
    };

    if (tid == 0) {
        for (int k = 0; k < LY::NBAR; ++k)
            mbar_init(&bar[k], (k == 2 * S + 2 || k == 2 * S + 3 || k >= 2 * S + 5 + MB) ? xlp::EPI_WARPS : 1);
        *consumed_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(LY::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    bool fail = false;
    int issued = 0, masks_issued = 0;
    if (warp == xlp::EPI_WARPS) {
        if (lane == 0) {
            // the boxes of (tile k, phase ph) into buffer q % S, q = k NPHASE + ph: the halo t-plane of
            // the slab (dt = sign (slab - 1)) in padded coordinates, one box per 8-channel half, then
            // the slab's weights
            for (int q = 0; q < nt * NPHASE; ++q) {
                const int slot = q % S;
                if (q >= S && !mbar_wait(&empty[slot], (uint32_t)((q / S - 1) & 1))) {
                    fail = true;
                    break;
                }
                const int k = q / NPHASE, ph = q - k * NPHASE;
                int y0, z0, t0;
                tile_of(k, y0, z0, t0);
                if (MASKED && ph == NPHASE - 1) {
                    // the tile's mask: in the padded copy without x ghosts, one channel group of a plane's
                    // 128 sites is one contiguous run of 2 KB; the O / 8 groups of both planes go into
                    // mask buffer k % MB once the epilogue has read tile k - MB's (issued with the tile's
                    // last boxes: that epilogue has begun before the tile's first MMAs)
                    const int mb = k % MBD;
                    if (k >= MB && !mbar_wait(&mask_empty[mb], (uint32_t)((k / MBD - 1) & 1))) {
                        fail = true;
                        break;
                    }
                    const int MG = O / 8;
                    const long Py = g.L[1] + 2, Pz = g.L[2] + 2, Pt = g.L[3] + 2;
                    mbar_expect_tx(&mask_full[mb], (uint32_t)(TZ * MG * LY::MASK_GROUP));
                    for (int zz = 0; zz < TZ; ++zz)
                        for (int c = 0; c < MG; ++c) {
                            const long run = ((((long)c * Pt + t0 + 1) * Pz + z0 + zz + 1) * Py + y0 + 1) * Lx;
                            bulk_load(smem + LY::MASK_OFF + mb * LY::MASK_TILE + zz * LY::MASK_PLANE +
                                          c * LY::MASK_GROUP,
                                      mask + 8 * run, LY::MASK_GROUP, &mask_full[mb]);
                        }
                    masks_issued = k + 1;
                }
                const int ch0 = 16 * (ph / 3), slab = ph % 3;
                const int ht = sign > 0 ? slab : 2 - slab;
                mbar_expect_tx(&full[slot], 2 * raw + (uint32_t)LY::W_BYTES);
                uint8_t *A = smem + slot * LY::STAGE;
#pragma unroll
                for (int kc = 0; kc < 2; ++kc)
                    tma_load_4d(A + kc * raw, &tx, x0, y0, z0, (ch0 / 8 + kc) * (g.L[3] + 2) + t0 + ht, &full[slot]);
                uint8_t *B = A + A_BYTES;
#pragma unroll
                for (int kc = 0; kc < 2; ++kc)
                    tma_load_3d(B + kc * LY::W_HALF, &tw, 0, 27 * slab, ch0 / 8 + kc, &full[slot]);
                issued = q + 1;
            }
        }
    } else if (warp == xlp::EPI_WARPS + 1) {
        if (lane == 0) {
            int consumed = 0;
            for (int k = 0; k < nt && !fail; ++k) {
                const int buf = k & 1;
                // the epilogue has read this accumulator set (tile k - 2)
                if (k >= 2 && !mbar_wait(&acc_empty[buf], (uint32_t)((k / 2 - 1) & 1))) {
                    fail = true;
                    break;
                }
                fence_after_sync();
                for (int ph = 0; ph < NPHASE; ++ph) {
                    const int q = k * NPHASE + ph, slot = q % S;
                    if (!mbar_wait(&full[slot], (uint32_t)((q / S) & 1))) {
                        fail = true;
                        break;
                    }
                    consumed = q + 1;
                    fence_after_sync();
                    // the descriptors of this buffer once; each MMA adds its view's offset to the start
                    // address field (16-byte units; shared memory stays below 256 KiB, so no carry)
                    const uint32_t A = smem_u32(smem + slot * LY::STAGE);
                    const uint64_t a0 = smem_desc(A, raw, 128), b0 = smem_desc(A + A_BYTES, LY::W_HALF, 128);
                    const uint32_t d0 = tmem + (uint32_t)(buf * LY::ACC_COLS);
                    // Halo z plane zp (0..3) of the view serves plane zz = 0 with one dz tap and plane 1
                    // with the next: the weight rows of one jy are ordered by z block Zb (slab_row), and
                    // plane 0 at zp takes block 2 - zp, plane 1 block 3 - zp.  So zp = 1, 2 are one MMA
                    // each with N = 2 NM (both planes, adjacent in TMEM), zp = 0 and 3 one plane each.
#pragma unroll
                    for (int jy = 0; jy < 3; ++jy) {
                        const int dy = sign * (jy - 1);
                        const uint64_t av = a0 + (uint64_t)((dy + 1) * Lx);    // view of halo plane 0
                        const uint64_t bj = b0 + (uint64_t)(9 * jy * N);       // rows of this jy, block 0
                        const uint64_t zpl = (uint64_t)(HY * Lx);              // one halo z plane further
                        const uint32_t first = (ph | jy) != 0;
                        mma_bf16(d0, av, bj + (uint64_t)(6 * N), idesc1, first);                  // zp 0: plane 0
                        mma_bf16(d0 + (uint32_t)LY::PS, av + 3 * zpl, bj, idesc1, first);       // zp 3: plane 1
                        mma_bf16(d0, av + zpl, bj + (uint64_t)(3 * N), idesc2, 1u);              // zp 1: both
                        mma_bf16(d0, av + 2 * zpl, bj, idesc2, 1u);                             // zp 2: both
                    }
                    mma_commit(&empty[slot]);
                }
                if (!fail) mma_commit(&acc_full[buf]);
            }
            *consumed_sh = consumed;
            mma_commit(drain);
            if (!mbar_wait(drain, 0)) fail = true;
        }
    } else {
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 of plane w / 4; row = x + Lx y, a warp holds
        // 32 / Lx whole lines; the column block of input x contributes to output x - dx: tap jx has
        // dx = sign (jx - 1), so output x takes block 1 - sign from x - 1 and block 1 + sign from x + 1
        const int zz = warp >> 2, qd = warp & 3, row = qd * 32 + lane;
        const int x = row & (Lx - 1), seg = lane & ~(Lx - 1);
        const int from_left = seg | ((x + Lx - 1) & (Lx - 1)), from_right = seg | ((x + 1) & (Lx - 1));
        // (MASKED writes a padded copy and has no staging area)
        uint4 *stage = MASKED ? nullptr : reinterpret_cast<uint4 *>(smem + LY::EPI_OFF + warp * xlp::EPI_STAGE);
        for (int k = 0; k < nt; ++k) {
            const int buf = k & 1;
            int y0, z0, t0;
            tile_of(k, y0, z0, t0);
            const long first = (long)Lx * (y0 + (long)g.L[1] * ((z0 + zz) + (long)g.L[2] * t0)) + qd * 32;
            bool landed = mbar_wait_idle(&acc_full[buf], (uint32_t)((k / 2) & 1));
            const int mb = k % MBD;
            if (MASKED) landed = landed && mbar_wait_idle(&mask_full[mb], (uint32_t)((k / MBD) & 1));
            if (!__all_sync(0xffffffffu, landed)) {  // one decision per warp, the warp converged
                fail = true;
                break;
            }
            fence_after_sync();
            const uint32_t taddr =
                tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(buf * LY::ACC_COLS + zz * LY::PS);
            float acc[N], v[N];
            tmem_load_cols<N>(taddr + (uint32_t)N, acc);
            tmem_load_cols<N>(taddr + (uint32_t)((1 - sign) * N), v);
#pragma unroll
            for (int o = 0; o < N; ++o) acc[o] += __shfl_sync(0xffffffffu, v[o], from_left);
            tmem_load_cols<N>(taddr + (uint32_t)((1 + sign) * N), v);
#pragma unroll
            for (int o = 0; o < N; ++o) acc[o] += __shfl_sync(0xffffffffu, v[o], from_right);
            // the accumulator set is free for tile k + 2 once every lane of the warp has read it
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
            if (MASKED || Yp) {
                // bias, ReLU and the mask (MASKED: this row's channel groups as the TMA warp copied them),
                // then the row straight into the padded copy Yp
#pragma unroll
                for (int o = 0; o < N; ++o) {
                    const float v = acc[o] + (bias && o < O ? bias[o] : 0.0f);
                    acc[o] = relu && !(v > 0.0f) ? 0.0f : v;
                }
                if (MASKED) {
                    const uint8_t *mrow = smem + LY::MASK_OFF + mb * LY::MASK_TILE + zz * LY::MASK_PLANE + row * 16;
#pragma unroll
                    for (int c = 0; c < N / 8; ++c)
                        if (c < O / 8) {
                            const uint4 u = *reinterpret_cast<const uint4 *>(mrow + c * LY::MASK_GROUP);
                            const uint32_t w[4] = { u.x, u.y, u.z, u.w };
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const uint16_t h = (uint16_t)(w[j / 2] >> (16 * (j % 2)));
                                if (!(__bfloat162float(__ushort_as_bfloat16(h)) > 0.0f)) acc[8 * c + j] = 0.0f;
                            }
                        }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&mask_empty[mb]);
                }
                store_padded_row<N>(acc, O, Yp, ygx, g, x, y0 + row / Lx, z0 + zz, t0);
            } else {
                epilogue_rows<N>(acc, O, bias, relu, nullptr, Yb, Yf, stage, lane, [&](int r) { return first + r; });
            }
        }
    }
    fail = __syncthreads_or(fail);
    if (fail) {
        if (tid == 0) atomicExch(err, GF_ETIMEOUT);
        // boxes issued but not consumed land before the buffers go away (bounded)
        if (warp == xlp::EPI_WARPS && lane == 0) {
            for (int q = *consumed_sh; q < issued; ++q) mbar_wait(&full[q % S], (uint32_t)((q / S) & 1));
            // the last mask copy into each buffer (an earlier one was read before the next was issued)
            for (int b = 0; b < MB; ++b) {
                const int uses = (masks_issued - b + MB - 1) / MBD;  // tiles k < masks_issued with k % MB == b
                if (uses > 0) mbar_wait(&mask_full[b], (uint32_t)((uses - 1) & 1));
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(LY::TMEM_COLS)
                     : "memory");
    }
}

// X [V][I] through the padded copy into the persistent x-line kernel (gx: x ghosts in the copy;
// padded: xpad already holds it); Wblk = the weights blocked by 8 input channels
template <int IP, int N, bool MASKED>
cudaError_t conv_line_ptc_launch(const bf16 *X, int I, const bf16 *Wblk, int O, const float *b, const Lat &g,
                                 int sign, int relu, const bf16 *mask, bf16 *Yb, float *Yf, bf16 *Yp, int ygx,
                                 int *err, bf16 *xpad, cudaStream_t s, int gx, bool padded)
{
    typedef LinePLayout<N, line_mask_bufs<IP, MASKED>()> LY;
    static std::atomic<unsigned long long> configured{ 0 };
    int nsm = 0;
    cudaError_t e = kernel_setup((const void *)k_conv_line_ptc<IP, N, MASKED>, LY::SMEM, configured, &nsm);
    if (e != cudaSuccess) return e;
    // the epilogue stages 32 rows of at most 64 bytes per warp; one output; the mask is read from a
    // padded copy, so it goes with a padded output
    if (O > 32 || O % 8 || (Yf && O > 16) || (Yb != nullptr) + (Yf != nullptr) + (Yp != nullptr) != 1 ||
        (MASKED && !Yp) || ygx < 0 || ygx > 1)
        return cudaErrorInvalidValue;
    const int TYL = 128 / g.L[0];
    CUtensorMap tx, tw;
    e = halo_prepare(X, I, Wblk, O, N, g, gx, g.L[0], TYL + 2, xline::HZ, xpad, s, &tx, &tw, padded);
    if (e != cudaSuccess) return e;
    const int tiles = (g.L[1] / TYL) * (g.L[2] / xline::TZ) * g.L[3];
    k_conv_line_ptc<IP, N, MASKED><<<std::min(tiles, nsm), xlp::THREADS, LY::SMEM, s>>>(
        tx, tw, O, b, g, sign, relu, mask, Yb, Yf, Yp, ygx, err, 8 * gx);
    return cudaGetLastError();
}

// (a ReLU mask, itself a padded copy without x ghosts, selects the variant that stages it with
// the boxes; Yp, ygx: the output as a padded copy with ygx x ghosts instead of rows Yb or Yf)
template <int IP, int N>
cudaError_t conv_line_ptc(const bf16 *X, int I, const bf16 *Wblk, int O, const float *b, const Lat &g, int sign,
                          int relu, const bf16 *mask, bf16 *Yb, float *Yf, bf16 *Yp, int ygx, int *err, bf16 *xpad,
                          cudaStream_t s, int gx, bool padded)
{
    if (mask)
        return conv_line_ptc_launch<IP, N, true>(X, I, Wblk, O, b, g, sign, relu, mask, Yb, Yf, Yp, ygx, err, xpad,
                                                 s, gx, padded);
    return conv_line_ptc_launch<IP, N, false>(X, I, Wblk, O, b, g, sign, relu, mask, Yb, Yf, Yp, ygx, err, xpad, s,
                                              gx, padded);
}

// ---------------------------------------------------------------------------
// weight gradient on the tensor cores:
//   dW[k][o][i] = sum_s dY[s][o] X[s + d(k)][i]
// as D[(tap, i)][o] = sum_s A[(tap, i)][s] B[o][s] with M = 128 rows (TG taps x
// IP input channels, padded), N = output channels (padded), K = sites.  A CTA
// takes one tap group and a chunk of sites, in stages of 64 sites (4 MMAs of
// K = 16); both operands are gathered transposed (site index along K) into the
// K-major core layout; the FP32 result is added to dW with atomics.
// ---------------------------------------------------------------------------
constexpr int kDwStageSites = 64;
constexpr int kDwChunk = 1024;  // sites per CTA

template <int IP, int N>
struct DwLayout {
    static constexpr int TG = gf::tc::kM / IP;  // taps per group (IP = 32 -> 4, IP = 80 or 128 -> 1)
    static constexpr int A_BYTES = gf::tc::kM * kDwStageSites * 2;
    static constexpr int B_BYTES = N * kDwStageSites * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int BAR_OFF = 2 * STAGE;
    static constexpr int SMEM = BAR_OFF + 3 * 8 + 16;
};

template <int IP, int N>
__global__ void __launch_bounds__(128) k_conv_dw_tc(const bf16 *__restrict__ dY, int O, const bf16 *__restrict__ X,
                                                    int I, Lat g, float *__restrict__ dW, int *__restrict__ err)
{
    using namespace gf::tc;
    typedef DwLayout<IP, N> LY;
    constexpr int TG = LY::TG;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + LY::BAR_OFF);  // 2 stages + final
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + LY::BAR_OFF + 3 * 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int k0 = blockIdx.y * TG;  // first tap of the group
    const int s_begin = blockIdx.x * kDwChunk;
    const int s_end = min(s_begin + kDwChunk, g.V);
    constexpr uint32_t idesc = instr_desc(kM, N);

    // operands start at zero (padding rows stay zero)
    for (int e = tid; e < 2 * LY::STAGE / 16; e += kThreads)
        reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int st = 0; st < 3; ++st) mbar_init(&bar[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    bool fail = false;
    const int nstage = (s_end - s_begin + kDwStageSites - 1) / kDwStageSites;
    for (int t = 0; t < nstage; ++t) {
        const int st = t & 1;
        if (t >= 2) {
            if (!mbar_wait(&bar[st], (uint32_t)((t / 2 - 1) & 1))) fail = true;
        }
        if (__syncthreads_or(fail)) {
            fail = true;
            break;
        }
        uint8_t *A = smem + st * LY::STAGE;
        uint8_t *B = A + LY::A_BYTES;
        const int s0 = s_begin + t * kDwStageSites;
        // A[(kl, i)][s] = X[s + d(k0 + kl)][i]: core (r/8, s/8) at ((s/8) * 16 + r/8) * 128,
        // row r%8 (16 B), element s%8 (2 B)
        for (int it = tid; it < kDwStageSites * TG; it += kThreads) {
            const int sl = it % kDwStageSites, kl = it / kDwStageSites;
            const int s = s0 + sl, k = k0 + kl;
            const bool ok = s < s_end && k < 81;
            const int nb = ok ? shift_site(g, s, k, 1) : 0;
            for (int c = 0; c < IP / 8; ++c) {
                uint4 v = make_uint4(0, 0, 0, 0);
                if (ok && 8 * c < I) v = *reinterpret_cast<const uint4 *>(X + (long)nb * I + 8 * c);
                const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int r = kl * IP + 8 * c + q;
                    *reinterpret_cast<bf16 *>(A + ((sl >> 3) * 16 + (r >> 3)) * 128 + (r & 7) * 16 + (sl & 7) * 2) = e[q];
                }
            }
        }
        // B[o][s] = dY[s][o]: core (o/8, s/8) at ((s/8) * (N/8) + o/8) * 128
        for (int it = tid; it < kDwStageSites; it += kThreads) {
            const int s = s0 + it;
            for (int c = 0; c < (O + 7) / 8; ++c) {
                uint4 v = make_uint4(0, 0, 0, 0);
                if (s < s_end) v = *reinterpret_cast<const uint4 *>(dY + (long)s * O + 8 * c);
                const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int o = 8 * c + q;
                    *reinterpret_cast<bf16 *>(B + ((it >> 3) * (N / 8) + (o >> 3)) * 128 + (o & 7) * 16 + (it & 7) * 2) = e[q];
                }
            }
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < kDwStageSites / 16; ++kk) {
                uint64_t ad = smem_desc(smem_u32(A + kk * 2 * 2048), 2048, 128);
                uint64_t bd = smem_desc(smem_u32(B + kk * 2 * (N / 8) * 128), (N / 8) * 128, 128);
                mma_bf16(tmem, ad, bd, idesc, (t | kk) != 0);
            }
            mma_commit(&bar[st]);
        }
    }
    if (tid == 0) mma_commit(&bar[2]);
    if (!mbar_wait(&bar[2], 0)) fail = true;
    fail = __syncthreads_or(fail);
    if (!fail && nstage > 0) {
        fence_after_sync();
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        if (N == 32) {
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
        } else {
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
                " [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int row = tid, kl = row / IP, i = row - kl * IP, k = k0 + kl;
        if (kl < TG && k < 81 && i < I) {
#pragma unroll
            for (int o = 0; o < N; ++o) {
                if (o >= O) break;
                atomicAdd(&dW[((long)k * O + o) * I + i], __uint_as_float(r[o]));
            }
        }
    } else if (fail && tid == 0) {
        atomicExch(err, GF_ETIMEOUT);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
    }
}

// db[o] = sum_s dY[s][o]
__global__ void k_bias_grad(const bf16 *__restrict__ dY, int O, int V, float *__restrict__ db)
{
    __shared__ float acc[32];
    if (threadIdx.x < 32) acc[threadIdx.x] = 0.0f;
    __syncthreads();
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)V * O; e += (long)gridDim.x * blockDim.x)
        atomicAdd(&acc[e % O], __bfloat162float(dY[e]));
    __syncthreads();
    if (threadIdx.x < O) atomicAdd(&db[threadIdx.x], acc[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// weight gradient on the tensor cores, x-line form (Lx in {8, 16, 32},
// Ly % (128 / Lx) == 0).  With the x part of a tap moved onto dY,
//
//   dW[k][o][i] = sum_s X[s + (0, dy, dz, dt)][i] dY[s - (dx, 0, 0, 0)][o],
//
// the GEMM D[(dz, i)][(dx, o)] = sum_s A[(dz, i)][s] B[(dx, o)][s], one per
// (dy, dt), gives the taps k = (dx+1) + 3 (dy+1) + 9 (dz+1) + 27 (dt+1).  The
// site sum is the MMA's K dimension and both operands are MN-major: in the
// ghost-padded copies, blocked by 8 channels, a run of sites along x with its
// 8 channels is already a column of 8-site x 16-byte core matrices, so TMA
// boxes land in shared memory as operands without a transpose.  A stage is
// 128 sites, 128 / Lx whole x lines at one (z, t):
// - A: one 5D box of the X copy per stage: channel groups g0 .. g0 + CH - 1,
//   z - 1 .. z + 1, the lines y0 - 1 .. y0 + 128 / Lx at t + dt.  Slot
//   3 (g - g0) + (dz + 1) of the box is one M column of 8 channels, the slots
//   at a uniform stride, and the MMA of tap row dy reads each slot from its
//   line dy + 1 on: a view that starts on a whole line.  So one box serves the
//   3 dy x 3 dz taps of 3 CH M columns (CH = 4 of 4 groups, or 5 of 10).
// - B: one box per dx, dY at x - dx from the copy with x ghosts, all output
//   groups: N = 3 O columns (padded to a multiple of 32).
// A stage issues 3 x 8 MMAs of K = 16 (dy, K step) into 3 accumulators.  Each
// CTA takes one (dt, channel chunk) and every R-th stage from its first, so the
// CTAs move through the lattice together and the planes they read stay in L2;
// it adds its accumulators into dW (FP32 atomics) at the end.  The bias
// gradient db[o] = sum_s dY[s][o] comes out of the same MMAs: the CTAs of
// dt = 0 and the first chunk hold ones in the unused M column 3 CH.  Roles: warp 4
// issues the boxes into a ring of STAGES buffers, warp 5 the MMAs, warps 0-3
// read the accumulators (warp w: TMEM lanes 32 w .. 32 w + 31).  Every wait is
// bounded.
// ---------------------------------------------------------------------------
namespace dwline {
constexpr int SLOT_MAX = 3072;            // one M column: 128 / Lx + 2 lines of Lx sites x 16 bytes (Lx = 32)
constexpr int A_BYTES = 16 * SLOT_MAX;    // 16 M columns of an MMA (only 3 CH <= 15 are loaded)
constexpr int B_BOX = 128 * 16;           // 128 sites x 8 channels
constexpr int THREADS = 192;
}  // namespace dwline

template <int NP>  // accumulator columns per tap row: 3 x output channels, padded to a multiple of 32
struct DwLineLayout {
    static_assert(NP % 32 == 0 && NP <= 128, "accumulator read in blocks of 32 columns");
    static constexpr int B_BYTES = (NP / 8) * dwline::B_BOX;
    static constexpr int STAGE = dwline::A_BYTES + B_BYTES;
    // as many stages as fit, up to four (NP = 32: 4 of 56 KB, NP = 96: 3 of 72 KB)
    static constexpr int STAGES = (xlp::SMEM_MAX - 256) / STAGE < 4 ? (xlp::SMEM_MAX - 256) / STAGE : 4;
    static_assert(STAGES >= 2, "two buffers at least");
    // bar[0..S-1] boxes landed, bar[S..2S-1] MMAs done with the buffer, bar[2S] accumulators final,
    // bar[2S+1] drain
    static constexpr int NBAR = 2 * STAGES + 2;
    static constexpr int BAR_OFF = STAGES * STAGE;
    static constexpr int SMEM = BAR_OFF + NBAR * 8 + 16;
    static constexpr int TMEM_COLS = 3 * NP <= 128 ? 128 : (3 * NP <= 256 ? 256 : 512);
};

static bool dw_line_ok(const Lat &g)
{
    const int Lx = g.L[0];
    return (Lx == 8 || Lx == 16 || Lx == 32) && g.L[1] % (128 / Lx) == 0;
}

__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(gf::tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(gf::tc::smem_u32(bar))
        : "memory");
}

// Shared-memory descriptor of an MN-major operand without swizzle: core
// matrices of 8 K-rows x 16 bytes (8 MN elements), lbo = byte offset between
// core matrices adjacent in K, sbo = between core matrices adjacent in M or N.
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t addr, uint32_t lbo_k, uint32_t sbo_mn)
{
    return gf::tc::smem_desc(addr, lbo_k, sbo_mn);
}

// grid = 3 * nchunk * R CTAs: CTA b has dt = b / (nchunk R) - 1, channel chunk (b / R) % nchunk, member b % R
template <int NP, int TD>
__global__ void __launch_bounds__(dwline::THREADS) k_conv_dw_line_tc(const __grid_constant__ CUtensorMap tx,
                                                                     const __grid_constant__ CUtensorMap ty, int I,
                                                                     int O, int CH, Lat g, float *__restrict__ dW,
                                                                     float *__restrict__ db, int *__restrict__ err)
{
    using namespace gf::tc;
    using dwline::B_BOX;
    typedef DwLineLayout<NP> LY;
    constexpr int S = LY::STAGES;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + LY::BAR_OFF);
    uint64_t *acc_done = &bar[2 * S], *drain = &bar[2 * S + 1];
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + LY::BAR_OFF + LY::NBAR * 8);
    int *consumed_sh = reinterpret_cast<int *>(smem + LY::BAR_OFF + LY::NBAR * 8 + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // kind::f16, D = F32, A = B = BF16, both operands MN-major (bits 15, 16)
    constexpr uint32_t idesc = instr_desc(kM, NP) | (1u << 15) | (1u << 16);
    const int G = I / 8, OG = O / 8, Lx = g.L[0], TYL = 128 / Lx, nby = g.L[1] / TYL;
    const uint32_t line = (uint32_t)Lx * 16, slot = (uint32_t)(TYL + 2) * line;
    // TD = 1: a CTA type per (dt, chunk); TD = 3: dt rides on dY as dx does, a type per chunk
    const int nchunk = (G + CH - 1) / CH, R = gridDim.x / ((3 / TD) * nchunk);
    const int type = blockIdx.x / R, member = blockIdx.x - type * R;
    const int dti = TD == 3 ? 1 : type / nchunk, g0 = (type - (TD == 3 ? 0 : dti) * nchunk) * CH;
    const int nch = min(CH, G - g0);
    constexpr int BIAS_BLK = TD == 3 ? 4 : 1;  // column block of dt = 0, dx = 0
    const int NS = g.V / 128;
    const int n = member < NS ? (NS - member + R - 1) / R : 0;  // stages member, member + R, ...

    // M columns beyond 3 nch and the N padding stay zero, except that the CTAs of dt = 0 (all,
    // TD = 3) and the first chunk fill M column 3 CH (never loaded) with ones in every buffer:
    // its first row of the dy = -1 accumulator is then sum_s dY[s - (dx, 0, 0, dt)][o], the
    // bias gradient in the column block of dx = dt = 0
    const bool bias = dti == 1 && g0 == 0 && 3 * CH < 16;
    const uint32_t ones_lo = bias ? (uint32_t)(3 * CH) * slot : 0u, ones_hi = bias ? ones_lo + slot : 0u;
    for (int e = tid; e < LY::BAR_OFF / 16; e += dwline::THREADS) {
        const uint32_t off = (uint32_t)(e * 16) % (uint32_t)LY::STAGE;
        const uint32_t one = 0x3F803F80u;  // two BF16 ones
        reinterpret_cast<uint4 *>(smem)[e] =
            off >= ones_lo && off < ones_hi ? make_uint4(one, one, one, one) : make_uint4(0, 0, 0, 0);
    }
    fence_proxy_async();
    if (tid == 0) {
        for (int k = 0; k < LY::NBAR; ++k) mbar_init(&bar[k], 1);
        *consumed_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(LY::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    bool fail = false;
    int issued = 0;
    if (warp == 4 && lane == 0) {
        // producer: the boxes of stage p into buffer p % S once the MMAs of stage p - S are done
        const uint32_t bytes = (uint32_t)(3 * nch) * slot + (uint32_t)(3 * TD * OG) * B_BOX;
        for (int p = 0; p < n; ++p) {
            const int b = p % S;
            if (p >= S && !mbar_wait(&bar[S + b], (uint32_t)((p / S - 1) & 1))) {
                fail = true;
                break;
            }
            const int st = member + p * R;
            const int y0 = (st % nby) * TYL, zt = st / nby, z = zt % g.L[2], t = zt / g.L[2];
            uint8_t *A = smem + b * LY::STAGE;
            uint8_t *B = A + dwline::A_BYTES;
            mbar_expect_tx(&bar[b], bytes);
            // padded coordinates: lines y0 - 1 .. (padded y0), planes z - 1 .. z + 1 (padded z), t + dt
            tma_load_5d(A, &tx, 0, y0, z, t + dti, g0, &bar[b]);
            // dY at x - dx: padded x from 1 - dx, dx = dxi - 1; TD = 3: and at t - dt, padded t
            // 2 + t - dtc, dt = dtc - 1 (the X box above is then at dt = 0), column block 3 dtc + dxi
            for (int dtc = 0; dtc < TD; ++dtc)
                for (int dxi = 0; dxi < 3; ++dxi)
                    tma_load_5d(B + (3 * dtc + dxi) * OG * B_BOX, &ty, 8 * (2 - dxi), y0 + 1, z + 1,
                                TD == 3 ? t + 2 - dtc : t + 1, 0, &bar[b]);
            issued = p + 1;
        }
    } else if (warp == 5 && lane == 0) {
        // MMA issuer: accumulator dyi = tap row dy = dyi - 1, at columns dyi NP
        int consumed = 0;
        for (int p = 0; p < n; ++p) {
            if (!mbar_wait(&bar[p % S], (uint32_t)((p / S) & 1))) {
                fail = true;
                break;
            }
            consumed = p + 1;
            fence_after_sync();
            // the descriptors of this buffer once; each MMA adds its view's offset to the start address
            // field (16-byte units; shared memory stays below 256 KiB, so no carry)
            const uint32_t A = smem_u32(smem + (p % S) * LY::STAGE);
            const uint64_t a0 = smem_desc_mn(A, 128, slot), b0 = smem_desc_mn(A + dwline::A_BYTES, 128, B_BOX);
#pragma unroll
            for (int dyi = 0; dyi < 3; ++dyi)
#pragma unroll
                for (int kk = 0; kk < 8; ++kk)
                    mma_bf16(tmem + (uint32_t)(dyi * NP), a0 + (uint64_t)(dyi * Lx + kk * 16), b0 + (uint64_t)(kk * 16),
                             idesc, (p | kk) != 0);
            mma_commit(&bar[S + p % S]);
        }
        *consumed_sh = consumed;
        if (!fail && n > 0) mma_commit(acc_done);
        mma_commit(drain);
        if (!mbar_wait(drain, 0)) fail = true;
    } else if (warp < 4 && n > 0) {
        // row 32 w + lane = M column m = 3 (g - g0) + (dz + 1), channel i = 8 g + (row % 8);
        // row 8 (3 CH) of the dy = -1 accumulator is the bias gradient where ones fill column 3 CH
        const int row = 32 * warp + lane, m = row >> 3, gl = m / 3, dzi = m - 3 * gl;
        const int i = 8 * (g0 + gl) + (row & 7);
        const bool bias_row = bias && row == 8 * 3 * CH;
        // one decision per warp (and the warp converged) before the warp-wide accumulator loads
        const bool landed = mbar_wait_idle(acc_done, 0);
        if (!__all_sync(0xffffffffu, landed)) {
            fail = true;
        } else {
            fence_after_sync();
#pragma unroll 1
            for (int dyi = 0; dyi < 3; ++dyi) {
                const int k0 = 3 * dyi + 9 * dzi;  // tap of dx = -1, dt = -1
#pragma unroll 1
                for (int c0 = 0; c0 < NP; c0 += 32) {
                    float v[32];
                    tmem_load_cols<32>(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(dyi * NP + c0), v);
                    if (bias_row && dyi == 0) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const int col = c0 + c;
                            if (col >= BIAS_BLK * O && col < (BIAS_BLK + 1) * O) atomicAdd(&db[col - BIAS_BLK * O], v[c]);
                        }
                    }
                    if (gl < nch) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const int col = c0 + c;  // (3 dtc + dx + 1) O + o (TD = 1: dtc = 0, dt from the type)
                            if (col < 3 * TD * O) {
                                const int blk = col / O, o = col - blk * O;
                                const int dtk = TD == 3 ? blk / 3 : dti, dxi = blk % 3;
                                atomicAdd(&dW[((long)(k0 + 27 * dtk + dxi) * O + o) * I + i], v[c]);
                            }
                        }
                    }
                }
            }
        }
    }
    fail = __syncthreads_or(fail);
    if (fail) {
        if (tid == 0) atomicExch(err, GF_ETIMEOUT);
        // boxes issued but not consumed land before the buffers go away (bounded)
        if (warp == 4 && lane == 0)
            for (int p = *consumed_sh; p < issued; ++p) mbar_wait(&bar[p % S], (uint32_t)((p / S) & 1));
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(LY::TMEM_COLS)
                     : "memory");
    }
}

// dW and db of one layer through the x-line weight-gradient kernel: X [V][I] is
// padded without x ghosts into xpad (unless x_padded: xpad holds it already),
// dY [V][O] with them into ypad (unless y_padded)
// (TD = 3: the three dt columns of each tap ride on dY in N as the dx ones do, for
// 3 TD O <= NP; one CTA type per channel chunk instead of three)
template <int NP, int TD>
cudaError_t conv_dw_line_tc(const bf16 *dY, int O, const bf16 *X, int I, const Lat &g, float *dW, float *db,
                            int *err, bf16 *xpad, bf16 *ypad, cudaStream_t s, bool x_padded = false,
                            bool y_padded = false)
{
    static_assert(TD == 1 || TD == 3, "dt per CTA type or all three in N");
    typedef DwLineLayout<NP> LY;
    static std::atomic<unsigned long long> configured{ 0 };
    int nsm = 0;
    cudaError_t e = kernel_setup((const void *)k_conv_dw_line_tc<NP, TD>, LY::SMEM, configured, &nsm);
    if (e != cudaSuccess) return e;
    const EncodeTiledFn enc = encode_tiled();
    const int G = I / 8, OG = O / 8;
    if (!enc || !xpad || !ypad || I % 8 || O % 8 || 3 * TD * O > NP) return cudaErrorNotSupported;
    // channel groups per chunk: the largest divisor of G with 3 CH <= 15 M columns
    int CH = 1;
    for (int d = 1; d <= 5; ++d)
        if (G % d == 0) CH = d;
    const int Lx = g.L[0], TYL = 128 / Lx;
    const long px = padded_sites(g, 0), py = padded_sites(g, 1);
    if (!x_padded) {
        k_pad_periodic<<<(int)std::min<long>((px + 255) / 256, 152L * 32), 256, 0, s>>>(X, I, g, 0, xpad);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (!y_padded) {
        k_pad_periodic<<<(int)std::min<long>((py + 255) / 256, 152L * 32), 256, 0, s>>>(dY, O, g, 1, ypad);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const cuuint64_t es = sizeof(bf16);
    const cuuint64_t Py = g.L[1] + 2, Pz = g.L[2] + 2, Pt = g.L[3] + 2;
    const cuuint32_t ones[5] = { 1, 1, 1, 1, 1 };
    CUtensorMap tmap[2];
    for (int which = 0; which < 2; ++which) {  // 0: X (no x ghosts), 1: dY (x ghosts)
        const cuuint64_t Px = Lx + 2 * which, groups = (cuuint64_t)(which ? OG : G);
        const cuuint64_t dim[5] = { 8 * Px, Py, Pz, Pt, groups };
        const cuuint64_t str[4] = { 8 * es * Px, 8 * es * Px * Py, 8 * es * Px * Py * Pz,
                                    8 * es * Px * Py * Pz * Pt };
        const cuuint32_t box[5] = { (cuuint32_t)(8 * Lx), (cuuint32_t)(which ? TYL : TYL + 2), which ? 1u : 3u, 1,
                                    (cuuint32_t)(which ? OG : CH) };
        if (enc(&tmap[which], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, which ? ypad : xpad, dim, str, box, ones,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const int NT = (3 / TD) * ((G + CH - 1) / CH);
    const int NS = g.V / 128;
    const int R = std::max(1, std::min(nsm / NT, NS));
    k_conv_dw_line_tc<NP, TD><<<NT * R, dwline::THREADS, LY::SMEM, s>>>(tmap[0], tmap[1], I, O, CH, g, dW, db, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (3 * CH >= 16) {  // no free M column for the ones: the bias gradient on its own
        if (!dY) return cudaErrorInvalidValue;
        k_bias_grad<<<256, 256, 0, s>>>(dY, O, g.V, db);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

template <int IP, int N>
cudaError_t conv_dw_tc(const bf16 *dY, int O, const bf16 *X, int I, const Lat &g, float *dW, float *db, int *err,
                       cudaStream_t s)
{
    typedef DwLayout<IP, N> LY;
    static std::atomic<unsigned long long> configured{ 0 };
    cudaError_t e = kernel_setup((const void *)k_conv_dw_tc<IP, N>, LY::SMEM, configured);
    if (e != cudaSuccess) return e;
    dim3 grid((g.V + kDwChunk - 1) / kDwChunk, (81 + LY::TG - 1) / LY::TG);
    k_conv_dw_tc<IP, N><<<grid, gf::tc::kThreads, LY::SMEM, s>>>(dY, O, X, I, g, dW, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_bias_grad<<<256, 256, 0, s>>>(dY, O, g.V, db);
    return cudaGetLastError();
}

template <int I, int O>
cudaError_t conv_cc(const bf16 *X, const bf16 *W, const float *b, const Lat &g, int sign, int relu, const bf16 *mask,
                    bf16 *Yb, float *Yf, cudaStream_t s)
{
    constexpr int SITES = 256 / (O / 8);
    k_conv_cc<I, O><<<(g.V + SITES - 1) / SITES, 256, 0, s>>>(X, W, b, g, sign, relu, mask, Yb, Yf);
    return cudaGetLastError();
}

template <int I, int O>
cudaError_t conv_dw(const bf16 *dY, const bf16 *X, const Lat &g, float *dW, float *db, cudaStream_t s)
{
    dim3 grid((g.V + 63) / 64, 81);
    k_conv_dw<I, O><<<grid, 256, 0, s>>>(dY, X, g, dW, db);
    return cudaGetLastError();
}

}  // namespace

struct gf_net {
    Lat g;
    cudaStream_t stream = nullptr;
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    long np = 0;
    long woff[4], boff[4];
    bf16 *Wb[4] = { nullptr }, *Wt[4] = { nullptr };
    bf16 *Wh[4] = { nullptr }, *Wth[4] = { nullptr };  // the same, blocked by 8 input channels
    bf16 *act[4] = { nullptr };  // act[1..3] owned; act[0] = caller's features
    float *out = nullptr;
    bf16 *dA = nullptr, *dB = nullptr;  // [V][32] gradient scratch (ping-pong)
    bf16 *xpad = nullptr;  // halo-tile convolutions: the input with periodic ghost sites, up to 80 channels
    // x-line weight gradients: dY with periodic ghost sites (x included), up to 32 channels; on the
    // x-line path the data gradients write their output into the other one of the two
    bf16 *ypad = nullptr, *ypad2 = nullptr;
    // x-line path: each layer's input as a padded copy without x ghosts; layer 1's is padded from
    // the features, the others are written by the previous layer's epilogue (act[] is unused there)
    bf16 *xin[4] = { nullptr };
    double *partial = nullptr, *dloss = nullptr;
    int *derr = nullptr;  // tensor-core kernels: bounded-wait expiry
    int use_tc = 1;       // forward and backward-data on tcgen05 (else CUDA cores)
    int use_halo = 1;     // ... staged by halo: 1 x-line kernel first, 2 halo-tile kernel only, 0 neither
    int step = 0;
    std::string err;
};

static int nfail(gf_net *n, int code, const std::string &m)
{
    if (code == GF_ECUDA || code == GF_ENOMEM) cudaGetLastError();
    n->err = m;
    return code;
}

#define NCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return nfail(n, e_ == cudaErrorMemoryAllocation ? GF_ENOMEM : GF_ECUDA,        \
                         std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

static long param_count()
{
    long n = 0;
    for (int l = 0; l < 4; ++l) n += 81L * kC[l + 1] * kC[l] + kC[l + 1];
    return n;
}

static int refresh_weights(gf_net *n)
{
    for (int l = 0; l < 4; ++l) {
        long cnt = 81L * kC[l + 1] * kC[l];
        k_cast_weights<<<(int)((cnt + 255) / 256), 256, 0, n->stream>>>(n->params + n->woff[l], kC[l], kC[l + 1],
                                                                          n->Wb[l], n->Wt[l], n->Wh[l],
                                                                          n->Wth[l]);
        NCK(cudaGetLastError());
    }
    return GF_OK;
}

// the x-line path (forward_line, backward_line): conv_halo 1 on a lattice the x-line kernels take
static bool line_path(const gf_net *n) { return n->use_tc && n->use_halo == 1 && line_ok(n->g) && n->ypad2; }

// forward / backward-data convolution on the tensor cores off the x-line path: the
// halo-tile kernel where the extents allow it and conv_halo is not 0, otherwise
// the per-tap gather kernel (W = weights [81][O][I], Wblk = the same blocked by 8
// input channels)
template <int IP, int N>
static cudaError_t conv_tensor(const gf_net *n, const bf16 *X, int I, const bf16 *W, const bf16 *Wblk, int O,
                               const float *b, int sign, int relu, const bf16 *mask, bf16 *Yb, float *Yf)
{
    if (n->use_halo != 0 && halo_ok(n->g))
        return conv_halo_tc<IP, N>(X, I, Wblk, O, b, n->g, sign, relu, mask, Yb, Yf, n->derr, n->xpad, n->stream);
    return conv_tc<IP, N>(X, I, W, O, b, n->g, sign, relu, mask, Yb, Yf, n->derr, n->stream);
}

// weight and bias gradients of one layer on the tensor cores off the x-line path:
// with conv_halo 1 the x-line weight-gradient kernel where the extents allow it
// (Lz odd, say), otherwise the gather kernel
template <int IP, int N>
static cudaError_t dw_tensor(const gf_net *n, const bf16 *dY, int O, const bf16 *X, int I, float *dW, float *db)
{
    if (n->use_halo == 1 && n->ypad && dw_line_ok(n->g)) {
        if (O <= 8) return conv_dw_line_tc<96, 3>(dY, O, X, I, n->g, dW, db, n->derr, n->xpad, n->ypad, n->stream);
        return conv_dw_line_tc<96, 1>(dY, O, X, I, n->g, dW, db, n->derr, n->xpad, n->ypad, n->stream);
    }
    return conv_dw_tc<IP, N>(dY, O, X, I, n->g, dW, db, n->derr, n->stream);
}

// the padded layer inputs of the x-line path
static int ensure_line_buffers(gf_net *n)
{
    if (n->xin[0]) return GF_OK;
    const long P = padded_sites(n->g, 0);
    for (int l = 0; l < 4; ++l) {
        const cudaError_t e = cudaMalloc(&n->xin[l], sizeof(bf16) * P * kC[l]);
        if (e != cudaSuccess) {
            for (int k = 0; k < 4; ++k) {
                cudaFree(n->xin[k]);
                n->xin[k] = nullptr;
            }
            return nfail(n, e == cudaErrorMemoryAllocation ? GF_ENOMEM : GF_ECUDA,
                         std::string("padded layer inputs: ") + cudaGetErrorString(e));
        }
    }
    return GF_OK;
}

// forward pass on the x-line path: the features are padded into xin[0]; each
// layer's epilogue writes the next layer's padded input xin[l + 1] itself
static int forward_line(gf_net *n, const bf16 *f)
{
    const int r = ensure_line_buffers(n);
    if (r != GF_OK) return r;
    const Lat &g = n->g;
    cudaStream_t s = n->stream;
    bf16 *const *xi = n->xin;
    NCK((conv_line_ptc<80, 32>(f, 80, n->Wh[0], 32, n->params + n->boff[0], g, 1, 1, nullptr, nullptr, nullptr,
                               xi[1], 0, n->derr, xi[0], s, 0, false)));
    NCK((conv_line_ptc<32, 32>(nullptr, 32, n->Wh[1], 32, n->params + n->boff[1], g, 1, 1, nullptr, nullptr,
                               nullptr, xi[2], 0, n->derr, xi[1], s, 0, true)));
    NCK((conv_line_ptc<32, 32>(nullptr, 32, n->Wh[2], 32, n->params + n->boff[2], g, 1, 1, nullptr, nullptr,
                               nullptr, xi[3], 0, n->derr, xi[2], s, 0, true)));
    NCK((conv_line_ptc<32, 16>(nullptr, 32, n->Wh[3], 8, n->params + n->boff[3], g, 1, 0, nullptr, nullptr, n->out,
                               nullptr, 0, n->derr, xi[3], s, 0, true)));
    return GF_OK;
}

// backward pass on the x-line path after forward_line, from dY of layer 4 as the
// loss kernel wrote it into ypad (ghost-padded, x ghosts included): each data
// gradient reads dY from one padded copy, masks by the layer's padded input and
// writes its output into the other copy, which the weight gradient of the layer
// below and the next data gradient read as they are
static int backward_line(gf_net *n, const bf16 *f)
{
    const Lat &g = n->g;
    cudaStream_t s = n->stream;
    bf16 *const *xi = n->xin;
    bf16 *yp[2] = { n->ypad, n->ypad2 };
    NCK((conv_dw_line_tc<96, 3>(nullptr, 8, nullptr, 32, g, n->grad + n->woff[3], n->grad + n->boff[3], n->derr,
                             xi[3], yp[0], s, true, true)));
    NCK((conv_line_ptc<16, 32>(nullptr, 8, n->Wth[3], 32, nullptr, g, -1, 0, xi[3], nullptr, nullptr, yp[1], 1,
                               n->derr, yp[0], s, 1, true)));
    int cur = 1;  // yp[cur] holds dY of layer l
    for (int l = 2; l >= 1; --l) {
        NCK((conv_dw_line_tc<96, 1>(nullptr, 32, nullptr, 32, g, n->grad + n->woff[l], n->grad + n->boff[l], n->derr,
                                 xi[l], yp[cur], s, true, true)));
        NCK((conv_line_ptc<32, 32>(nullptr, 32, n->Wth[l], 32, nullptr, g, -1, 0, xi[l], nullptr, nullptr,
                                   yp[1 - cur], 1, n->derr, yp[cur], s, 1, true)));
        cur = 1 - cur;
    }
    NCK((conv_dw_line_tc<96, 1>(nullptr, 32, f, 80, g, n->grad + n->woff[0], n->grad + n->boff[0], n->derr, xi[0],
                             yp[cur], s, true, true)));
    return GF_OK;
}

static int forward(gf_net *n, const bf16 *f)
{
    const Lat &g = n->g;
    cudaStream_t s = n->stream;
    n->act[0] = const_cast<bf16 *>(f);
    if (line_path(n)) return forward_line(n, f);
    if (n->use_tc) {
        NCK((conv_tensor<80, 32>(n, f, 80, n->Wb[0], n->Wh[0], 32, n->params + n->boff[0], 1, 1, nullptr, n->act[1],
                                 nullptr)));
        NCK((conv_tensor<32, 32>(n, n->act[1], 32, n->Wb[1], n->Wh[1], 32, n->params + n->boff[1], 1, 1, nullptr,
                                 n->act[2], nullptr)));
        NCK((conv_tensor<32, 32>(n, n->act[2], 32, n->Wb[2], n->Wh[2], 32, n->params + n->boff[2], 1, 1, nullptr,
                                 n->act[3], nullptr)));
        NCK((conv_tensor<32, 16>(n, n->act[3], 32, n->Wb[3], n->Wh[3], 8, n->params + n->boff[3], 1, 0, nullptr,
                                 nullptr, n->out)));
        return GF_OK;
    }
    NCK((conv_cc<80, 32>(f, n->Wb[0], n->params + n->boff[0], g, 1, 1, nullptr, n->act[1], nullptr, s)));
    NCK((conv_cc<32, 32>(n->act[1], n->Wb[1], n->params + n->boff[1], g, 1, 1, nullptr, n->act[2], nullptr, s)));
    NCK((conv_cc<32, 32>(n->act[2], n->Wb[2], n->params + n->boff[2], g, 1, 1, nullptr, n->act[3], nullptr, s)));
    NCK((conv_cc<32, 8>(n->act[3], n->Wb[3], n->params + n->boff[3], g, 1, 0, nullptr, nullptr, n->out, s)));
    return GF_OK;
}

// backward data of layer l (l = 3, 2, 1) off the x-line path: dX = conv^T(dY) masked by act[l] > 0
static int backward_data(gf_net *n, int l, const bf16 *dY, bf16 *dX)
{
    const Lat &g = n->g;
    cudaStream_t s = n->stream;
    if (l == 3) {
        if (n->use_tc) NCK((conv_tensor<16, 32>(n, dY, 8, n->Wt[3], n->Wth[3], 32, nullptr, -1, 0, n->act[3], dX, nullptr)));
        else NCK((conv_cc<8, 32>(dY, n->Wt[3], nullptr, g, -1, 0, n->act[3], dX, nullptr, s)));
    } else {
        if (n->use_tc) NCK((conv_tensor<32, 32>(n, dY, 32, n->Wt[l], n->Wth[l], 32, nullptr, -1, 0, n->act[l], dX, nullptr)));
        else NCK((conv_cc<32, 32>(dY, n->Wt[l], nullptr, g, -1, 0, n->act[l], dX, nullptr, s)));
    }
    return GF_OK;
}

static int check_status(gf_net *n)
{
    int e = 0;
    NCK(cudaMemcpyAsync(&e, n->derr, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    NCK(cudaStreamSynchronize(n->stream));
    if (e) {
        cudaMemsetAsync(n->derr, 0, sizeof(int), n->stream);
        return nfail(n, e, "a bounded wait expired in a tensor-core convolution");
    }
    return GF_OK;
}

// forward + loss + backward into n->grad; loss left in n->dloss (device)
static int backward(gf_net *n, const bf16 *f, const float *target)
{
    const Lat &g = n->g;
    cudaStream_t s = n->stream;
    int r = forward(n, f);
    if (r != GF_OK) return r;
    long nout = (long)g.V * 8;
    int nblk = 1024;  // (n->partial holds 1024 block sums)
    // x-line path: dY of layer 4 straight into the padded copy its weight gradient reads
    if (line_path(n)) k_mse<true><<<nblk, 256, 0, s>>>(n->out, target, g, 1.0f / (float)nout, n->ypad, n->partial);
    else k_mse<false><<<nblk, 256, 0, s>>>(n->out, target, g, 1.0f / (float)nout, n->dA, n->partial);
    NCK(cudaGetLastError());
    k_sum_partials<<<1, 32, 0, s>>>(n->partial, nblk, 1.0 / (double)nout, n->dloss);
    NCK(cudaGetLastError());
    NCK(cudaMemsetAsync(n->grad, 0, sizeof(float) * n->np, s));
    if (line_path(n)) return backward_line(n, f);
    // layer 4: dY = dA [V][8]
    if (n->use_tc)
        NCK((dw_tensor<32, 16>(n, n->dA, 8, n->act[3], 32, n->grad + n->woff[3], n->grad + n->boff[3])));
    else NCK((conv_dw<32, 8>(n->dA, n->act[3], g, n->grad + n->woff[3], n->grad + n->boff[3], s)));
    r = backward_data(n, 3, n->dA, n->dB);
    if (r != GF_OK) return r;
    // layer 3
    if (n->use_tc)
        NCK((dw_tensor<32, 32>(n, n->dB, 32, n->act[2], 32, n->grad + n->woff[2], n->grad + n->boff[2])));
    else NCK((conv_dw<32, 32>(n->dB, n->act[2], g, n->grad + n->woff[2], n->grad + n->boff[2], s)));
    r = backward_data(n, 2, n->dB, n->dA);
    if (r != GF_OK) return r;
    // layer 2
    if (n->use_tc)
        NCK((dw_tensor<32, 32>(n, n->dA, 32, n->act[1], 32, n->grad + n->woff[1], n->grad + n->boff[1])));
    else NCK((conv_dw<32, 32>(n->dA, n->act[1], g, n->grad + n->woff[1], n->grad + n->boff[1], s)));
    r = backward_data(n, 1, n->dA, n->dB);
    if (r != GF_OK) return r;
    // layer 1 (no input gradient needed)
    if (n->use_tc)
        NCK((dw_tensor<128, 32>(n, n->dB, 32, f, 80, n->grad + n->woff[0], n->grad + n->boff[0])));
    else NCK((conv_dw<80, 32>(n->dB, f, g, n->grad + n->woff[0], n->grad + n->boff[0], s)));
    return GF_OK;
}

static bool device_ptr(const void *p) { return gf::pointer_kind(p) == gf::PTR_DEVICE; }

extern "C" {

size_t gf_net_param_count(void) { return (size_t)param_count(); }

int gf_net_create(const int dims[4], gf_net **out)
{
    if (!dims || !out) return GF_EINVAL;
    *out = nullptr;
    long V = 1;
    for (int m = 0; m < 4; ++m) {
        if (dims[m] < 3) return GF_EINVAL;
        V *= dims[m];
    }
    if (V >= (1L << 31)) return GF_EINVAL;
    gf_net *n = new (std::nothrow) gf_net;
    if (!n) return GF_ENOMEM;
    for (int m = 0; m < 4; ++m) n->g.L[m] = dims[m];
    n->g.V = (int)V;
    long off = 0;
    for (int l = 0; l < 4; ++l) {
        n->woff[l] = off;
        off += 81L * kC[l + 1] * kC[l];
        n->boff[l] = off;
        off += kC[l + 1];
    }
    n->np = off;
    *out = n;
    return GF_OK;
}

static int ensure_buffers(gf_net *n)
{
    if (n->params) return GF_OK;
    long V = n->g.V;
    NCK(cudaMalloc(&n->params, sizeof(float) * n->np));
    NCK(cudaMalloc(&n->grad, sizeof(float) * n->np));
    NCK(cudaMalloc(&n->m, sizeof(float) * n->np));
    NCK(cudaMalloc(&n->v, sizeof(float) * n->np));
    for (int l = 0; l < 4; ++l) {
        long cnt = 81L * kC[l + 1] * kC[l];
        NCK(cudaMalloc(&n->Wb[l], sizeof(bf16) * cnt));
        NCK(cudaMalloc(&n->Wt[l], sizeof(bf16) * cnt));
        NCK(cudaMalloc(&n->Wh[l], sizeof(bf16) * cnt));
        NCK(cudaMalloc(&n->Wth[l], sizeof(bf16) * cnt));
    }
    for (int l = 1; l < 4; ++l) NCK(cudaMalloc(&n->act[l], sizeof(bf16) * V * 32));
    NCK(cudaMalloc(&n->out, sizeof(float) * V * 8));
    NCK(cudaMalloc(&n->dA, sizeof(bf16) * V * 32));
    NCK(cudaMalloc(&n->dB, sizeof(bf16) * V * 32));
    if (halo_ok(n->g) || line_ok(n->g) || dw_line_ok(n->g))
        NCK(cudaMalloc(&n->xpad, sizeof(bf16) * padded_sites(n->g) * GF_NET_CIN));
    if (dw_line_ok(n->g)) NCK(cudaMalloc(&n->ypad, sizeof(bf16) * padded_sites(n->g) * 32));
    if (line_ok(n->g)) NCK(cudaMalloc(&n->ypad2, sizeof(bf16) * padded_sites(n->g) * 32));
    NCK(cudaMalloc(&n->partial, sizeof(double) * 1024));
    NCK(cudaMalloc(&n->dloss, sizeof(double)));
    NCK(cudaMalloc(&n->derr, sizeof(int)));
    NCK(cudaMemset(n->derr, 0, sizeof(int)));
    return GF_OK;
}

int gf_net_destroy(gf_net *n)
{
    if (!n) return GF_OK;
    cudaFree(n->params);
    cudaFree(n->grad);
    cudaFree(n->m);
    cudaFree(n->v);
    for (int l = 0; l < 4; ++l) {
        cudaFree(n->Wb[l]);
        cudaFree(n->Wt[l]);
        cudaFree(n->Wh[l]);
        cudaFree(n->Wth[l]);
    }
    for (int l = 1; l < 4; ++l) cudaFree(n->act[l]);
    cudaFree(n->out);
    cudaFree(n->dA);
    cudaFree(n->dB);
    cudaFree(n->xpad);
    cudaFree(n->ypad);
    cudaFree(n->ypad2);
    for (int l = 0; l < 4; ++l) cudaFree(n->xin[l]);
    cudaFree(n->partial);
    cudaFree(n->dloss);
    cudaFree(n->derr);
    delete n;
    return GF_OK;
}

const char *gf_net_last_error(const gf_net *n) { return n ? n->err.c_str() : "null network"; }

int gf_net_set_stream(gf_net *n, void *stream)
{
    if (!n) return GF_EINVAL;
    n->stream = (cudaStream_t)stream;
    return GF_OK;
}

int gf_net_set_params(gf_net *n, const float *params)
{
    if (!n || !params) return GF_EINVAL;
    int r = ensure_buffers(n);
    if (r != GF_OK) return r;
    NCK(cudaMemcpyAsync(n->params, params, sizeof(float) * n->np, cudaMemcpyDefault, n->stream));
    NCK(cudaMemsetAsync(n->m, 0, sizeof(float) * n->np, n->stream));
    NCK(cudaMemsetAsync(n->v, 0, sizeof(float) * n->np, n->stream));
    n->step = 0;
    r = refresh_weights(n);
    if (r != GF_OK) return r;
    NCK(cudaStreamSynchronize(n->stream));
    return GF_OK;
}

int gf_net_get_params(gf_net *n, float *params)
{
    if (!n || !params) return GF_EINVAL;
    if (!n->params) return nfail(n, GF_ESTATE, "parameters not set");
    NCK(cudaMemcpyAsync(params, n->params, sizeof(float) * n->np, cudaMemcpyDefault, n->stream));
    NCK(cudaStreamSynchronize(n->stream));
    return GF_OK;
}

int gf_net_forward(gf_net *n, const void *features, float *out)
{
    if (!n || !features || !out) return GF_EINVAL;
    if (!n->params) return nfail(n, GF_ESTATE, "parameters not set");
    if (!device_ptr(features) || !device_ptr(out)) return nfail(n, GF_EINVAL, "device pointers of the current device required");
    int r = forward(n, static_cast<const bf16 *>(features));
    if (r != GF_OK) return r;
    NCK(cudaMemcpyAsync(out, n->out, sizeof(float) * n->g.V * 8, cudaMemcpyDeviceToDevice, n->stream));
    return check_status(n);
}

int gf_net_set_option(gf_net *n, const char *key, double value)
{
    if (!n || !key) return GF_EINVAL;
    if (std::string(key) == "tensor_cores") {
        n->use_tc = value != 0.0;
        return GF_OK;
    }
    if (std::string(key) == "conv_halo") {
        if (value != 0.0 && value != 1.0 && value != 2.0) return nfail(n, GF_EINVAL, "conv_halo is 0, 1 or 2");
        n->use_halo = (int)value;
        return GF_OK;
    }
    return nfail(n, GF_EINVAL, std::string("unknown option ") + key);
}

int gf_net_gradient(gf_net *n, const void *features, const float *target, float *grad, double *loss)
{
    if (!n || !features || !target) return GF_EINVAL;
    if (!n->params) return nfail(n, GF_ESTATE, "parameters not set");
    if (!device_ptr(features) || !device_ptr(target)) return nfail(n, GF_EINVAL, "device pointers of the current device required");
    int r = backward(n, static_cast<const bf16 *>(features), target);
    if (r != GF_OK) return r;
    if (grad) NCK(cudaMemcpyAsync(grad, n->grad, sizeof(float) * n->np, cudaMemcpyDefault, n->stream));
    if (loss) NCK(cudaMemcpyAsync(loss, n->dloss, sizeof(double), cudaMemcpyDefault, n->stream));
    return check_status(n);
}

int gf_net_train_step(gf_net *n, const void *features, const float *target, float lr, double *loss)
{
    if (!n || !features || !target || !(lr > 0.0f)) return GF_EINVAL;
    if (!n->params) return nfail(n, GF_ESTATE, "parameters not set");
    int r = backward(n, static_cast<const bf16 *>(features), target);
    if (r != GF_OK) return r;
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.0f / (1.0f - powf(b1, (float)n->step));
    float c2 = 1.0f / (1.0f - powf(b2, (float)n->step));
    WeightCopies wc;
    for (int l = 0; l < 4; ++l) {
        wc.woff[l] = n->woff[l];
        wc.I[l] = kC[l];
        wc.O[l] = kC[l + 1];
        wc.Wb[l] = n->Wb[l];
        wc.Wt[l] = n->Wt[l];
        wc.Wh[l] = n->Wh[l];
        wc.Wth[l] = n->Wth[l];
    }
    k_adam<<<(int)((n->np + 255) / 256), 256, 0, n->stream>>>(n->params, n->grad, n->m, n->v, n->np, lr, b1, b2,
                                                              1e-8f, c1, c2, wc);
    NCK(cudaGetLastError());
    if (loss) NCK(cudaMemcpyAsync(loss, n->dloss, sizeof(double), cudaMemcpyDefault, n->stream));
    return check_status(n);
}

}  // extern "C"
