// gf_conv_tc.cuh -- periodic 4D convolution with 3^4 taps as an implicit GEMM
// on the 5th-generation tensor cores (tcgen05, sm_103a):
//
//   Y[s][o] = b[o] + sum_k sum_i W[k][o][i] X[nb(s, k)][i],  nb(s,k) = s + sign d(k)
//
// One CTA (128 threads) computes a tile of M = 128 output sites x N output
// channels (N = 16 or 32) with FP32 accumulators in tensor memory.  The
// reduction runs over the 81 taps, each tap contributing K = I_pad (input
// channels padded to 16) in steps of 16: for every tap the CTA gathers the
// 128 neighbour rows X[nb(s,k)][:] (A, 128 x I_pad, BF16) and the weights
// W[k][:][:] (B, N x I_pad, BF16) into shared memory in the canonical
// K-major no-swizzle layout (8-row x 16-byte core matrices), and one thread
// issues the tcgen05.mma instructions; a tcgen05.commit arrives on the
// stage's mbarrier when they have consumed the stage.  NSTAGE stages let the
// gather of tap k+1.. overlap the MMAs of tap k.  Epilogue: tcgen05.ld of the
// accumulator rows (warp w reads lanes 32w..32w+31), bias, ReLU or a ReLU
// mask, BF16/FP32 store.
//
// Every wait is bounded (%globaltimer, 1 s): on expiry the kernel records an
// error code, waits (bounded) for its own outstanding MMAs, frees its tensor
// memory and returns.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace gf {
namespace tc {

constexpr int kThreads = 128;
constexpr int kM = 128;
constexpr int kStages = 4;
constexpr long long kWaitNs = 1000000000LL;  // 1 s
constexpr int kGuardBytes = 0;  // no slack needed after the operand stages: operands stay inside their stage

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ long long now_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    long long t0 = now_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (now_ns() - t0 > kWaitNs) return false;
    }
    return true;
}

// Shared-memory matrix descriptor, K-major, no swizzle: start address,
// leading-dimension byte offset (between the two 8-element core columns of a
// K = 16 step), stride-dimension byte offset (between 8-row groups), version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;                // base offset 0, layout: no swizzle
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace tc
}  // namespace gf
