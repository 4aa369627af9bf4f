// Blackwell (sm_103a) tensor-core primitives in inline PTX: TMEM allocation,
// tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulator in TMEM), commit to
// an mbarrier, bounded mbarrier waits and TMEM loads. Used by the MLP
// kernels (mlp.cu) for their GEMMs.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// "core matrices" of 8 rows x 16 bytes (8 bf16), 128 contiguous bytes each.
// An operand tile of R rows (R a multiple of 8) and K = 16 (one MMA step) is
// stored as [R/8 row groups][2 K halves][8 rows][8 values]: the two K halves
// of a row group are 128 bytes apart (leading-dimension byte offset, LBO)
// and consecutive row groups 256 bytes apart (stride-dimension byte offset,
// SBO). Successive K steps follow each other (R * 32 bytes apart).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace vl {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row r, k) of a K-major operand with R rows
__host__ __device__ constexpr int kmajor_offset(int r, int k, int R) {
    return (k >> 4) * (R * 32) + (r >> 3) * 256 + ((k >> 3) & 1) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor (no swizzle, K-major)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);          // start address
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;      // LBO: next K half
    d |= (uint64_t)((256u >> 4) & 0x3FFFu) << 32;      // SBO: next 8-row group
    d |= (uint64_t)1 << 46;                            // descriptor version (tcgen05)
    return d;                                          // base offset 0, no swizzle
}

// instruction descriptor: D = FP32, A = B = BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4)                     // D format: F32
         | (1u << 7)                     // A format: BF16
         | (1u << 10)                    // B format: BF16
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

// ---- TMEM allocation (one full warp) ------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---- fences ---------------------------------------------------------------------
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// ---- mbarrier -----------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// Waits for the phase with the given parity to complete; gives up after
// max_tries polls and returns false (the caller records an error).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t max_tries = (1u << 24)) {
    const uint32_t a = smem_addr(bar);
    for (uint32_t i = 0; i < max_tries; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ---- MMA (one thread) ----------------------------------------------------------
// D[tmem] (+)= A[smem] * B[smem]^T for one K = 16 step
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// the mbarrier completes one arrival when all MMAs issued so far by this
// thread have completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// D[128 x N] (+)= A[128 x K] * B[N x K]^T, both operands K-major in shared
// memory (kmajor_offset layout with R = 128 and R = N); one thread issues
// K / 16 MMAs.
__device__ __forceinline__ void gemm_issue(uint32_t tmem_d, const void* A, const void* B, int N, int K,
                                           bool accumulate) {
    const uint32_t a0 = smem_addr(A), b0 = smem_addr(B);
    const uint32_t idesc = idesc_bf16(128, N);
    for (int ks = 0; ks < K / 16; ++ks) {
        const uint64_t ad = smem_desc(a0 + ks * 128 * 32);
        const uint64_t bd = smem_desc(b0 + ks * N * 32);
        mma_bf16(tmem_d, ad, bd, idesc, (accumulate || ks > 0) ? 1u : 0u);
    }
}

// ---- TMEM -> registers: 16 consecutive FP32 columns of this thread's lane ----
// (warp w reads lanes 32 (w mod 4) .. +31; lane = thread's row)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// TMEM address of (lane, column) relative to a base
__device__ __forceinline__ uint32_t tmem_at(uint32_t base, int lane, int col) {
    return base + ((uint32_t)lane << 16) + (uint32_t)col;
}

}  // namespace tc
}  // namespace vl
