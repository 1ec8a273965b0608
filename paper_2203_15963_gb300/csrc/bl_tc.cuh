// Fifth-generation tensor-core primitives for sm_103a (inline PTX): tensor-memory allocation,
// single-CTA BF16 MMA with FP32 accumulation in tensor memory, completion through an
// mbarrier, and tensor-memory loads.
//
// Operand layout: K-major without swizzle. A tile of R rows x K columns of bf16 is a grid of
// 8 x 8 "core matrices" (8 rows of 16 bytes, 128 contiguous bytes); core matrix (r/8, k/8)
// starts at (r/8) (K/8) 128 + (k/8) 128 bytes. In the shared-memory descriptor the leading
// byte offset (adjacent core matrices along K) is 128 and the stride byte offset (adjacent
// core matrices along M or N) is (K/8) 128; one MMA consumes K = 16 (two core matrices), so
// step s of a longer K starts 256 s bytes further.
// Accumulator (M = 128, cta_group::1): row m of D is tensor-memory lane m, column n is column
// n (FP32). Warp w of the CTA may access lanes 32 (w % 4) .. 32 (w % 4) + 31.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace bl {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) in a K-major no-swizzle tile with K columns
__host__ __device__ constexpr uint32_t kmajor(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void st_bf16(unsigned char* tile, int r, int k, int K, float v) {
    *reinterpret_cast<__nv_bfloat16*>(tile + kmajor(r, k, K)) = __float2bfloat16_rn(v);
}

// two floats rounded to bf16 (nearest even) and packed, a in the low half (the lower column)
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// Shared-memory matrix descriptor: start address, leading / stride byte offsets (all >> 4),
// descriptor version 1 (bits 46-47), base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// descriptor of K-step s of a K-major tile with K columns
__device__ __forceinline__ uint64_t kdesc(const void* tile, int K, int s) {
    return sdesc(smem_addr(tile) + 256u * (uint32_t)s, 128u, (uint32_t)(K >> 3) * 128u);
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 =
// 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// --- tensor memory (one full warp executes these) ---
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_addr(dst_smem)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// --- ordering ---
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes made visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_smem_to_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// --- mbarrier ---
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity to complete, for at most ~max_cycles SM cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long max_cycles) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (clock64() - t0 < max_cycles)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// --- MMA (issued by one thread) ---
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, bool accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate ? 1u : 0u));
}
// D[M=128][N] (+)= A[128][K] B[N][K]^T over K in steps of 16
__device__ __forceinline__ void gemm_bf16(uint32_t d_tmem, const void* A, const void* B, int N,
                                          int K) {
    const uint32_t id = idesc_bf16_f32(128, N);
    for (int s = 0; s < (K >> 4); ++s) mma_bf16(d_tmem, kdesc(A, K, s), kdesc(B, K, s), id, s > 0);
}
// arrive on bar once every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_addr(bar)) : "memory");
}

// --- tensor-memory loads (warp-collective): 16 consecutive FP32 columns of this thread's
// lane. The wait is tied to the destination registers (in/out operands), so no use of them
// can be scheduled before the load has completed.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
                 "%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
// address of (this warp's first lane, column col)
__device__ __forceinline__ uint32_t tmem_lane_addr(uint32_t base, int col) {
    const uint32_t warp = (threadIdx.x >> 5) & 3u;
    return base + ((warp * 32u) << 16) + (uint32_t)col;
}

}  // namespace tc
}  // namespace bl
