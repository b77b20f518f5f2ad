// Blackwell (sm_103a) tensor-core primitives used by the large-state kernels:
// tensor-memory allocation, shared-memory matrix descriptors, tcgen05.mma of
// kind::tf32 with float32 accumulation in tensor memory, completion through
// an mbarrier, and tcgen05.ld of the accumulator.  Written from the PTX ISA
// description of the tcgen05 instructions.
//
// Operand layout in shared memory (no swizzle, "K-major"): a tile of R rows
// by KB bytes per row is stored as core matrices of 8 rows x 16 bytes
// (128 contiguous bytes, row r of the core matrix at byte 16 r).  Core matrix
// (row group g, 16-byte chunk c) sits at byte offset (g * (KB / 16) + c) * 128.
// In the descriptor, the leading byte offset is the distance between core
// matrices adjacent along K (128 bytes here) and the stride byte offset the
// distance between adjacent 8-row groups ((KB / 16) * 128 bytes).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hopf {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, k) of a K-major tile with kb bytes per row and
// elements of esz bytes, in the core-matrix layout above
__device__ __forceinline__ uint32_t core_offset(int row, int k, int kb, int esz) {
    const int byte = k * esz;
    return (uint32_t)(((row >> 3) * (kb >> 4) + (byte >> 4)) * 128 + (row & 7) * 16 + (byte & 15));
}

// shared-memory matrix descriptor (no swizzle)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;                          // descriptor version for tcgen05
    return d;                                        // base offset 0, no swizzle
}

// instruction descriptor: D float32, A and B of format ab (2 = tf32), both K-major
__host__ __device__ __forceinline__ uint32_t make_idesc(int M, int N, uint32_t ab) {
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t FMT_TF32 = 2;   // with kind::tf32
constexpr uint32_t FMT_BF16 = 1;   // with kind::f16

// allocate ncols tensor-memory columns (power of two >= 32); whole warp
__device__ __forceinline__ void tmem_alloc(uint32_t *smem_dst, int ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (tmem) (+)= A (smem desc) * B (smem desc)^T, issued by one thread
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// same with bf16 operands (kind::f16, K = 16 per instruction)
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive on the mbarrier once every tcgen05.mma issued so far by this thread completes
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// bounded wait on an mbarrier phase; false if the bound was hit
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t phase, long long max_spins = (1LL << 26)) {
    for (long long i = 0; i < max_spins; ++i)
        if (mbar_try_wait(mbar, phase)) return true;
    return false;
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes become visible to the tensor core
__device__ __forceinline__ void fence_smem_to_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16 consecutive accumulator columns of this thread's lane (warp w reads
// lanes 32 w .. 32 w + 31); taddr already carries the lane offset
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace hopf
