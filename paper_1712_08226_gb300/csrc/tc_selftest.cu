// Self-test of the tensor-core primitives (tc.cuh): one thread block computes
// D[128 x N] = A[128 x K] B[N x K]^T with tcgen05.mma (kind::tf32) into tensor
// memory and reads it back with tcgen05.ld.  Used by the tests to check the
// operand layout, the descriptors and the accumulator read-out exactly.
#include "common.cuh"
#include "tc.cuh"

namespace hopf {

__global__ void __launch_bounds__(128) tc_selftest_kernel(int N, int K, const float *__restrict__ A,
                                                          const float *__restrict__ B, float *__restrict__ D,
                                                          int *err) {
    extern __shared__ __align__(1024) unsigned char tc_sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_taddr;
    const int KB = K * 4;
    unsigned char *As = tc_sm, *Bs = tc_sm + 128 * KB;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tc::tmem_alloc(&s_taddr, 256);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    for (int e = tid; e < 128 * K; e += 128) {
        int r = e / K, k = e % K;
        *reinterpret_cast<float *>(As + tc::core_offset(r, k, KB, 4)) = A[e];
    }
    for (int e = tid; e < N * K; e += 128) {
        int r = e / K, k = e % K;
        *reinterpret_cast<float *>(Bs + tc::core_offset(r, k, KB, 4)) = B[e];
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = s_taddr;
    if (tid == 0) {
        const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs);
        const uint32_t idesc = tc::make_idesc(128, N, tc::FMT_TF32);
        const uint32_t sbo = (uint32_t)(KB / 16) * 128u;
        for (int kc = 0; kc < K / 8; ++kc) {
            const uint64_t ad = tc::make_desc(a0 + 2u * kc * 128u, 128u, sbo);
            const uint64_t bd = tc::make_desc(b0 + 2u * kc * 128u, 128u, sbo);
            tc::mma_tf32(taddr, ad, bd, idesc, kc > 0 ? 1u : 0u);
        }
        tc::mma_commit(&mbar);
    }
    bool ok = tc::mbar_wait(&mbar, 0);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
        if ((tid & 31) == 0) atomicExch(err, 1);
        tc::mbar_wait(&mbar, 0);              // give in-flight work a second bounded chance
    }
    tc::fence_after_sync();
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) D[(size_t)tid * N + c0 + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 256);
}

cudaError_t launch_tc_selftest(int N, int K, const float *A, const float *B, float *D, int *err, cudaStream_t s) {
    const size_t smem = (size_t)(128 + N) * K * 4;
    cudaError_t e = cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tc_selftest_kernel<<<1, 128, smem, s>>>(N, K, A, B, D, err);
    return cudaGetLastError();
}

}  // namespace hopf
