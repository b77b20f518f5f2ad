// Warm-start network: forward, backward and Adam kernels.
//
// The network maps a query point x to a prediction of the optimal dual p*
// (used as the primal warm start of the primal-dual iteration):
//   h0 = (x - x_shift) / x_scale
//   h1 = gelu(W1 h0 + b1),  h2 = gelu(W2 h1 + b2),  out = W3 h2 + b3
//   prediction = out * y_scale + y_shift,
// with the exact GELU g(a) = a (1 + erf(a / sqrt 2)) / 2.  Weights are used
// as bfloat16 (a float32 master copy is kept for the optimiser), every
// product accumulates in float32.  The loss is the mean squared error of
// `out` against the standardised target.  The paper has no learned part.
//
// Parameter layout (float32 master and bfloat16 copy share offsets):
//   W1 [h][n_in], b1 [h], W2 [h][h], b2 [h], W3 [n_out][h], b3 [n_out].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "tc.cuh"

namespace hopf {

struct MlpDims {
    int n_in, h, n_out;
    __host__ __device__ long long oW1() const { return 0; }
    __host__ __device__ long long ob1() const { return (long long)h * n_in; }
    __host__ __device__ long long oW2() const { return ob1() + h; }
    __host__ __device__ long long ob2() const { return oW2() + (long long)h * h; }
    __host__ __device__ long long oW3() const { return ob2() + h; }
    __host__ __device__ long long ob3() const { return oW3() + (long long)n_out * h; }
    __host__ __device__ long long count() const { return ob3() + n_out; }
};

__device__ __forceinline__ float gelu_f(float a) { return 0.5f * a * (1.f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float a) {
    return 0.5f * (1.f + erff(a * 0.70710678118654752f)) + a * 0.39894228040143268f * expf(-0.5f * a * a);
}

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// C[M x N] = opA(A)[M x K] * opB(B)[K x N], fp32 accumulation.
//   opA(A)[i][k] = TA ? A[k*lda + i] : A[i*lda + k]
//   opB(B)[k][j] = TB ? B[j*ldb + k] : B[k*ldb + j]
// 64 x 64 block tile, k-chunks of 16 staged in shared memory, 256 threads each
// computing a 4 x 4 sub-tile; the epilogue functor writes the result.
constexpr int GT = 64, GK = 16;

template <bool TA, bool TB, typename TBT, class Epi>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float *__restrict__ A, int lda,
                                                   const TBT *__restrict__ B, int ldb, Epi epi) {
    __shared__ float As[GK][GT + 4];
    __shared__ float Bs[GK][GT + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            int r, kk;
            if (TA) { kk = e / GT; r = e % GT; }     // consecutive threads along i (contiguous for TA)
            else { r = e / GK; kk = e % GK; }        // consecutive threads along k
            int gi = i0 + r, gk = k0 + kk;
            float v = 0.f;
            if (gi < M && gk < K) v = TA ? A[(long long)gk * lda + gi] : A[(long long)gi * lda + gk];
            As[kk][r] = v;
        }
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            int c, kk;
            if (TB) { c = e / GK; kk = e % GK; }
            else { kk = e / GT; c = e % GT; }
            int gj = j0 + c, gk = k0 + kk;
            float v = 0.f;
            if (gj < N && gk < K) v = TB ? to_f(B[(long long)gj * ldb + gk]) : to_f(B[(long long)gk * ldb + gj]);
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[kk][ty * 4 + u];
#pragma unroll
            for (int u = 0; u < 4; ++u) b[u] = Bs[kk][tx * 4 + u];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
            if (i < M && j < N) epi(i, j, acc[u][v]);
        }
}

// ---- epilogues
struct EpiBiasGelu {           // hidden layer forward: a = acc + b; store a (optional) and gelu(a)
    const float *b;
    float *pre;                // may be null (inference)
    float *act;
    int ld;
    __device__ void operator()(int i, int j, float acc) const {
        float a = acc + b[j];
        if (pre) pre[(long long)i * ld + j] = a;
        act[(long long)i * ld + j] = gelu_f(a);
    }
};
struct EpiBiasOut {            // output layer: out = acc + b (optionally de-standardised)
    const float *b;
    float *out;
    int ld;
    const float *y_shift, *y_scale;   // null: standardised output
    __device__ void operator()(int i, int j, float acc) const {
        float o = acc + b[j];
        if (y_scale) o = fmaf(o, y_scale[j], y_shift[j]);
        out[(long long)i * ld + j] = o;
    }
};
struct EpiStore {              // plain store (weight gradients)
    float *C;
    int ld;
    __device__ void operator()(int i, int j, float acc) const { C[(long long)i * ld + j] = acc; }
};
struct EpiGeluBack {           // dA_prev = dH * gelu'(A_prev)
    const float *pre;
    float *dpre;
    int ld;
    __device__ void operator()(int i, int j, float acc) const {
        long long e = (long long)i * ld + j;
        dpre[e] = acc * gelu_grad_f(pre[e]);
    }
};

template <bool TA, bool TB, typename TBT, class Epi>
cudaError_t gemm(int M, int N, int K, const float *A, int lda, const TBT *B, int ldb, Epi epi, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
    gemm_kernel<TA, TB, TBT, Epi><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, epi);
    return cudaGetLastError();
}

__global__ void standardize_kernel(int B, int n, const float *x, const float *shift, const float *scale, float *h0) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)B * n) return;
    int j = (int)(e % n);
    h0[e] = (x[e] - shift[j]) / scale[j];
}

// d loss / d out for loss = sum (out - (y - y_shift)/y_scale)^2 / (B n_out); loss accumulated in *loss.
__global__ void mse_grad_kernel(int B, int n_out, const float *out, const float *y, const float *y_shift,
                                const float *y_scale, float *dout, float *loss) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float part = 0.f;
    if (e < (long long)B * n_out) {
        int j = (int)(e % n_out);
        float d = out[e] - (y[e] - y_shift[j]) / y_scale[j];
        float inv = 1.f / ((float)B * (float)n_out);
        dout[e] = 2.f * d * inv;
        part = d * d * inv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && part != 0.f) atomicAdd(loss, part);
}

// column sums: db[j] = sum_i dA[i][j]
__global__ void colsum_kernel(int B, int n, const float *dA, float *db) {
    int j = blockIdx.x;
    float s = 0.f;
    for (int i = threadIdx.x; i < B; i += blockDim.x) s += dA[(long long)i * n + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) db[j] = s;
    }
}

// Adam (Kingma and Ba 2015) with bias correction; also refreshes the bf16 copy.
__global__ void adam_kernel(long long count, float *w, __nv_bfloat16 *wb, const float *g, float *m, float *v,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    float gi = g[e];
    float mi = fmaf(b1, m[e], (1.f - b1) * gi);
    float vi = fmaf(b2, v[e], (1.f - b2) * gi * gi);
    m[e] = mi;
    v[e] = vi;
    float wi = w[e] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[e] = wi;
    wb[e] = __float2bfloat16_rn(wi);
}

__global__ void to_bf16_kernel(long long count, const float *w, __nv_bfloat16 *wb) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) wb[e] = __float2bfloat16_rn(w[e]);
}

// C[M x N] = A[M x K] W[N x K]^T on the tensor cores (tcgen05.mma, kind::f16):
// A (float32 activations) and W (bfloat16 weights) are staged in shared memory
// as bfloat16, in K chunks of 64, in the core-matrix layout of tc.cuh; the
// float32 accumulator (128 rows x up to 256 columns) lives in tensor memory
// and the epilogue functor writes the result.  One 128-thread block per 128
// rows (thread t owns row t, i.e. tensor-memory lane t); N <= 256.
constexpr int TC_KC = 64;

template <class Epi>
__global__ void __launch_bounds__(128) gemm_tc_kernel(int M, int N, int K, const float *__restrict__ A, int lda,
                                                      const __nv_bfloat16 *__restrict__ W, int ldw, Epi epi,
                                                      int *err) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_taddr;
    const int Np = (N + 15) & ~15;
    constexpr int KB = TC_KC * 2;                 // bytes per staged row
    unsigned char *As = gsm, *Ws = gsm + 128 * KB;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row0 = blockIdx.x * 128;
    if (warp == 0) tc::tmem_alloc(&s_taddr, 256);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = s_taddr;
    const uint32_t idesc = tc::make_idesc(128, Np, tc::FMT_BF16);
    const int nchunks = (K + TC_KC - 1) / TC_KC;
    int ok = 1;
    for (int ch = 0; ch < nchunks && ok; ++ch) {
        const int k0 = ch * TC_KC;
        for (int e = tid; e < 128 * TC_KC; e += 128) {
            const int r = e / TC_KC, k = e % TC_KC;
            const int gr = row0 + r, gk = k0 + k;
            const float v = (gr < M && gk < K) ? A[(size_t)gr * lda + gk] : 0.f;
            *reinterpret_cast<__nv_bfloat16 *>(As + tc::core_offset(r, k, KB, 2)) = __float2bfloat16_rn(v);
        }
        for (int e = tid; e < Np * TC_KC; e += 128) {
            const int r = e / TC_KC, k = e % TC_KC;
            const int gk = k0 + k;
            const __nv_bfloat16 v = (r < N && gk < K) ? W[(size_t)r * ldw + gk] : __float2bfloat16_rn(0.f);
            *reinterpret_cast<__nv_bfloat16 *>(Ws + tc::core_offset(r, k, KB, 2)) = v;
        }
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Ws);
            const uint32_t sbo = (uint32_t)(KB / 16) * 128u;
#pragma unroll
            for (int kc = 0; kc < TC_KC / 16; ++kc)
                tc::mma_bf16(taddr, tc::make_desc(a0 + 2u * kc * 128u, 128u, sbo),
                             tc::make_desc(b0 + 2u * kc * 128u, 128u, sbo), idesc, (ch > 0 || kc > 0) ? 1u : 0u);
            tc::mma_commit(&mbar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&mbar, (uint32_t)(ch & 1)) ? 1 : 0);
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        tc::mbar_wait(&mbar, (uint32_t)((nchunks - 1) & 1));   // second bounded chance for work in flight
    }
    tc::fence_after_sync();
    if (ok) {
        const int row = row0 + tid;
        for (int c0 = 0; c0 < Np; c0 += 16) {
            float v[16];
            tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row < M) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (c0 + i < N) epi(row, c0 + i, v[i]);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 256);
}

template <class Epi>
cudaError_t gemm_tc(int M, int N, int K, const float *A, int lda, const __nv_bfloat16 *W, int ldw, Epi epi, int *err,
                    cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    // 100 KB of dynamic shared memory keeps at most two blocks (2 x 256 tensor-memory columns) per SM
    const size_t smem = 100 * 1024;
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gemm_tc_kernel<Epi><<<(M + 127) / 128, 128, smem, s>>>(M, N, K, A, lda, W, ldw, epi, err);
    return cudaGetLastError();
}

// ------------------------------------------------------------ host drivers
long long mlp_param_count(int n_in, int h, int n_out) { return MlpDims{n_in, h, n_out}.count(); }

// scratch floats for a batch of B: h0, a1, h1, a2, h2, out (+ gradients for training)
long long mlp_scratch_floats(int n_in, int h, int n_out, int B, bool train) {
    long long f = (long long)B * (n_in + 4LL * h + n_out);
    if (train) f += (long long)B * (2LL * h + n_out) + 8;
    return f;
}

cudaError_t mlp_forward_tc(int n_in, int h, int n_out, const __nv_bfloat16 *wb, const float *w,
                           const float *x_shift, const float *x_scale, const float *y_shift, const float *y_scale,
                           int B, const float *x, float *y, float *scratch, int *err, cudaStream_t s) {
    MlpDims d{n_in, h, n_out};
    float *h0 = scratch, *h1 = h0 + (long long)B * n_in + (long long)B * h, *h2 = h1 + (long long)B * h + (long long)B * h;
    long long tot = (long long)B * n_in;
    standardize_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(B, n_in, x, x_shift, x_scale, h0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = gemm_tc(B, h, n_in, h0, n_in, wb + d.oW1(), n_in, EpiBiasGelu{w + d.ob1(), nullptr, h1, h}, err, s);
    if (e != cudaSuccess) return e;
    e = gemm_tc(B, h, h, h1, h, wb + d.oW2(), h, EpiBiasGelu{w + d.ob2(), nullptr, h2, h}, err, s);
    if (e != cudaSuccess) return e;
    return gemm_tc(B, n_out, h, h2, h, wb + d.oW3(), h, EpiBiasOut{w + d.ob3(), y, n_out, y_shift, y_scale}, err, s);
}

cudaError_t mlp_forward(int n_in, int h, int n_out, const __nv_bfloat16 *wb, const float *w, const float *x_shift,
                        const float *x_scale, const float *y_shift, const float *y_scale, int B, const float *x,
                        float *y, float *scratch, bool keep_pre, cudaStream_t s) {
    MlpDims d{n_in, h, n_out};
    float *h0 = scratch, *a1 = h0 + (long long)B * n_in, *h1 = a1 + (long long)B * h, *a2 = h1 + (long long)B * h,
          *h2 = a2 + (long long)B * h;
    long long tot = (long long)B * n_in;
    standardize_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(B, n_in, x, x_shift, x_scale, h0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = gemm<false, true>(B, h, n_in, h0, n_in, wb + d.oW1(), n_in, EpiBiasGelu{w + d.ob1(), keep_pre ? a1 : nullptr, h1, h}, s);
    if (e != cudaSuccess) return e;
    e = gemm<false, true>(B, h, h, h1, h, wb + d.oW2(), h, EpiBiasGelu{w + d.ob2(), keep_pre ? a2 : nullptr, h2, h}, s);
    if (e != cudaSuccess) return e;
    return gemm<false, true>(B, n_out, h, h2, h, wb + d.oW3(), h, EpiBiasOut{w + d.ob3(), y, n_out, y_shift, y_scale}, s);
}

// Forward in standardised units, loss and full gradient (count() floats in grad).
cudaError_t mlp_loss_grad(int n_in, int h, int n_out, const __nv_bfloat16 *wb, const float *w, const float *x_shift,
                          const float *x_scale, const float *y_shift, const float *y_scale, int B, const float *x,
                          const float *y, float *loss, float *grad, float *scratch, cudaStream_t s) {
    MlpDims d{n_in, h, n_out};
    float *h0 = scratch, *a1 = h0 + (long long)B * n_in, *h1 = a1 + (long long)B * h, *a2 = h1 + (long long)B * h,
          *h2 = a2 + (long long)B * h, *out = h2 + (long long)B * h;
    float *dout = out + (long long)B * n_out, *dA2 = dout + (long long)B * n_out, *dA1 = dA2 + (long long)B * h;
    cudaError_t e = mlp_forward(n_in, h, n_out, wb, w, x_shift, x_scale, nullptr, nullptr, B, x, out, scratch, true, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    long long tot = (long long)B * n_out;
    mse_grad_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(B, n_out, out, y, y_shift, y_scale, dout, loss);
    // layer 3: dW3 = dout^T h2, db3 = colsum(dout), dA2 = (dout W3) * gelu'(a2)
    e = gemm<true, false>(n_out, h, B, dout, n_out, h2, h, EpiStore{grad + d.oW3(), h}, s);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<n_out, 256, 0, s>>>(B, n_out, dout, grad + d.ob3());
    e = gemm<false, false>(B, h, n_out, dout, n_out, wb + d.oW3(), h, EpiGeluBack{a2, dA2, h}, s);
    if (e != cudaSuccess) return e;
    // layer 2
    e = gemm<true, false>(h, h, B, dA2, h, h1, h, EpiStore{grad + d.oW2(), h}, s);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<h, 256, 0, s>>>(B, h, dA2, grad + d.ob2());
    e = gemm<false, false>(B, h, h, dA2, h, wb + d.oW2(), h, EpiGeluBack{a1, dA1, h}, s);
    if (e != cudaSuccess) return e;
    // layer 1
    e = gemm<true, false>(h, n_in, B, dA1, h, h0, n_in, EpiStore{grad + d.oW1(), n_in}, s);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<h, 256, 0, s>>>(B, h, dA1, grad + d.ob1());
    return cudaGetLastError();
}

cudaError_t mlp_adam(long long count, float *w, __nv_bfloat16 *wb, const float *g, float *m, float *v, float lr,
                     float b1, float b2, float eps, int step, cudaStream_t s) {
    float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, w, wb, g, m, v, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t mlp_sync_bf16(long long count, const float *w, __nv_bfloat16 *wb, cudaStream_t s) {
    to_bf16_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, w, wb);
    return cudaGetLastError();
}

}  // namespace hopf
