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

// ------------------------------------------------------------ host drivers
long long mlp_param_count(int n_in, int h, int n_out) { return MlpDims{n_in, h, n_out}.count(); }

// scratch floats for a batch of B: h0, a1, h1, a2, h2, out (+ gradients for training)
long long mlp_scratch_floats(int n_in, int h, int n_out, int B, bool train) {
    long long f = (long long)B * (n_in + 4LL * h + n_out);
    if (train) f += (long long)B * (2LL * h + n_out) + 8;
    return f;
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
