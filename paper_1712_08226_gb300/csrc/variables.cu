// Maps between the paper's variable p of Eq. 18 and the terminal-time
// variable q of the substitution p = e^{T A^T} q.
//
// The substitution leaves every term of Eq. 18 in place: <z0, p> = <e^{TA} z0, q>,
// so the query point enters the iteration as x' = e^{TA} x; a warm start p0
// enters as q0 = e^{-T A^T} p0; the solution q* leaves as p* = e^{T A^T} q*.
// E = e^{TA} and Ei = e^{-TA} come from the float64 node-table instance of
// each point's horizon (tables.cu).  One thread per output component, float64
// accumulation, result rounded to the caller's element type.
#include "common.cuh"

namespace hopf {

template <typename R>
__global__ void to_terminal_kernel(const double *__restrict__ inst64, InstanceLayout L, int inst_stride, int P, int n,
                                   const R *__restrict__ x, const R *__restrict__ p0, R *__restrict__ xq,
                                   R *__restrict__ q0, const int *__restrict__ active) {
    const long long total = (long long)P * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), i = (int)(e % n);
        if (active && !active[k]) continue;
        const double *I = inst64 + (inst_stride ? (long long)k * L.stride : 0LL);
        const double *E = I + L.E + (long long)i * n;            // row i of e^{TA}
        const R *xk = x + (long long)k * n;
        double s = 0.0;
        for (int j = 0; j < n; ++j) s = fma(E[j], (double)xk[j], s);
        xq[e] = (R)s;
        if (p0) {
            const double *Ei = I + L.Ei + i;                      // column i of e^{-TA}
            const R *pk = p0 + (long long)k * n;
            double t = 0.0;
            for (int j = 0; j < n; ++j) t = fma(Ei[(long long)j * n], (double)pk[j], t);
            q0[e] = (R)t;
        }
    }
}

template <typename R>
__global__ void from_terminal_kernel(const double *__restrict__ inst64, InstanceLayout L, int inst_stride, int P,
                                     int n, const R *__restrict__ q, R *__restrict__ p,
                                     const int *__restrict__ active) {
    const long long total = (long long)P * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), i = (int)(e % n);
        if (active && !active[k]) continue;
        const double *E = inst64 + (inst_stride ? (long long)k * L.stride : 0LL) + L.E + i;   // column i
        const R *qk = q + (long long)k * n;
        double s = 0.0;
        for (int j = 0; j < n; ++j) s = fma(E[(long long)j * n], (double)qk[j], s);
        p[e] = (R)s;
    }
}

static int map_grid(long long total) {
    long long g = (total + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 65535 ? 65535 : g));
}

template <typename R>
cudaError_t launch_to_terminal(const double *inst64, int n, int m, int N, int inst_stride, int P, const R *x,
                               const R *p0, R *xq, R *q0, const int *active, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    to_terminal_kernel<R><<<map_grid((long long)P * n), 256, 0, s>>>(inst64, L, inst_stride, P, n, x, p0, xq, q0,
                                                                     active);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_from_terminal(const double *inst64, int n, int m, int N, int inst_stride, int P, const R *q,
                                 R *p, const int *active, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    from_terminal_kernel<R><<<map_grid((long long)P * n), 256, 0, s>>>(inst64, L, inst_stride, P, n, q, p, active);
    return cudaGetLastError();
}

template cudaError_t launch_to_terminal<float>(const double *, int, int, int, int, int, const float *, const float *,
                                               float *, float *, const int *, cudaStream_t);
template cudaError_t launch_to_terminal<double>(const double *, int, int, int, int, int, const double *,
                                                const double *, double *, double *, const int *, cudaStream_t);
template cudaError_t launch_from_terminal<float>(const double *, int, int, int, int, int, const float *, float *,
                                                 const int *, cudaStream_t);
template cudaError_t launch_from_terminal<double>(const double *, int, int, int, int, int, const double *, double *,
                                                  const int *, cudaStream_t);

}  // namespace hopf
