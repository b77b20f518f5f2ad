// Fixed-step quadrature: the left Riemann sum with a step that does not
// depend on the horizon, dt = t_max / N.  Horizon T uses the nodes
// t_i = i dt with t_i < T, i.e. the first nk = ceil(T / dt) of them, each
// weighted dt except the last, weighted T - (nk - 1) dt (§III.A allows other
// quadratures than its N equal steps of T / N; at T = k dt this is Eq. 17
// with k nodes).
//
// In terminal-time variables (p = e^{T A^T} q) the node matrices are
// K'_i = (-e^{t_i A} B Q)^T, independent of T, and M' = W, V' = W^-1,
// S' = (I + tau W / 2)^-1 are too.  So one table on [0, t_max] serves every
// point and every horizon; what changes with T is
//   * the node count nk and the last weight (per point),
//   * the dual step sigma = 1 / (tau |K_{<nk}|^2): the largest eigenvalue of
//     the prefix Gram matrix sum_{i < k} K_i^T K_i is taken every FX_SNAP
//     nodes (the table build stores those partial sums); a point uses the
//     value at the next multiple of FX_SNAP at or above nk, an upper bound of
//     its own |K|^2 since prefix Gram matrices grow in the Loewner order,
//   * the maps of the query point and of p: x' = e^{TA} x, p = e^{TA^T} q
//     and q0 = e^{-TA^T} p0.  With T = (nk - 1) dt + r, 0 < r <= dt,
//     e^{TA} = (e^{dt A})^{nk - 1} e^{rA}: the integer power is a product of
//     the binary powers e^{2^j dt A} (built once by repeated squaring), and
//     e^{rA} v is summed as its Taylor series on the vector (r |A| <= 1/2
//     per sub-step, 16 terms: truncation below 1e-17 relative).
#include "common.cuh"
#include "cta_linalg.cuh"

namespace hopf {

// largest eigenvalue of each stored prefix Gram matrix (one block each)
__global__ void fixed_lam_kernel(const double *__restrict__ snaps, int nsnap, int n, double *__restrict__ lam,
                                 double *__restrict__ scratch) {
    double *v = scratch + (long long)blockIdx.x * (2LL * n + 8);
    double *u = v + n, *red = u + n;
    for (int g = blockIdx.x; g < nsnap; g += gridDim.x) {
        const double L2 = cta::lambda_max(snaps + (long long)g * n * n, n, v, u, red);
        if (threadIdx.x == 0) lam[g] = L2;
        __syncthreads();
    }
}

// binary powers: block 0 writes e^{2^j dt A}, block 1 e^{-2^j dt A}, j < J
__global__ void fixed_powers_kernel(const double *__restrict__ A, int n, double dt, int J, double *__restrict__ Ep,
                                    double *__restrict__ Em, double *__restrict__ scratch) {
    const double sgn = blockIdx.x == 0 ? 1.0 : -1.0;
    double *E = blockIdx.x == 0 ? Ep : Em;
    double *X = scratch + (long long)blockIdx.x * (2LL * n * n + 8);
    double *T1 = X + (long long)n * n, *red = T1 + (long long)n * n;
    cta::expm(E, A, sgn * dt, n, X, T1, red);
    for (int j = 1; j < J; ++j)
        cta::matmul(E + (long long)j * n * n, E + (long long)(j - 1) * n * n, E + (long long)(j - 1) * n * n, n, n, n);
}

// per point: node count, last weight and dual step of its horizon; a horizon
// outside [0, t_max] (or not finite) gets nk = -1 and the outputs NaN /
// HOPF_NONFINITE.  T = 0 keeps one node of weight 0 (the iteration then
// solves min_p p^T W p / 4 + 1 - <x, p>, whose value is J_x(x)).
template <typename R>
__global__ void fixed_prep_kernel(int P, const double *__restrict__ Tv, int t_stride, double t_max, double dt,
                                  int N, double tau, double sigma_scale, const double *__restrict__ lam, int snap,
                                  const int *__restrict__ active, int *__restrict__ nk, double *__restrict__ wl,
                                  double *__restrict__ sig, int n, R *__restrict__ phi, R *__restrict__ pstar,
                                  R *__restrict__ gap, int *__restrict__ iters, int *__restrict__ status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P || (active && !active[k])) return;
    const double T = Tv[t_stride ? k : 0];
    if (!(T >= 0.0) || !(T <= t_max)) {
        nk[k] = -1;
        wl[k] = 0.0;
        sig[k] = 0.0;
        const R nan = R(__longlong_as_double(0x7ff8000000000000LL));
        if (phi) phi[k] = nan;
        if (gap) gap[k] = nan;
        if (iters) iters[k] = 0;
        if (status) status[k] = HOPF_NONFINITE;
        if (pstar)
            for (int j = 0; j < n; ++j) pstar[(long long)k * n + j] = nan;
        return;
    }
    int c = 1;
    double w = 0.0;
    if (T > 0.0) {
        c = (int)ceil(T / dt);
        c = c < 1 ? 1 : (c > N ? N : c);
        w = __dsub_rn(T, __dmul_rn((double)(c - 1), dt));     // T - (nk - 1) dt, rounded as written
    }
    nk[k] = c;
    wl[k] = w;
    const double L2 = lam[(c - 1) / snap];
    sig[k] = L2 > 0.0 ? sigma_scale / (tau * L2) : 0.0;
}

// out = e^{TA} v (mode 0), e^{T A^T} v (mode 1) or e^{-T A^T} v (mode 2)
// for every point at its own horizon; one block per point, threads over
// state components.  Points with nk < 0 are left alone.
template <typename R>
__global__ void fixed_map_kernel(int mode, int P, int n, const double *__restrict__ A, double anorm,
                                 const double *__restrict__ pw, int J, const int *__restrict__ nk,
                                 const double *__restrict__ wl, const R *__restrict__ in, R *__restrict__ out,
                                 const int *__restrict__ active) {
    extern __shared__ double fsm[];
    double *v = fsm, *t = v + n, *acc = t + n;
    const bool trans = mode != 0;
    const double sgn = mode == 2 ? -1.0 : 1.0;
    for (int k = blockIdx.x; k < P; k += gridDim.x) {
        if (active && !active[k]) continue;
        const int c = nk[k];
        if (c < 0) continue;              // out-of-range horizon: outputs set by fixed_prep
        for (int a = threadIdx.x; a < n; a += blockDim.x) v[a] = (double)in[(long long)k * n + a];
        __syncthreads();
        // (e^{+-dt A})^{nk - 1}: one product per set bit of the exponent
        const int e = c - 1;
        for (int j = 0; j < J; ++j) {
            if (!((e >> j) & 1)) continue;
            const double *M = pw + (long long)j * n * n;
            for (int a = threadIdx.x; a < n; a += blockDim.x) {
                double s = 0.0;
                if (trans)
                    for (int b = 0; b < n; ++b) s = fma(M[(long long)b * n + a], v[b], s);
                else
                    for (int b = 0; b < n; ++b) s = fma(M[(long long)a * n + b], v[b], s);
                t[a] = s;
            }
            __syncthreads();
            for (int a = threadIdx.x; a < n; a += blockDim.x) v[a] = t[a];
            __syncthreads();
        }
        // e^{+-r A} v, r = T - (nk - 1) dt, by its Taylor series in sub-steps
        // of size h with |h A| <= 1/2
        const double r = wl[k];
        const int steps = (r * anorm > 0.5) ? (int)ceil(r * anorm / 0.5) : 1;
        const double h = sgn * r / (double)steps;
        for (int st = 0; st < steps && r > 0.0; ++st) {
            for (int a = threadIdx.x; a < n; a += blockDim.x) {
                acc[a] = v[a];
                t[a] = v[a];
            }
            __syncthreads();
            for (int q = 1; q <= 16; ++q) {
                // t <- (h A) t / q  (A^T for the maps of p); every thread keeps
                // its (at most two) new components until all have read t
                double nv[2] = {0.0, 0.0};
                for (int a = threadIdx.x, c2 = 0; a < n; a += blockDim.x, ++c2) {
                    double s = 0.0;
                    if (trans)
                        for (int b = 0; b < n; ++b) s = fma(A[(long long)b * n + a], t[b], s);
                    else
                        for (int b = 0; b < n; ++b) s = fma(A[(long long)a * n + b], t[b], s);
                    nv[c2] = s * h / (double)q;
                }
                __syncthreads();
                for (int a = threadIdx.x, c2 = 0; a < n; a += blockDim.x, ++c2) {
                    t[a] = nv[c2];
                    acc[a] += nv[c2];
                }
                __syncthreads();
            }
            for (int a = threadIdx.x; a < n; a += blockDim.x) v[a] = acc[a];
            __syncthreads();
        }
        for (int a = threadIdx.x; a < n; a += blockDim.x) out[(long long)k * n + a] = (R)v[a];
        __syncthreads();
    }
}

// ------------------------------------------------------------ host side
int fixed_powers_count(int N) {
    int J = 1;
    while ((1LL << J) <= (long long)(N - 1)) ++J;
    return J;
}

cudaError_t launch_fixed_lam(const double *snaps, int nsnap, int n, double *lam, double *scratch, cudaStream_t s) {
    fixed_lam_kernel<<<nsnap, 256, 0, s>>>(snaps, nsnap, n, lam, scratch);
    return cudaGetLastError();
}

cudaError_t launch_fixed_powers(const double *A, int n, double dt, int J, double *Ep, double *Em, double *scratch,
                                cudaStream_t s) {
    fixed_powers_kernel<<<2, 256, 0, s>>>(A, n, dt, J, Ep, Em, scratch);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fixed_prep(int P, const double *Tv, int t_stride, double t_max, double dt, int N, double tau,
                              double sigma_scale, const double *lam, int snap, const int *active, int *nk,
                              double *wl, double *sig, int n, R *phi, R *pstar, R *gap, int *iters, int *status,
                              cudaStream_t s) {
    fixed_prep_kernel<R><<<(P + 255) / 256, 256, 0, s>>>(P, Tv, t_stride, t_max, dt, N, tau, sigma_scale, lam, snap,
                                                        active, nk, wl, sig, n, phi, pstar, gap, iters, status);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fixed_map(int mode, int P, int n, const double *A, double anorm, const double *pw, int J,
                             const int *nk, const double *wl, const R *in, R *out, const int *active, int sms,
                             cudaStream_t s) {
    if (n > 512) return cudaErrorInvalidValue;     // two components per thread at most
    const int grid = P < 8 * sms ? P : 8 * sms;
    const size_t smem = sizeof(double) * 3 * (size_t)n;
    fixed_map_kernel<R><<<grid > 0 ? grid : 1, 256, smem, s>>>(mode, P, n, A, anorm, pw, J, nk, wl, in, out, active);
    return cudaGetLastError();
}

template cudaError_t launch_fixed_prep<float>(int, const double *, int, double, double, int, double, double,
                                              const double *, int, const int *, int *, double *, double *, int,
                                              float *, float *, float *, int *, int *, cudaStream_t);
template cudaError_t launch_fixed_prep<double>(int, const double *, int, double, double, int, double, double,
                                               const double *, int, const int *, int *, double *, double *, int,
                                               double *, double *, double *, int *, int *, cudaStream_t);
template cudaError_t launch_fixed_map<float>(int, int, int, const double *, double, const double *, int,
                                             const int *, const double *, const float *, float *, const int *, int,
                                             cudaStream_t);
template cudaError_t launch_fixed_map<double>(int, int, int, const double *, double, const double *, int,
                                              const int *, const double *, const double *, double *, const int *,
                                              int, cudaStream_t);

}  // namespace hopf
