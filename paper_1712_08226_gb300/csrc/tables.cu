// Node tables of the discretised generalized Hopf formula, built on the
// device in float64 (one thread block per horizon T).
//
// For horizon T and N nodes the quadrature of §III.A gives node times t_i and
// weights w_i (left Riemann, Eq. 17: t_i = i T/N, w_i = T/N; trapezoid:
// t_i = i T/(N-1), end weights halved).  The node matrices of Eq. 20,
//   K_i = (-e^{-s_i A} B Q)^T,   s_i = T - t_i,
// are generated without one exponential per node: with h the node spacing,
// s_i = k h for an integer k, so e^{-s_i A} B Q = (e^{-hA})^k B Q is obtained
// by repeated multiplication with E_h = e^{-hA} (the paper evaluates the same
// products with the Al-Mohy-Higham action of the exponential; §III.A and §VI).
// The same pass accumulates the Gram matrix sum_i K_i^T K_i, whose largest
// eigenvalue is |K|^2 for the dual step sigma = 1/(tau |K|^2) of §VI.
// The quadratic target of §VI.A needs M = V(0)^-1 = e^{-TA} W e^{-TA^T}
// (Eq. 35), V = M^-1 and the prox matrix S = (I + tau M/2)^-1 (Eq. 37).
//
// Terminal-time variables (terminal != 0): with p = e^{T A^T} q every term of
// Eq. 18 keeps its form with K'_i = K_i e^{T A^T} = (-e^{t_i A} B Q)^T,
// M' = W, V' = W^-1, S' = (I + tau W/2)^-1 and the query point mapped to
// e^{TA} z0.  K'_i is generated the same way, by repeated multiplication
// with e^{hA} from t_0 = 0.  E = e^{TA} and Ei = e^{-TA} are stored for the
// maps of the query point and of p (identity in the paper's variable).
#include "common.cuh"
#include "cta_linalg.cuh"

namespace hopf {

__global__ void build_instances_kernel(const double *__restrict__ A, const double *__restrict__ B,
                                       const double *__restrict__ qd, const double *__restrict__ W,
                                       const double *__restrict__ Tv, const int *__restrict__ active,
                                       int n_inst, int n, int m, int N, int rule, double tau,
                                       double sigma_scale, double *out64, float *out32,
                                       double *scratch, bool smem_scratch, int w_count, int need_eig,
                                       int terminal, double *gram_snap, int snap) {
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    // scratch in shared memory when the launch provides it (small n), else global
    extern __shared__ double tsm[];
    double *sc = smem_scratch ? tsm : scratch + (long long)blockIdx.x * table_scratch_doubles(n, m);
    double *X = sc, *T1 = X + n * n, *Eh = T1 + n * n, *ET = Eh + n * n, *T2 = ET + n * n;
    double *C = T2 + n * n, *Aug = C + n * n;             // Aug: 2 n^2
    double *Ga = Aug + 2 * n * n, *Gb = Ga + n * m;
    double *v = Gb + n * m, *u = v + n;
    double *red = u + n;                                  // 8 doubles
    double *rot = red + 8;                                // 3n + 8 doubles (Jacobi rotations)
    int *piv = (int *)(rot + 3 * n + 8);

    for (int inst = blockIdx.x; inst < n_inst; inst += gridDim.x) {
        if (active && !active[inst]) continue;
        const double T = Tv[inst];
        double *o = out64 + (long long)inst * L.stride;
        const bool ends = rule == HOPF_TRAPEZOID || rule == HOPF_SIMPSON;   // samples include t = T
        const double h = ends ? T / (double)(N - 1) : T / (double)N;

        cta::expm(Eh, A, terminal ? h : -h, n, X, T1, red);
        // G = B Q, Gram accumulator C = 0
        for (int e = threadIdx.x; e < n * m; e += blockDim.x) Ga[e] = B[e] * qd[e % m];
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) C[e] = 0.0;
        __syncthreads();
        double *cur = Ga, *nxt = Gb;
        for (int idx = 0; idx < N; ++idx) {
            if (terminal ? idx > 0 : (!ends || idx > 0)) {
                cta::matmul(nxt, Eh, cur, n, n, m);     // advance s (or t) by h
                double *t = cur; cur = nxt; nxt = t;
            }
            // paper's variable: node with s_i = (idx + [left]) h; terminal
            // variables: node idx at t = idx h
            const int i = terminal ? idx : N - 1 - idx;
            double *Ki = o + L.K + (long long)i * m * n;
            for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
                int c = e / n, j = e % n;
                Ki[e] = -cur[j * m + c];
            }
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
                int a = e / n, b = e % n;
                double s = 0.0;
                for (int c = 0; c < m; ++c) s = fma(cur[a * m + c], cur[b * m + c], s);
                C[e] += s;
            }
            __syncthreads();
            // fixed-step rule (terminal variables, nodes in time order): the
            // prefix Gram sum of the first idx + 1 nodes every snap nodes
            if (gram_snap && terminal && ((idx + 1) % snap == 0 || idx == N - 1))
                cta::copy(gram_snap + (long long)(idx / snap) * n * n, C, n * n);
        }
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            double wi = h;
            if (rule == HOPF_TRAPEZOID && (i == 0 || i == N - 1)) wi = 0.5 * h;
            if (rule == HOPF_SIMPSON) wi = (i == 0 || i == N - 1) ? h / 3.0 : ((i & 1) ? 4.0 * h / 3.0 : 2.0 * h / 3.0);
            o[L.w + i] = wi;
        }
        // M = e^{-TA} W e^{-TA}^T (symmetrised; W itself in terminal-time
        // variables), V = M^-1, S = (I + tau M / 2)^-1
        cta::expm(ET, A, -T, n, X, T1, red);
        const double *Wk = W + (long long)(inst % w_count) * n * n;
        if (terminal) {
            cta::copy(o + L.Ei, ET, n * n);
            cta::copy(T1, Wk, n * n);
        } else {
            cta::matmul(T2, ET, Wk, n, n, n);
            cta::matmul_bt(T1, T2, ET, n, n, n);
        }
        double *Mo = o + L.M, *Vo = o + L.V, *So = o + L.S;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            int a = e / n, b = e % n;
            Mo[e] = 0.5 * (T1[a * n + b] + T1[b * n + a]);
        }
        __syncthreads();
        bool okV = cta::invert(T2, Mo, n, Aug, piv, red);
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            int a = e / n, b = e % n;
            Vo[e] = okV ? 0.5 * (T2[a * n + b] + T2[b * n + a]) : __longlong_as_double(0x7ff8000000000000LL);
        }
        for (int e = threadIdx.x; e < n * n; e += blockDim.x)
            X[e] = ((e / n == e % n) ? 1.0 : 0.0) + 0.5 * tau * Mo[e];
        __syncthreads();
        bool okS = cta::invert(T2, X, n, Aug, piv, red);
        for (int e = threadIdx.x; e < n * n; e += blockDim.x)
            So[e] = okS ? T2[e] : __longlong_as_double(0x7ff8000000000000LL);
        __syncthreads();
        // maps of the query point and of p: e^{TA}, e^{-TA} (identity in the
        // paper's variable)
        if (terminal) {
            cta::expm(T2, A, T, n, X, T1, red);
            cta::copy(o + L.E, T2, n * n);
        } else {
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
                const double id = (e / n == e % n) ? 1.0 : 0.0;
                o[L.E + e] = id;
                o[L.Ei + e] = id;
            }
        }
        __syncthreads();
        cta::copy(o + L.G, C, n * n);
        // |K|^2 = largest eigenvalue of the Gram matrix: Jacobi for small n
        // (a few hundred block barriers), the power method otherwise
        double L2;
        if (n <= 64) {
            cta::copy(X, C, n * n);
            cta::sym_eig(X, T1, v, n, red, rot);
            if (threadIdx.x == 0) {
                double mx = v[0];
                for (int i = 1; i < n; ++i) mx = fmax(mx, v[i]);
                red[6] = mx;
            }
            __syncthreads();
            L2 = red[6];
            __syncthreads();
        } else {
            L2 = cta::lambda_max(C, n, v, u, red);
        }
        // M = U diag(lam) U^T for the accelerated prox (I + tau M/2)^-1 =
        // U diag(1/(1 + tau lam/2)) U^T; only the accelerated iteration uses it
        if (need_eig) {
            cta::copy(T2, Mo, n * n);
            cta::sym_eig(T2, T1, v, n, red, rot);
            cta::copy(o + L.U, T1, n * n);
            cta::copy(o + L.lam, v, n);
        } else {
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) o[L.U + e] = 0.0;
            for (int e = threadIdx.x; e < n; e += blockDim.x) o[L.lam + e] = 0.0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double lmin = o[L.lam];
            for (int i = 1; i < n; ++i) lmin = fmin(lmin, o[L.lam + i]);
            double *s = o + L.sc;
            s[SC_SIGMA] = (L2 > 0.0) ? sigma_scale / (tau * L2) : 0.0;
            s[SC_T] = T;
            s[SC_L2] = L2;
            s[SC_ZERO] = (T == 0.0) ? 1.0 : 0.0;
            s[SC_GAMMA] = fmax(0.5 * lmin, 0.0);
        }
        __syncthreads();
        if (out32) {
            float *f = out32 + (long long)inst * L.stride;
            for (long long e = threadIdx.x; e < L.stride; e += blockDim.x) f[e] = (float)o[e];
        }
        __syncthreads();
    }
}

__global__ void to_double_kernel(const float *src, double *dst, int count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = (double)src[i];
}

__global__ void copy_double_kernel(const double *src, double *dst, int count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = src[i];
}

cudaError_t launch_build_instances(int grid, int threads, cudaStream_t s, const double *A, const double *B,
                                   const double *qd, const double *W, const double *Tv, const int *active,
                                   int n_inst, int n, int m, int N, int rule, double tau, double sigma_scale,
                                   double *out64, float *out32, double *scratch) {
    const size_t bytes = sizeof(double) * (size_t)table_scratch_doubles(n, m);
    const bool in_smem = bytes <= 48 * 1024;
    build_instances_kernel<<<grid, threads, in_smem ? bytes : 0, s>>>(A, B, qd, W, Tv, active, n_inst, n, m, N, rule,
                                                                      tau, sigma_scale, out64, out32, scratch, in_smem, 1,
                                                                      1, 0, nullptr, 0);
    return cudaGetLastError();
}

// as launch_build_instances, with the eigen-decomposition of M (used only by
// the accelerated iteration) optional, the choice of variables and, for the
// fixed-step rule, the prefix Gram sums every snap nodes (gram_snap, null: off)
cudaError_t launch_build_instances_opt(int grid, int threads, cudaStream_t s, const double *A, const double *B,
                                       const double *qd, const double *W, const double *Tv, const int *active,
                                       int n_inst, int n, int m, int N, int rule, double tau, double sigma_scale,
                                       double *out64, float *out32, double *scratch, int need_eig, int terminal,
                                       double *gram_snap, int snap) {
    const size_t bytes = sizeof(double) * (size_t)table_scratch_doubles(n, m);
    const bool in_smem = bytes <= 48 * 1024;
    build_instances_kernel<<<grid, threads, in_smem ? bytes : 0, s>>>(A, B, qd, W, Tv, active, n_inst, n, m, N, rule,
                                                                      tau, sigma_scale, out64, out32, scratch, in_smem, 1,
                                                                      need_eig, terminal, gram_snap, snap);
    return cudaGetLastError();
}

// instance k uses the target weight block W + (k % w_count) n^2 (stacked copies)
cudaError_t launch_build_instances_wblocks(int grid, int threads, cudaStream_t s, const double *A, const double *B,
                                           const double *qd, const double *W, int w_count, const double *Tv,
                                           int n_inst, int n, int m, int N, int rule, double tau,
                                           double sigma_scale, double *out64, float *out32, double *scratch) {
    const size_t bytes = sizeof(double) * (size_t)table_scratch_doubles(n, m);
    const bool in_smem = bytes <= 48 * 1024;
    build_instances_kernel<<<grid, threads, in_smem ? bytes : 0, s>>>(A, B, qd, W, Tv, nullptr, n_inst, n, m, N,
                                                                      rule, tau, sigma_scale, out64, out32, scratch,
                                                                      in_smem, w_count, 0, 0, nullptr, 0);
    return cudaGetLastError();
}

cudaError_t launch_horizons(int count, cudaStream_t s, const void *t, bool t_is_float, double *Tv) {
    if (t_is_float) to_double_kernel<<<(count + 255) / 256, 256, 0, s>>>((const float *)t, Tv, count);
    else copy_double_kernel<<<(count + 255) / 256, 256, 0, s>>>((const double *)t, Tv, count);
    return cudaGetLastError();
}

}  // namespace hopf
