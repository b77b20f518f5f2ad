// Small dense float64 linear algebra executed cooperatively by one thread
// block (all threads call every routine; routines end with __syncthreads()).
// Matrices are row-major in global or shared memory.  Used to build the node
// tables and the trajectory propagators on the device.
#pragma once
#include <cuda_runtime.h>

namespace hopf {
namespace cta {

// C[r x c] = A[r x k] * B[k x c]   (C must not alias A or B)
__device__ inline void matmul(double *C, const double *A, const double *B, int r, int k, int c) {
    for (int e = threadIdx.x; e < r * c; e += blockDim.x) {
        int i = e / c, j = e % c;
        double s = 0.0;
        for (int l = 0; l < k; ++l) s = fma(A[i * k + l], B[l * c + j], s);
        C[e] = s;
    }
    __syncthreads();
}

// C[r x c] = A[r x k] * B[c x k]^T
__device__ inline void matmul_bt(double *C, const double *A, const double *B, int r, int k, int c) {
    for (int e = threadIdx.x; e < r * c; e += blockDim.x) {
        int i = e / c, j = e % c;
        double s = 0.0;
        for (int l = 0; l < k; ++l) s = fma(A[i * k + l], B[j * k + l], s);
        C[e] = s;
    }
    __syncthreads();
}

__device__ inline void copy(double *D, const double *S, int len) {
    for (int e = threadIdx.x; e < len; e += blockDim.x) D[e] = S[e];
    __syncthreads();
}

__device__ inline void set_identity(double *D, int n, double diag = 1.0) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) D[e] = (e / n == e % n) ? diag : 0.0;
    __syncthreads();
}

// Maximum absolute column sum (matrix 1-norm), result broadcast through *red.
__device__ inline double norm1(const double *X, int n, double *red) {
    if (threadIdx.x == 0) *red = 0.0;
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += fabs(X[i * n + j]);
        // non-negative doubles order like their bit patterns
        atomicMax((unsigned long long *)red, (unsigned long long)__double_as_longlong(s));
    }
    __syncthreads();
    double v = *red;
    __syncthreads();
    return v;
}

// E = exp(alpha * A) by scaling and squaring with a truncated Taylor series
// (Moler and Van Loan, "Nineteen dubious ways to compute the exponential of a
// matrix", 1978/2003): X = alpha A / 2^s with |X|_1 <= 1/4, degree-18 Taylor
// polynomial by Horner's rule (truncation below 1e-24 relative), then s
// squarings.  Scratch: X, T1 (n x n each).  E must not alias the scratch.
__device__ inline void expm(double *E, const double *A, double alpha, int n, double *X, double *T1,
                            double *red) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) X[e] = alpha * A[e];
    __syncthreads();
    double nrm = norm1(X, n, red);
    int s = 0;
    while (nrm > 0.25 && s < 1000) { nrm *= 0.5; ++s; }
    double scale = ldexp(1.0, -s);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) X[e] *= scale;
    set_identity(E, n);
    const int degree = 18;
    for (int k = degree; k >= 1; --k) {
        matmul(T1, X, E, n, n, n);              // T1 = X E
        double inv = 1.0 / (double)k;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x)
            E[e] = ((e / n == e % n) ? 1.0 : 0.0) + T1[e] * inv;
        __syncthreads();
    }
    for (int q = 0; q < s; ++q) {
        matmul(T1, E, E, n, n, n);
        copy(E, T1, n * n);
    }
}

// In-place inverse of an n x n matrix by Gauss-Jordan elimination with
// partial pivoting on the augmented block [A | I] (Aug: n x 2n scratch).
// Returns false (to every thread) if a pivot vanishes.
__device__ inline bool invert(double *Ainv, const double *A, int n, double *Aug, int *piv_row,
                              double *red) {
    const int w2 = 2 * n;
    for (int e = threadIdx.x; e < n * w2; e += blockDim.x) {
        int i = e / w2, j = e % w2;
        Aug[e] = (j < n) ? A[i * n + j] : ((j - n == i) ? 1.0 : 0.0);
    }
    __syncthreads();
    bool ok = true;
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            int best = k;
            double bv = fabs(Aug[k * w2 + k]);
            for (int i = k + 1; i < n; ++i) {
                double v = fabs(Aug[i * w2 + k]);
                if (v > bv) { bv = v; best = i; }
            }
            *piv_row = best;
            *red = bv;
        }
        __syncthreads();
        int pr = *piv_row;
        if (!(*red > 0.0)) { ok = false; }
        __syncthreads();
        if (!ok) break;
        if (pr != k) {
            for (int j = threadIdx.x; j < w2; j += blockDim.x) {
                double t = Aug[k * w2 + j];
                Aug[k * w2 + j] = Aug[pr * w2 + j];
                Aug[pr * w2 + j] = t;
            }
            __syncthreads();
        }
        double pinv = 1.0 / Aug[k * w2 + k];
        __syncthreads();
        for (int j = threadIdx.x; j < w2; j += blockDim.x) Aug[k * w2 + j] *= pinv;
        __syncthreads();
        for (int e = threadIdx.x; e < n * w2; e += blockDim.x) {
            int i = e / w2, j = e % w2;
            if (i != k) {
                double f = Aug[i * w2 + k];
                if (j != k) Aug[e] = fma(-f, Aug[k * w2 + j], Aug[e]);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            if (i != k) Aug[i * w2 + k] = 0.0;
        __syncthreads();
    }
    if (ok) {
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) Ainv[e] = Aug[(e / n) * w2 + n + e % n];
    }
    __syncthreads();
    return ok;
}

// Largest eigenvalue of a symmetric positive semi-definite matrix C by the
// power method with Rayleigh quotients (v, u: n scratch).
__device__ inline double lambda_max(const double *C, int n, double *v, double *u, double *red,
                                    int max_iter = 4000) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) v[j] = 1.0 + 0.37 * (double)j / (double)n;
    __syncthreads();
    double lam_prev = 0.0, lam = 0.0;
    for (int it = 0; it < max_iter; ++it) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double s = 0.0;
            for (int l = 0; l < n; ++l) s = fma(C[i * n + l], v[l], s);
            u[i] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double vu = 0.0, vv = 0.0, uu = 0.0;
            for (int i = 0; i < n; ++i) { vu += v[i] * u[i]; vv += v[i] * v[i]; uu += u[i] * u[i]; }
            red[0] = (vv > 0.0) ? vu / vv : 0.0;
            red[1] = (uu > 0.0) ? rsqrt(uu) : 0.0;
        }
        __syncthreads();
        lam = red[0];
        double sc = red[1];
        for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = u[i] * sc;
        __syncthreads();
        if (sc == 0.0) break;
        if (it > 8 && fabs(lam - lam_prev) <= 1e-15 * fabs(lam)) break;
        lam_prev = lam;
    }
    return lam;
}

// Eigen-decomposition of a symmetric matrix by Jacobi rotations (Jacobi
// 1846) in the parallel round-robin order of Brent and Luk (1985): each round
// pairs the indices into disjoint planes (p, q) (circle method), every pair's
// rotation is computed from the same matrix, then all column rotations and
// all row rotations are applied at once (disjoint planes commute).  The
// rotation of plane (p, q) annihilates a_pq: theta = (a_qq - a_pp)/(2 a_pq),
// t = sgn(theta)/(|theta| + sqrt(theta^2 + 1)), c = 1/sqrt(t^2 + 1), s = t c,
// and the 2 x 2 block becomes diag(a_pp - t a_pq, a_qq + t a_pq).
// A (n x n, destroyed) becomes diagonal; U collects the rotations so that
// A_in = U diag(lam) U^T.  rot: scratch of 6 * ceil(n/2) + 2 doubles.
__device__ inline void sym_eig(double *A, double *U, double *lam, int n, double *red, double *rot) {
    set_identity(U, n);
    const int ne = n + (n & 1), half = ne / 2;
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (threadIdx.x == 0) { red[0] = 0.0; red[1] = 0.0; }
        __syncthreads();
        double off = 0.0, tot = 0.0;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            double v = A[e] * A[e];
            tot += v;
            if (e / n != e % n) off += v;
        }
        atomicAdd(&red[0], off);
        atomicAdd(&red[1], tot);
        __syncthreads();
        const bool done = !(red[0] > 1e-30 * red[1]);
        __syncthreads();
        if (done) break;
        for (int r = 0; r < ne - 1; ++r) {
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                int a = k == 0 ? r : (r + k) % (ne - 1);
                int b = k == 0 ? ne - 1 : (r - k + (ne - 1)) % (ne - 1);
                int p = a < b ? a : b, q = a < b ? b : a;
                double *R = rot + 6 * k;
                R[0] = 1.0; R[1] = 0.0; R[2] = 0.0; R[3] = 0.0;
                if (q < n) {
                    const double apq = A[p * n + q];
                    R[4] = A[p * n + p];
                    R[5] = A[q * n + q];
                    if (apq != 0.0) {
                        double th = (R[5] - R[4]) / (2.0 * apq);
                        double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        double c = 1.0 / sqrt(t * t + 1.0);
                        R[0] = c; R[1] = t * c; R[2] = t; R[3] = apq;
                    }
                }
            }
            __syncthreads();
            // column rotations (A and U), then row rotations, then the 2 x 2 blocks
            for (int e = threadIdx.x; e < half * n; e += blockDim.x) {
                int k = e / n, i = e % n;
                int a = k == 0 ? r : (r + k) % (ne - 1);
                int b = k == 0 ? ne - 1 : (r - k + (ne - 1)) % (ne - 1);
                int p = a < b ? a : b, q = a < b ? b : a;
                const double *R = rot + 6 * k;
                if (q >= n || R[3] == 0.0) continue;
                double c = R[0], sn = R[1];
                double ap = A[i * n + p], aq = A[i * n + q];
                A[i * n + p] = c * ap - sn * aq;
                A[i * n + q] = sn * ap + c * aq;
                double up = U[i * n + p], uq = U[i * n + q];
                U[i * n + p] = c * up - sn * uq;
                U[i * n + q] = sn * up + c * uq;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < half * n; e += blockDim.x) {
                int k = e / n, j = e % n;
                int a = k == 0 ? r : (r + k) % (ne - 1);
                int b = k == 0 ? ne - 1 : (r - k + (ne - 1)) % (ne - 1);
                int p = a < b ? a : b, q = a < b ? b : a;
                const double *R = rot + 6 * k;
                if (q >= n || R[3] == 0.0) continue;
                double c = R[0], sn = R[1];
                double ap = A[p * n + j], aq = A[q * n + j];
                A[p * n + j] = c * ap - sn * aq;
                A[q * n + j] = sn * ap + c * aq;
            }
            __syncthreads();
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                int a = k == 0 ? r : (r + k) % (ne - 1);
                int b = k == 0 ? ne - 1 : (r - k + (ne - 1)) % (ne - 1);
                int p = a < b ? a : b, q = a < b ? b : a;
                const double *R = rot + 6 * k;
                if (q >= n || R[3] == 0.0) continue;
                A[p * n + p] = R[4] - R[2] * R[3];
                A[q * n + q] = R[5] + R[2] * R[3];
                A[p * n + q] = 0.0;
                A[q * n + p] = 0.0;
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = A[i * n + i];
    __syncthreads();
}

}  // namespace cta
}  // namespace hopf
