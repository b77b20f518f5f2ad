// Shared device-side definitions of the generalized-Hopf GB300 library.
//
// Data layout of one "instance" (the node table and prox matrices of one
// system at one horizon T; built in float64 by tables.cu):
//   K    [N][m][n]  K_i = (-e^{-(T - t_i) A} B Q)^T            (Eq. 20)
//   w    [N]        quadrature weights (§III.A, Eq. 17 / trapezoid)
//   M    [n][n]     V(0)^-1 = e^{-TA} W e^{-TA^T}               (§VI.A, Eq. 35)
//   V    [n][n]     M^-1
//   S    [n][n]     (I + tau M / 2)^-1                          (Eq. 37)
//   sc   [4]        sigma, T, |K|^2, flag (1 = T == 0)
// A float32 copy with the same layout is made for the float32 kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hopf.h"

namespace hopf {

struct InstanceLayout {
    // element offsets (in elements of the instance's type) inside one instance
    long long K, w, M, V, S, sc, stride;
    __host__ __device__ static InstanceLayout make(int n, int m, int N) {
        InstanceLayout L;
        long long o = 0;
        auto al = [](long long v) { return (v + 3) & ~3LL; };  // 32-byte alignment for doubles
        L.K = o;  o = al(o + (long long)N * m * n);
        L.w = o;  o = al(o + N);
        L.M = o;  o = al(o + (long long)n * n);
        L.V = o;  o = al(o + (long long)n * n);
        L.S = o;  o = al(o + (long long)n * n);
        L.sc = o; o = al(o + 4);
        L.stride = o;
        return L;
    }
};

// Per-call parameters handed to the kernels (by value).
struct SolveParams {
    int n, m, N, P;
    int ctrl_kind;
    int max_iter, gap_every;
    int warm;          // p_init given
    int sign_mode;     // time-to-reach: stop once the sign of phi is certified
    int inst_stride;   // 0: one shared instance, 1: instance k for point k
    double tau, tol_gap, sign_floor;
};

// float64 scratch (elements) one thread block needs to build one instance
__host__ __device__ inline long long table_scratch_doubles(int n, int m) {
    return 9LL * n * n + 2LL * n * m + 2LL * n + 16;
}

enum { SC_SIGMA = 0, SC_T = 1, SC_L2 = 2, SC_ZERO = 3 };

// Relative duality gap (P - D) / max(1, |P|, |D|).
template <typename R>
__device__ __forceinline__ R rel_gap(R Pv, R Dv) {
    R s = fmax(R(1), fmax(fabs(Pv), fabs(Dv)));
    return (Pv - Dv) / s;
}

}  // namespace hopf
