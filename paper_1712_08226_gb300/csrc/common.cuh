// Shared device-side definitions of the generalized-Hopf GB300 library.
//
// Data layout of one "instance" (the node table and prox matrices of one
// system at one horizon T; built in float64 by tables.cu):
//   K    [N][m][n]  K_i = (-e^{-(T - t_i) A} B Q)^T            (Eq. 20)
//   w    [N]        quadrature weights (§III.A, Eq. 17 / trapezoid)
//   M    [n][n]     V(0)^-1 = e^{-TA} W e^{-TA^T}               (§VI.A, Eq. 35)
//   V    [n][n]     M^-1
//   S    [n][n]     (I + tau M / 2)^-1                          (Eq. 37)
//   U    [n][n]     eigenvectors of M (M = U diag(lam) U^T), for the
//   lam  [n]        accelerated iteration whose step tau changes every step
//   G    [n][n]     Gram matrix sum_i K_i^T K_i (|K|^2 is its largest
//                   eigenvalue; |K d|^2 = d^T G d for the adaptive steps)
//   E    [n][n]     e^{TA}: maps the query point to the terminal-time variable
//   Ei   [n][n]     e^{-TA}  (both the identity for the paper's variable)
//   sc   [8]        sigma, T, |K|^2, flag (1 = T == 0), gamma = lambda_min(M)/2
// In terminal-time variables (p = e^{T A^T} q) the same slots hold
// K'_i = (-e^{t_i A} B Q)^T, M' = W, V' = W^-1, S' = (I + tau W/2)^-1.
// A float32 copy with the same layout is made for the float32 kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hopf.h"

namespace hopf {

struct InstanceLayout {
    // element offsets (in elements of the instance's type) inside one instance
    long long K, w, M, V, S, U, lam, G, E, Ei, sc, stride;
    __host__ __device__ static InstanceLayout make(int n, int m, int N) {
        InstanceLayout L;
        long long o = 0;
        auto al = [](long long v) { return (v + 3) & ~3LL; };  // 32-byte alignment for doubles
        L.K = o;  o = al(o + (long long)N * m * n);
        L.w = o;  o = al(o + N);
        L.M = o;  o = al(o + (long long)n * n);
        L.V = o;  o = al(o + (long long)n * n);
        L.S = o;  o = al(o + (long long)n * n);
        L.U = o;  o = al(o + (long long)n * n);
        L.lam = o; o = al(o + n);
        L.G = o;  o = al(o + (long long)n * n);
        L.E = o;  o = al(o + (long long)n * n);
        L.Ei = o; o = al(o + (long long)n * n);
        L.sc = o; o = al(o + 8);
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
    int accel;         // Chambolle-Pock accelerated variant (strongly convex G)
    int adaptive;      // residual-balanced step sizes (general kernel)
    const int *list;        // optional: solve only the points list[0 .. *list_count)
    const int *list_count;  // device count for `list`
    // multi-phase solve of the small-state kernels: a phase parks every point
    // still uncertified after carry_cap iterations (carry_cap > 0) into the
    // out_* buffers; a later phase (carry_in = 1) resumes the in_* points
    int carry_cap;
    int carry_in;
    float *in_y, *out_y;      // [slot][N m] parked dual variables
    float *in_st, *out_st;    // [slot][CARRY_W] p, pbar, tau, sigma, iteration count
    int *in_list, *out_list;  // point index of each slot
    int *in_count, *out_count;
    // fixed-step rule: per point node count (-1: horizon out of range, point
    // skipped), last node weight and dual step; null for the other rules
    const int *fx_nk;
    const double *fx_wl, *fx_sig;
    double tau, tol_gap, sign_floor;
};

// fixed-step rule: prefix Gram sums (and their largest eigenvalues) every
// FX_SNAP nodes
constexpr int FX_SNAP = 64;

// float64 scratch (elements) one thread block needs to build one instance
__host__ __device__ inline long long table_scratch_doubles(int n, int m) {
    return 9LL * n * n + 2LL * n * m + 8LL * n + 32;
}

constexpr int CARRY_W = 40;   // p [16], pbar [16], tau, sigma, iteration count, pad

enum { SC_SIGMA = 0, SC_T = 1, SC_L2 = 2, SC_ZERO = 3, SC_GAMMA = 4 };

// unit roundoff of the iteration's arithmetic
template <typename R> struct Unit;
template <> struct Unit<float> { static constexpr double u = 5.9604644775390625e-08; };
template <> struct Unit<double> { static constexpr double u = 1.1102230246251565e-16; };

// Float rounding allowance added to the computed relative gap before it is
// compared with the tolerance: 4 u times the magnitude of the terms of P and D.
template <typename R>
__device__ __forceinline__ R gap_allowance(R quad, R H, R Dv, R scale) {
    return R(4.0 * Unit<R>::u) * (fabs(quad) + H + fabs(Dv) + R(1)) / scale;
}

// Relative duality gap (P - D) / max(1, |P|, |D|).
template <typename R>
__device__ __forceinline__ R rel_gap(R Pv, R Dv) {
    R s = fmax(R(1), fmax(fabs(Pv), fabs(Dv)));
    return (Pv - Dv) / s;
}

}  // namespace hopf

namespace hopf {

// Geometry of the tiled large-state kernel (pdhg_tile.cu).  The control
// dimension is padded to mp (exact: the extra rows of K are zero), each of the
// 8 warps of a block owns npt consecutive nodes (rw = npt mp rows of K) of a
// node block of nc = 8 npt nodes (cr rows), and the state dimension is padded
// to n4 (a multiple of 4, zero columns) so rows can be read as float4.
constexpr int TILE_WARPS = 8;
struct TileGeom {
    int mp, n4, nq, npt, rw, nc, cr, chunks, pt;
};
__host__ __device__ inline int tile_mpad(int m) {
    return m <= 6 ? m : (m <= 8 ? 8 : (m <= 10 ? 10 : (m <= 12 ? 12 : 16)));
}
__host__ __device__ inline TileGeom tile_geom(int n, int m, int N, int ppt) {
    TileGeom g;
    g.mp = tile_mpad(m);
    g.n4 = (n + 3) & ~3;
    g.nq = g.n4 / 4;
    g.npt = g.mp >= 8 ? 1 : 8 / g.mp;
    g.rw = g.npt * g.mp;
    g.nc = TILE_WARPS * g.npt;
    g.cr = TILE_WARPS * g.rw;
    g.chunks = (N + g.nc - 1) / g.nc;
    g.pt = 32 * ppt;
    return g;
}
// dynamic shared memory of one block, in floats: K block (also the u buffer
// of the certificate), a second K block when double-buffered, pbar tile,
// dual block, vector buffer, 3 per-slot sums
__host__ __device__ inline long long tile_smem_floats(const TileGeom &g, bool dbuf) {
    const int kr = g.cr > g.pt ? g.cr : g.pt;
    return (long long)kr * g.n4 + (dbuf ? (long long)g.cr * g.n4 : 0LL) + 2LL * g.n4 * g.pt +
           (long long)g.cr * g.pt + 3LL * g.pt;
}

}  // namespace hopf
