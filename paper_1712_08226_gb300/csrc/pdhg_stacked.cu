// Chambolle-Pock iteration for k copies of one base system that share a
// single control (§VI.B unscented control, §VI.C dimensional scaling):
// state (chi_1, ..., chi_k), A~ = blockdiag(A, ..., A), B~ = (B; ...; B),
// target W = blockdiag(W_1, ..., W_k).
//
// The structure factorises every product of the iteration.  With
// e^{-s A~} = blockdiag(e^{-s A}), the node matrix of Eq. 20 of the stacked
// system is K~_i = (K_i, ..., K_i) with K_i the base node matrix, so
//   K~_i p = K_i (p_1 + ... + p_k),     K~^T y = (K^T y, ..., K^T y),
// |K~|^2 = k |K|^2, and M~ = e^{-T A~} W e^{-T A~}^T, V~ = M~^-1 and
// S~ = (I + tau M~/2)^-1 are block diagonal with the blocks of the base
// system for W_j.  One iteration of a point costs 4 N m n_b + O(k n_b^2)
// instead of the 4 N m k n_b + 2 (k n_b)^2 of the dense stacked system.
//
// Layout: one warp per point.  Lanes split the nodes in the dual step and in
// K^T y (one n_b-vector, reduced across the warp) and the copies in the prox
// (copy j on lane j mod 32, at most 64 copies, n_b <= 8 state components per
// copy in registers).  The base tables of the point's horizon are k
// instances (one per W_j) with the layout of common.cuh.
//
// Certificate (every gap_every iterations), as for the dense kernels: P at
// the pbar of the dual step, P = sum_j pbar_j^T M_j pbar_j / 4 + 1 -
// <x0, pbar> + sum_i w_i |K_i sum_j pbar_j|_*, and D at the new feasible y,
// D = 1 - sum_j u_j^T V_j u_j with u_j = x0_j - K^T y.
#include "common.cuh"

namespace hopf {

constexpr int ST_NB = 8;   // base state dimension <= 8
constexpr int ST_C = 2;    // copies per lane: k <= 64
constexpr int ST_M = 16;   // control dimension <= 16

namespace {
template <typename R>
__device__ __forceinline__ R wsum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
}  // namespace

template <typename R>
__global__ void pdhg_stacked_kernel(const R *__restrict__ inst_base, SolveParams prm, int k,
                                    const R *__restrict__ x, const R *__restrict__ p_init, R *__restrict__ phi,
                                    R *__restrict__ pstar, R *__restrict__ gap_out, int *__restrict__ iters,
                                    int *__restrict__ status, R *__restrict__ y_scratch) {
    const int nb = prm.n, m = prm.m, N = prm.N, n = nb * k;
    const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pt = blockIdx.x * warps + warp;
    if (pt >= prm.P) return;
    const InstanceLayout L = InstanceLayout::make(nb, m, N);
    const R *I0 = inst_base + (prm.inst_stride ? (long long)pt * k * L.stride : 0LL);
    const R *K = I0 + L.K, *w = I0 + L.w, *sc = I0 + L.sc;
    const R sigma = sc[SC_SIGMA] / R(k);
    const R tau = (R)prm.tau;
    const bool ball = prm.ctrl_kind == HOPF_BALL;
    R *y = y_scratch + (long long)pt * N * m;

    R p[ST_C][ST_NB], pb[ST_C][ST_NB], x0[ST_C][ST_NB];
#pragma unroll
    for (int c = 0; c < ST_C; ++c) {
        const int j = lane + 32 * c;
#pragma unroll
        for (int a = 0; a < ST_NB; ++a) {
            const bool ok = j < k && a < nb;
            x0[c][a] = ok ? x[(long long)pt * n + j * nb + a] : R(0);
            p[c][a] = ok ? (prm.warm ? p_init[(long long)pt * n + j * nb + a] : x0[c][a]) : R(0);
            pb[c][a] = p[c][a];
        }
    }

    if (sc[SC_ZERO] != R(0)) {
        // T = 0: phi = sum_j x_j^T V_j x_j - 1, p* = 2 V_j x_j per copy
        R part = 0;
#pragma unroll
        for (int c = 0; c < ST_C; ++c) {
            const int j = lane + 32 * c;
            if (j >= k) continue;
            const R *V = I0 + (long long)j * L.stride + L.V;
#pragma unroll
            for (int a = 0; a < ST_NB; ++a) {
                if (a >= nb) break;
                R s = 0;
#pragma unroll
                for (int b = 0; b < ST_NB; ++b)
                    if (b < nb) s = fma(V[a * nb + b], x0[c][b], s);
                pstar[(long long)pt * n + j * nb + a] = R(2) * s;
                part = fma(x0[c][a], s, part);
            }
        }
        const R J = wsum(part) - R(1);
        if (lane == 0) {
            phi[pt] = J;
            gap_out[pt] = 0;
            iters[pt] = 0;
            status[pt] = HOPF_OK;
        }
        return;
    }

    auto copy_sum = [&](R (&v)[ST_C][ST_NB], R (&out)[ST_NB]) {
#pragma unroll
        for (int a = 0; a < ST_NB; ++a) {
            R s = 0;
#pragma unroll
            for (int c = 0; c < ST_C; ++c) s += v[c][a];
            out[a] = wsum(s);
        }
    };

    // y0 = K~ p0 (cold, §VI) or w_i argmax_{c in U} <c, K~_i p0> (warm)
    {
        R ps[ST_NB];
        copy_sum(p, ps);
        for (int i = lane; i < N; i += 32) {
            R z[ST_M];
            R nt = 0;
#pragma unroll
            for (int c = 0; c < ST_M; ++c) {
                R s = 0;
                if (c < m) {
#pragma unroll
                    for (int a = 0; a < ST_NB; ++a)
                        if (a < nb) s = fma(K[((long long)i * m + c) * nb + a], ps[a], s);
                }
                z[c] = s;
                nt = fma(s, s, nt);
            }
            const R wi = w[i];
#pragma unroll
            for (int c = 0; c < ST_M; ++c) {
                if (c >= m) break;
                R v = z[c];
                if (prm.warm) {
                    if (ball) v = nt > R(0) ? wi * v / sqrt(nt) : R(0);
                    else v = v >= R(0) ? wi : -wi;
                }
                y[(long long)i * m + c] = v;
            }
        }
        __syncwarp();
    }

    const int g = prm.gap_every;
    R Pc = 0, Dc = 0, gc = 0;
    int st = HOPF_MAXITER, it = 1;
    for (;; ++it) {
        const bool check = it >= 2 && (it % g == 0 || it > prm.max_iter);
        R ps[ST_NB];
        copy_sum(pb, ps);
        // dual step (Eq. 22-23) on the lane's nodes
        R hs = 0;
        for (int i = lane; i < N; i += 32) {
            R z[ST_M];
            R nt = 0, nu = 0;
            const R wi = w[i];
#pragma unroll
            for (int c = 0; c < ST_M; ++c) {
                if (c >= m) break;
                R s = 0;
#pragma unroll
                for (int a = 0; a < ST_NB; ++a)
                    if (a < nb) s = fma(K[((long long)i * m + c) * nb + a], ps[a], s);
                nt += ball ? s * s : fabs(s);
                const R u = fma(sigma, s, y[(long long)i * m + c]);
                z[c] = u;
                nu = fma(u, u, nu);
            }
            if (check) hs = fma(wi, ball ? sqrt(nt) : nt, hs);
            const R scl = (ball && nu > wi * wi) ? wi / sqrt(nu) : R(1);
#pragma unroll
            for (int c = 0; c < ST_M; ++c) {
                if (c >= m) break;
                y[(long long)i * m + c] = ball ? z[c] * scl : fmin(fmax(z[c], -wi), wi);
            }
        }
        // r = K^T y, one base-size vector
        R r[ST_NB];
#pragma unroll
        for (int a = 0; a < ST_NB; ++a) r[a] = 0;
        for (int i = lane; i < N; i += 32) {
#pragma unroll
            for (int c = 0; c < ST_M; ++c) {
                if (c >= m) break;
                const R yv = y[(long long)i * m + c];
#pragma unroll
                for (int a = 0; a < ST_NB; ++a)
                    if (a < nb) r[a] = fma(K[((long long)i * m + c) * nb + a], yv, r[a]);
            }
        }
#pragma unroll
        for (int a = 0; a < ST_NB; ++a) r[a] = wsum(r[a]);
        if (check) {
            R qp = 0, dp = 0;
#pragma unroll
            for (int c = 0; c < ST_C; ++c) {
                const int j = lane + 32 * c;
                if (j >= k) continue;
                const R *Mj = I0 + (long long)j * L.stride + L.M;
                const R *Vj = I0 + (long long)j * L.stride + L.V;
                R u[ST_NB];
#pragma unroll
                for (int a = 0; a < ST_NB; ++a) u[a] = x0[c][a] - r[a];
#pragma unroll
                for (int a = 0; a < ST_NB; ++a) {
                    if (a >= nb) break;
                    R mq = 0, vq = 0;
#pragma unroll
                    for (int b = 0; b < ST_NB; ++b)
                        if (b < nb) {
                            mq = fma(Mj[a * nb + b], pb[c][b], mq);
                            vq = fma(Vj[a * nb + b], u[b], vq);
                        }
                    qp = fma(pb[c][a], R(0.25) * mq - x0[c][a], qp);
                    dp = fma(u[a], vq, dp);
                }
            }
            const R H = wsum(hs);
            const R quad = wsum(qp) + R(1);
            Pc = quad + H;
            Dc = R(1) - wsum(dp);
            gc = rel_gap(Pc, Dc);
            if (!isfinite(Pc) || !isfinite(Dc)) { st = HOPF_NONFINITE; break; }
            const R scl = fmax(R(1), fmax(fabs(Pc), fabs(Dc)));
            if (gc + gap_allowance(quad, H, Dc, scl) <= (R)prm.tol_gap) { st = HOPF_OK; break; }
            if (it > prm.max_iter) { st = HOPF_MAXITER; break; }
        }
        // prox of Eq. 37 per copy: p_j <- S_j (p_j - tau r + tau x0_j)
#pragma unroll
        for (int c = 0; c < ST_C; ++c) {
            const int j = lane + 32 * c;
            if (j >= k) continue;
            const R *Sj = I0 + (long long)j * L.stride + L.S;
            R v[ST_NB];
#pragma unroll
            for (int a = 0; a < ST_NB; ++a) v[a] = fma(tau, x0[c][a] - r[a], p[c][a]);
#pragma unroll
            for (int a = 0; a < ST_NB; ++a) {
                if (a >= nb) break;
                R s = 0;
#pragma unroll
                for (int b = 0; b < ST_NB; ++b)
                    if (b < nb) s = fma(Sj[a * nb + b], v[b], s);
                pb[c][a] = R(2) * s - p[c][a];
                p[c][a] = s;
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int c = 0; c < ST_C; ++c) {
        const int j = lane + 32 * c;
        if (j >= k) continue;
#pragma unroll
        for (int a = 0; a < ST_NB; ++a)
            if (a < nb) pstar[(long long)pt * n + j * nb + a] = pb[c][a];
    }
    if (lane == 0) {
        phi[pt] = -Pc;
        gap_out[pt] = gc;
        iters[pt] = it - 1;
        status[pt] = st;
    }
}

template <typename R>
cudaError_t launch_pdhg_stacked(const R *inst, const SolveParams &prm, int k, const R *x, const R *p_init, R *phi,
                                R *pstar, R *gap, int *iters, int *status, R *y, cudaStream_t s) {
    constexpr int warps = 4;
    const int grid = (prm.P + warps - 1) / warps;
    pdhg_stacked_kernel<R><<<grid, warps * 32, 0, s>>>(inst, prm, k, x, p_init, phi, pstar, gap, iters, status, y);
    return cudaGetLastError();
}

template cudaError_t launch_pdhg_stacked<float>(const float *, const SolveParams &, int, const float *,
                                                const float *, float *, float *, float *, int *, int *, float *,
                                                cudaStream_t);
template cudaError_t launch_pdhg_stacked<double>(const double *, const SolveParams &, int, const double *,
                                                 const double *, double *, double *, double *, int *, int *,
                                                 double *, cudaStream_t);

}  // namespace hopf
