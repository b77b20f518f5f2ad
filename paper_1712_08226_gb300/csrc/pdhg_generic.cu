// Chambolle-Pock iteration for the discretised generalized Hopf formula,
// general sizes: one warp per query point, any n, m (<= 16) and N, float64 or
// float32, one shared node table or one table per point (time-to-reach).
//
// Iteration (§III, Eq. 15 with theta = 1, §VI):
//   y_i   <- Proj_{w_i U}( y_i + sigma K_i pbar )            Eq. 22, Eq. 23
//   p_new <- S (p - tau sum_i K_i^T y_i + tau x0)             Eq. 37
//   pbar  <- 2 p_new - p
// Start (§VI): p = pbar = x0, y = K x0; a warm start p0 uses
// y_i = w_i argmax_{c in U} <c, K_i p0> instead (the dual point that the
// optimality condition pairs with p0).
//
// Certificate every gap_every iterations: the primal objective of Eq. 18 at
// pbar, P = pbar^T M pbar / 4 + 1 - <x0, pbar> + sum_i w_i |K_i pbar|_*, and
// the Fenchel dual D(y) = 1 - (x0 - K^T y)^T V (x0 - K^T y) at the feasible y
// of the same iteration, so that phi lies in [-P, -D].  K_i pbar is already
// formed by the dual step (as sigma K_i pbar), so the certificate costs no
// extra pass over the nodes.  Stop when (P - D)/max(1,|P|,|D|) <= tol_gap, or
// (time-to-reach) as soon as [-P, -D] excludes zero.
//
// Lanes of a warp split the nodes in the dual step and the state components
// in the K^T y, S and quadratic-form products.  The dual variable y lives in
// a global scratch array (N m values per point).
//
// Adaptive steps (prm.adaptive): after a step the residuals of §III.B,
//   r_p = (p^k - p^{k-1})/tau - K^T (y^k - y^{k-1}),
//   r_d = (y^k - y^{k-1})/sigma - K (p^k - p^{k-1}),
// are measured (|r_d|^2 = |dy|^2/sigma^2 - 2 <K^T dy, dp>/sigma + dp^T G dp
// with the Gram matrix G = K^T K of the table) and balanced (Goldstein et
// al.): tau /= (1 - a), sigma *= (1 - a) when |r_p| > 1.5 |r_d|, the reverse
// when 1.5 |r_p| < |r_d|, a *= 0.95 after a change; the prox of G is then
// taken at the current tau through M = U diag(lam) U^T.
//
// Fixed-step rule (prm.fx_nk set): one table on [0, t_max] in terminal-time
// variables; point k uses its first fx_nk[k] nodes, the last one weighted
// fx_wl[k], and its own dual step fx_sig[k] (nodes beyond take no part).
#include "common.cuh"

namespace hopf {

constexpr int GEN_MMAX = 16;

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R>
__global__ void pdhg_generic_kernel(const R *__restrict__ inst_base, SolveParams prm,
                                    const R *__restrict__ x, const R *__restrict__ p_init,
                                    R *__restrict__ phi, R *__restrict__ pstar, R *__restrict__ gap_out,
                                    int *__restrict__ iters, int *__restrict__ status,
                                    R *__restrict__ P_out, R *__restrict__ D_out,
                                    R *__restrict__ y_scratch, const int *__restrict__ active) {
    const int n = prm.n, m = prm.m, N = prm.N;
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int k = blockIdx.x * warps + warp;
    if (prm.list) {
        if (k >= *prm.list_count) return;        // uniform per warp
        k = prm.list[k];
    } else if (k >= prm.P) {
        return;
    }
    if (active && !active[k]) return;
    extern __shared__ unsigned char smem_raw[];
    R *sm = reinterpret_cast<R *>(smem_raw) + (size_t)warp * 7 * n;
    R *p = sm, *pb = sm + n, *qv = sm + 2 * n, *acc = sm + 3 * n, *x0 = sm + 4 * n, *vt = sm + 5 * n;
    R *accp = sm + 6 * n;                                      // K^T y of the previous step (adaptive)

    const InstanceLayout L = InstanceLayout::make(n, m, N);
    const R *I = inst_base + (prm.inst_stride ? (long long)k * L.stride : 0LL);
    const R *K = I + L.K, *w = I + L.w, *M = I + L.M, *V = I + L.V, *S = I + L.S, *sc = I + L.sc;
    const bool fx = prm.fx_nk != nullptr;
    const int Nk = fx ? prm.fx_nk[k] : N;
    if (Nk < 0) return;                                        // horizon out of range: outputs already set
    const R wlast = fx ? (R)prm.fx_wl[k] : R(0);
    auto wt = [&](int i) -> R { return (fx && i == Nk - 1) ? wlast : w[i]; };
    R sigma = fx ? (R)prm.fx_sig[k] : sc[SC_SIGMA];
    const R gamma = sc[SC_GAMMA];
    const bool zero = sc[SC_ZERO] != R(0);
    R tau = (R)prm.tau;
    const R *U = I + L.U, *lam = I + L.lam, *G = I + L.G;
    R alpha = R(0.5);
    R *y = y_scratch + (long long)k * N * m;
    const bool ball = prm.ctrl_kind == HOPF_BALL;

    for (int j = lane; j < n; j += 32) x0[j] = x[(long long)k * n + j];
    __syncwarp();

    if (zero) {
        // T = 0: phi = J_x(x) = x^T V x - 1 (V = W^-1 here), p* = grad J_x = 2 V x
        R part = 0;
        for (int j = lane; j < n; j += 32) {
            R s = 0;
            for (int l = 0; l < n; ++l) s = fma(V[j * n + l], x0[l], s);
            pstar[(long long)k * n + j] = R(2) * s;
            part = fma(x0[j], s, part);
        }
        R J = warp_sum(part) - R(1);
        if (lane == 0) {
            phi[k] = J;
            gap_out[k] = 0;
            iters[k] = 0;
            status[k] = HOPF_OK;
            if (P_out) P_out[k] = -J;
            if (D_out) D_out[k] = -J;
        }
        return;
    }

    for (int j = lane; j < n; j += 32) {
        R v = prm.warm ? p_init[(long long)k * n + j] : x0[j];
        p[j] = v;
        pb[j] = v;
    }
    __syncwarp();
    // y0: K p0 (cold, §VI) or w_i argmax_U <c, K_i p0> (warm)
    for (int i = lane; i < Nk; i += 32) {
        R t[GEN_MMAX];
        const R *Ki = K + (long long)i * m * n;
        R nrm2 = 0;
        for (int c = 0; c < m; ++c) {
            R s = 0;
            for (int j = 0; j < n; ++j) s = fma(Ki[c * n + j], p[j], s);
            t[c] = s;
            nrm2 = fma(s, s, nrm2);
        }
        R wi = wt(i);
        for (int c = 0; c < m; ++c) {
            R v = t[c];
            if (prm.warm) {
                if (ball) v = (nrm2 > R(0)) ? wi * v / sqrt(nrm2) : R(0);
                else v = (v >= R(0)) ? wi : -wi;
            }
            y[(long long)i * m + c] = v;
        }
    }
    __syncwarp();
    if (prm.adaptive) {
        for (int j = lane; j < n; j += 32) {
            R s = 0;
            for (int i = 0; i < Nk; ++i)
                for (int c = 0; c < m; ++c) s = fma(K[((long long)i * m + c) * n + j], y[(long long)i * m + c], s);
            accp[j] = s;
        }
        __syncwarp();
    }

    const int g = prm.gap_every;
    auto is_check = [&](int it) { return it >= 2 && (it % g == 0 || it > prm.max_iter); };
    R Dprev = 0, Pc = 0, Dc = 0, gc = 0;
    int st = HOPF_MAXITER;
    int it = 1;
    for (;; ++it) {
        const bool check = is_check(it);
        for (int j = lane; j < n; j += 32) qv[j] = sigma * pb[j];
        __syncwarp();
        R hs = 0, dy2 = 0;
        for (int i = lane; i < Nk; i += 32) {
            R t[GEN_MMAX];
            const R *Ki = K + (long long)i * m * n;
            R *yi = y + (long long)i * m;
            const R wi = wt(i);
            R nt = 0, nu = 0;
            for (int c = 0; c < m; ++c) {
                R s = 0;
                for (int j = 0; j < n; ++j) s = fma(Ki[c * n + j], qv[j], s);
                nt += ball ? s * s : fabs(s);
                R u = yi[c] + s;
                t[c] = u;
                nu = fma(u, u, nu);
            }
            if (check) hs = fma(wi, ball ? sqrt(nt) : nt, hs);
            if (ball) {
                R scale = (nu > wi * wi) ? wi / sqrt(nu) : R(1);
                for (int c = 0; c < m; ++c) {
                    const R yn = t[c] * scale;
                    if (prm.adaptive) dy2 = fma(yn - yi[c], yn - yi[c], dy2);
                    yi[c] = yn;
                }
            } else {
                for (int c = 0; c < m; ++c) {
                    const R yn = fmin(fmax(t[c], -wi), wi);
                    if (prm.adaptive) dy2 = fma(yn - yi[c], yn - yi[c], dy2);
                    yi[c] = yn;
                }
            }
        }
        if (check) {
            hs = warp_sum(hs);
            R H = (sigma > R(0)) ? hs / sigma : R(0);
            R part = 0;
            for (int j = lane; j < n; j += 32) {
                R s = 0;
                for (int l = 0; l < n; ++l) s = fma(M[j * n + l], pb[l], s);
                part += pb[j] * (R(0.25) * s - x0[j]);
            }
            const R quad = warp_sum(part) + R(1);
            Pc = quad + H;
            Dc = Dprev;
            gc = rel_gap(Pc, Dc);
            if (!isfinite(Pc) || !isfinite(Dc)) { st = HOPF_NONFINITE; break; }
            const R scl = fmax(R(1), fmax(fabs(Pc), fabs(Dc)));
            bool conv = gc + gap_allowance(quad, H, Dc, scl) <= (R)prm.tol_gap;
            if (prm.sign_mode) conv = conv || Pc < R(0) || Dc > R(0) || gc <= (R)prm.sign_floor;
            if (conv) { st = HOPF_OK; break; }
            if (it > prm.max_iter) { st = HOPF_MAXITER; break; }
        }
        __syncwarp();
        // K^T y: lanes over state components, sum over nodes
        for (int j = lane; j < n; j += 32) {
            R s = 0;
            for (int i = 0; i < Nk; ++i) {
                const R *Ki = K + (long long)i * m * n;
                const R *yi = y + (long long)i * m;
                for (int c = 0; c < m; ++c) s = fma(Ki[c * n + j], yi[c], s);
            }
            acc[j] = s;
            vt[j] = p[j] - tau * s + tau * x0[j];
        }
        __syncwarp();
        if (prm.accel) {
            // prox of G at the current tau: U diag(1 / (1 + tau lam / 2)) U^T vt
            for (int j = lane; j < n; j += 32) {
                R s = 0;
                for (int l = 0; l < n; ++l) s = fma(U[l * n + j], vt[l], s);
                qv[j] = s / fma(R(0.5) * tau, lam[j], R(1));
            }
            __syncwarp();
            const R th = R(1) / sqrt(fma(R(2) * gamma, tau, R(1)));
            for (int j = lane; j < n; j += 32) {
                R s = 0;
                for (int l = 0; l < n; ++l) s = fma(U[j * n + l], qv[l], s);
                pb[j] = fma(th, s - p[j], s);
                p[j] = s;
            }
            tau *= th;
            sigma /= th;
        } else if (prm.adaptive) {
            // prox of G at the current tau, then the residual balance
            for (int j = lane; j < n; j += 32) {
                R s = 0;
                for (int l = 0; l < n; ++l) s = fma(U[l * n + j], vt[l], s);
                qv[j] = s / fma(R(0.5) * tau, lam[j], R(1));
            }
            __syncwarp();
            for (int j = lane; j < n; j += 32) {
                R s = 0;
                for (int l = 0; l < n; ++l) s = fma(U[j * n + l], qv[l], s);
                vt[j] = s - p[j];                  // dp (vt is free until the next step)
                pb[j] = R(2) * s - p[j];
                p[j] = s;
            }
            __syncwarp();
            R rp2 = 0, cross = 0, qg = 0;
            for (int j = lane; j < n; j += 32) {
                const R da = acc[j] - accp[j];
                const R r = vt[j] / tau - da;
                rp2 = fma(r, r, rp2);
                cross = fma(da, vt[j], cross);
                R s = 0;
                for (int l = 0; l < n; ++l) s = fma(G[j * n + l], vt[l], s);
                qg = fma(vt[j], s, qg);
                accp[j] = acc[j];
            }
            rp2 = warp_sum(rp2);
            cross = warp_sum(cross);
            qg = warp_sum(qg);
            const R dyy = warp_sum(dy2);
            const R rd2 = fmax(dyy / (sigma * sigma) - R(2) * cross / sigma + qg, R(0));
            const R npr = sqrt(rp2), ndr = sqrt(rd2);
            if (npr > R(1.5) * ndr) {
                tau /= (R(1) - alpha);
                sigma *= (R(1) - alpha);
                alpha *= R(0.95);
            } else if (R(1.5) * npr < ndr) {
                tau *= (R(1) - alpha);
                sigma /= (R(1) - alpha);
                alpha *= R(0.95);
            }
        } else {
            for (int j = lane; j < n; j += 32) {
                R s = 0;
                for (int l = 0; l < n; ++l) s = fma(S[j * n + l], vt[l], s);
                pb[j] = R(2) * s - p[j];
                p[j] = s;
            }
        }
        __syncwarp();
        if (is_check(it + 1)) {
            for (int j = lane; j < n; j += 32) vt[j] = x0[j] - acc[j];
            __syncwarp();
            R part = 0;
            for (int j = lane; j < n; j += 32) {
                R s = 0;
                for (int l = 0; l < n; ++l) s = fma(V[j * n + l], vt[l], s);
                part = fma(vt[j], s, part);
            }
            Dprev = R(1) - warp_sum(part);
            __syncwarp();
        }
    }
    for (int j = lane; j < n; j += 32) pstar[(long long)k * n + j] = pb[j];
    if (lane == 0) {
        phi[k] = -Pc;
        gap_out[k] = gc;
        iters[k] = it - 1;
        status[k] = st;
        if (P_out) P_out[k] = Pc;
        if (D_out) D_out[k] = Dc;
    }
}

template <typename R>
cudaError_t launch_pdhg_generic(const R *inst, const SolveParams &prm, const R *x, const R *p_init, R *phi,
                                R *pstar, R *gap, int *iters, int *status, R *Pv, R *Dv, R *y,
                                const int *active, cudaStream_t s) {
    constexpr int warps = 4;
    const int threads = warps * 32;
    const int grid = (prm.P + warps - 1) / warps;
    const size_t smem = (size_t)warps * 7 * prm.n * sizeof(R);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(pdhg_generic_kernel<R>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    pdhg_generic_kernel<R><<<grid, threads, smem, s>>>(inst, prm, x, p_init, phi, pstar, gap, iters, status,
                                                       Pv, Dv, y, active);
    return cudaGetLastError();
}

template cudaError_t launch_pdhg_generic<double>(const double *, const SolveParams &, const double *,
                                                 const double *, double *, double *, double *, int *, int *,
                                                 double *, double *, double *, const int *, cudaStream_t);
template cudaError_t launch_pdhg_generic<float>(const float *, const SolveParams &, const float *,
                                                const float *, float *, float *, float *, int *, int *, float *,
                                                float *, float *, const int *, cudaStream_t);

}  // namespace hopf
