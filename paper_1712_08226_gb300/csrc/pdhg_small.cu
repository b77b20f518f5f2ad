// Persistent float32 Chambolle-Pock kernel for one shared node table and a
// small state (n <= 16, m <= 2): the batched value solve of many query points
// of one system at one horizon.
//
// Same iteration, start and certificate as pdhg_generic.cu (§III Eq. 15,
// Eq. 22, Eq. 23, Eq. 37; P at pbar and D at y as described there).
//
// Layout (one thread block per SM, persistent):
//   * the node table row of node i, [K_i (m x NS) | w_i | pad], lives in
//     shared memory (read by every point: one copy per SM);
//   * each query point is owned by a group of TPP consecutive lanes; lane q of
//     the group owns the nodes i = q, q + TPP, q + 2 TPP, ...; the point's dual
//     variable y (N m floats) lives in shared memory, the primal state
//     (p, pbar, sigma pbar, K^T y) in registers, replicated over the group;
//   * one pass over the lane's nodes forms sigma K_i pbar, the projection onto
//     w_i U and the lane's share of K^T y, all from one read of K_i; the group
//     then sums K^T y with TPP-lane shuffles;
//   * groups take new points from a global counter when they finish, so the
//     very uneven iteration counts of different points do not leave SMs idle.
// The dual step is ALU bound: 4 m n FMAs + the projection per node and point.
#include "common.cuh"

namespace hopf {

template <int MS, int NS>
struct KRow {
    static constexpr int used = MS * NS + 1;
    static constexpr int stride = (used + 3) & ~3;
};

template <int NS, int MS, int TPP, bool CHECK>
__device__ __forceinline__ void node_pass(const float *__restrict__ Ks, float *__restrict__ ys, int N,
                                          int q, bool ball, float sigma, const float (&pb)[NS],
                                          float (&acc)[NS], float &hs) {
    constexpr int KR = KRow<MS, NS>::stride;
#pragma unroll 2
    for (int i = q; i < N; i += TPP) {
        float kf[KR];
        const float4 *kr4 = reinterpret_cast<const float4 *>(Ks + (size_t)i * KR);
#pragma unroll
        for (int r = 0; r < KR / 4; ++r) {
            float4 v = kr4[r];
            kf[4 * r] = v.x; kf[4 * r + 1] = v.y; kf[4 * r + 2] = v.z; kf[4 * r + 3] = v.w;
        }
        const float wi = kf[MS * NS];
        float u[MS];
        if (MS == 2) {
            float2 yv = *reinterpret_cast<const float2 *>(ys + 2 * i);
            u[0] = yv.x;
            u[1] = yv.y;
        } else {
            u[0] = ys[i];
        }
        float tn = 0.f, un = 0.f;
#pragma unroll
        for (int c = 0; c < MS; ++c) {
            float t0 = 0.f, t1 = 0.f;       // two partial sums: half-length FMA chains
#pragma unroll
            for (int j = 0; j < NS; j += 2) {
                t0 = fmaf(kf[c * NS + j], pb[j], t0);
                if (j + 1 < NS) t1 = fmaf(kf[c * NS + j + 1], pb[j + 1], t1);
            }
            const float t = t0 + t1;
            if (CHECK) tn = ball ? fmaf(t, t, tn) : tn + fabsf(t);
            u[c] = fmaf(sigma, t, u[c]);
            un = fmaf(u[c], u[c], un);
        }
        if (CHECK) hs = fmaf(wi, ball ? sqrtf(tn) : tn, hs);   // sum_i w_i |K_i pbar|_*
        if (ball) {
            float scale = (un > wi * wi) ? wi * rsqrtf(un) : 1.f;
#pragma unroll
            for (int c = 0; c < MS; ++c) u[c] *= scale;
        } else {
#pragma unroll
            for (int c = 0; c < MS; ++c) u[c] = fminf(fmaxf(u[c], -wi), wi);
        }
        if (MS == 2) {
            *reinterpret_cast<float2 *>(ys + 2 * i) = make_float2(u[0], u[1]);
        } else {
            ys[i] = u[0];
        }
#pragma unroll
        for (int c = 0; c < MS; ++c)
#pragma unroll
            for (int j = 0; j < NS; ++j) acc[j] = fmaf(kf[c * NS + j], u[c], acc[j]);
    }
}

template <int NS, int MS, int TPP>
__global__ void __launch_bounds__(384, 1)
pdhg_small_kernel(const float *__restrict__ inst, SolveParams prm, int ys_stride,
                  const float *__restrict__ x, const float *__restrict__ p_init,
                  float *__restrict__ phi, float *__restrict__ pstar, float *__restrict__ gap_out,
                  int *__restrict__ iters, int *__restrict__ status, int *__restrict__ counter) {
    static_assert(32 % TPP == 0, "groups must tile a warp");
    constexpr int KR = KRow<MS, NS>::stride;
    const int n = prm.n, N = prm.N;
    const int P = prm.list ? *prm.list_count : prm.P;   // number of points to take
    const InstanceLayout L = InstanceLayout::make(n, prm.m, N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *Ks = reinterpret_cast<float *>(smem_raw);
    float *Ss = Ks + (size_t)N * KR;
    float *Msm = Ss + NS * NS;
    float *Vs = Msm + NS * NS;
    float *Us = Vs + NS * NS;
    float *lams = Us + NS * NS;
    float *X0s = lams + ((NS + 3) & ~3);          // [slots][NS] query points
    float *Ys = X0s + (size_t)(blockDim.x / TPP) * NS;

    // stage the table once per block, zero-padding the state to NS components
    for (int e = threadIdx.x; e < N * KR; e += blockDim.x) {
        int i = e / KR, r = e % KR;
        float v = 0.f;
        if (r < MS * NS) {
            int c = r / NS, j = r % NS;
            if (j < n) v = inst[L.K + ((size_t)i * MS + c) * n + j];
        } else if (r == MS * NS) {
            v = inst[L.w + i];
        }
        Ks[e] = v;
    }
    for (int e = threadIdx.x; e < NS * NS; e += blockDim.x) {
        int a = e / NS, b = e % NS;
        bool in = a < n && b < n;
        Ss[e] = in ? inst[L.S + a * n + b] : (a == b ? 1.f : 0.f);
        Msm[e] = in ? inst[L.M + a * n + b] : 0.f;
        Vs[e] = in ? inst[L.V + a * n + b] : 0.f;
        Us[e] = in ? inst[L.U + a * n + b] : (a == b ? 1.f : 0.f);
    }
    for (int e = threadIdx.x; e < NS; e += blockDim.x) lams[e] = e < n ? inst[L.lam + e] : 0.f;
    __syncthreads();

    const float sigma0 = inst[L.sc + SC_SIGMA];
    const float gamma = inst[L.sc + SC_GAMMA];
    const bool accel = prm.accel != 0;
    const bool zero = inst[L.sc + SC_ZERO] != 0.f;
    const float tau0 = (float)prm.tau;
    const float tol = (float)prm.tol_gap;
    const bool ball = prm.ctrl_kind == HOPF_BALL;
    const int g = prm.gap_every;

    const int lane = threadIdx.x & 31;
    const int q = threadIdx.x % TPP;
    const int slot = threadIdx.x / TPP;
    const int lead = lane - q;
    const unsigned gmask = (TPP == 32) ? 0xffffffffu : (((1u << TPP) - 1u) << lead);
    float *ys = Ys + (size_t)slot * ys_stride;
    float *x0 = X0s + (size_t)slot * NS;

    float p[NS], pb[NS], acc[NS];
    int pt = -1, it_pt = 0, slot_in = -1;
    bool idle = false, have_D = false, fresh = false;
    float Dprev = 0.f;
    float tau = tau0, sigma = sigma0;      // current steps (they change only when accelerated)
    const int n_carry = prm.carry_in ? *prm.in_count : 0;

    // take the next point for this group; T = 0 points finish on the spot
    auto fetch = [&]() {
        for (;;) {
            int nx = 0;
            if (q == 0) nx = atomicAdd(counter, 1);
            nx = __shfl_sync(gmask, nx, lead);
            if (nx >= (prm.carry_in ? n_carry : P)) { idle = true; pt = -1; return; }
            slot_in = nx;
            pt = prm.carry_in ? prm.in_list[nx] : (prm.list ? prm.list[nx] : nx);
            __syncwarp(gmask);
            if (q == 0) {
#pragma unroll
                for (int j = 0; j < NS; ++j) x0[j] = (j < n) ? x[(size_t)pt * n + j] : 0.f;
            }
            __syncwarp(gmask);
            if (!zero) break;
            float J = -1.f;
#pragma unroll
            for (int a = 0; a < NS; ++a) {
                float s = 0.f;
#pragma unroll
                for (int b = 0; b < NS; ++b) s = fmaf(Vs[a * NS + b], x0[b], s);
                J = fmaf(x0[a], s, J);
                if (a < n && (a % TPP) == q) pstar[(size_t)pt * n + a] = 2.f * s;
            }
            if (q == 0) {
                phi[pt] = J; gap_out[pt] = 0.f; iters[pt] = 0; status[pt] = HOPF_OK;
            }
        }
        have_D = false;
        fresh = true;
        if (prm.carry_in) {
            // resume a point parked by the throughput phase: primal state, step
            // sizes, iteration count and the dual variable y
            const float *st = prm.in_st + (size_t)slot_in * CARRY_W;
#pragma unroll
            for (int j = 0; j < NS; ++j) {
                p[j] = st[j];
                pb[j] = st[16 + j];
            }
            tau = st[32];
            sigma = st[33];
            it_pt = __float_as_int(st[34]);
            const float *cy = prm.in_y + (size_t)slot_in * N * MS;
            for (int i = q; i < N; i += TPP)
#pragma unroll
                for (int c = 0; c < MS; ++c) ys[i * MS + c] = cy[(size_t)i * MS + c];
            return;
        }
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            float v = (prm.warm && j < n) ? p_init[(size_t)pt * n + j] : x0[j];
            p[j] = v;
            pb[j] = v;
        }
        for (int i = q; i < N; i += TPP) {
            const float *kr = Ks + (size_t)i * KR;
            float t[MS], nr = 0.f;
#pragma unroll
            for (int c = 0; c < MS; ++c) {
                float s = 0.f;
#pragma unroll
                for (int j = 0; j < NS; ++j) s = fmaf(kr[c * NS + j], p[j], s);
                t[c] = s;
                nr = fmaf(s, s, nr);
            }
            if (prm.warm) {
                const float wi = kr[MS * NS];
                if (ball) {
                    float sc = nr > 0.f ? wi * rsqrtf(nr) : 0.f;
#pragma unroll
                    for (int c = 0; c < MS; ++c) t[c] *= sc;
                } else {
#pragma unroll
                    for (int c = 0; c < MS; ++c) t[c] = t[c] >= 0.f ? wi : -wi;
                }
            }
#pragma unroll
            for (int c = 0; c < MS; ++c) ys[i * MS + c] = t[c];
        }
        it_pt = 0;
        tau = tau0;
        sigma = sigma0;
    };

    fetch();
    fresh = false;            // the first iteration of the first point is a full one
    int wit = 0;
    for (;;) {
        ++wit;
        ++it_pt;
        const bool check = (wit % g) == 0;
        bool park = false;
        float hs = 0.f;
#pragma unroll
        for (int j = 0; j < NS; ++j) acc[j] = 0.f;
        if (check) node_pass<NS, MS, TPP, true>(Ks, ys, N, q, ball, sigma, pb, acc, hs);
        else node_pass<NS, MS, TPP, false>(Ks, ys, N, q, ball, sigma, pb, acc, hs);
#pragma unroll
        for (int o = TPP / 2; o > 0; o >>= 1) {
#pragma unroll
            for (int j = 0; j < NS; ++j) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
        }
        if (check) {
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1) hs += __shfl_xor_sync(0xffffffffu, hs, o);
            if (!idle && it_pt >= 2 && have_D) {
                float quad = 1.f;
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    float s = 0.f;
#pragma unroll
                    for (int b = 0; b < NS; ++b) s = fmaf(Msm[a * NS + b], pb[b], s);
                    quad = fmaf(pb[a], fmaf(0.25f, s, -x0[a]), quad);
                }
                const float Pc = quad + hs;
                const float Dc = Dprev;
                const float gc = rel_gap(Pc, Dc);
                const bool bad = !isfinite(Pc) || !isfinite(Dc);
                const float scl = fmaxf(1.f, fmaxf(fabsf(Pc), fabsf(Dc)));
                const bool conv = gc + gap_allowance(quad, hs, Dc, scl) <= tol;
                if (bad || conv || it_pt - 1 >= prm.max_iter) {
#pragma unroll
                    for (int j = 0; j < NS; ++j)
                        if (j < n && (j % TPP) == q) pstar[(size_t)pt * n + j] = pb[j];
                    if (q == 0) {
                        phi[pt] = -Pc;
                        gap_out[pt] = gc;
                        iters[pt] = it_pt - 1;
                        status[pt] = bad ? HOPF_NONFINITE : (conv ? HOPF_OK : HOPF_MAXITER);
                    }
                    fetch();
                } else if (prm.carry_cap > 0 &&
                           (it_pt - 1 >= prm.carry_cap || __ldcg(counter) >= (prm.carry_in ? n_carry : P))) {
                    // hand over to the next (lower-latency) phase after this step: after
                    // carry_cap iterations, or as soon as no new point is left to take
                    // (then the slots of this phase would only drain)
                    park = true;
                }
            }
            if (__all_sync(0xffffffffu, idle)) break;
        }
        if (!fresh) {
            float pn[NS], v[NS];
#pragma unroll
            for (int b = 0; b < NS; ++b) v[b] = fmaf(-tau, acc[b], fmaf(tau, x0[b], p[b]));
            float th = 1.f;
            if constexpr (TPP >= NS) {
                // one lane per row of the n x n products, rows gathered by shuffles
                const int a = q < NS ? q : 0;
                float r = 0.f;
                if (accel) {
#pragma unroll
                    for (int b = 0; b < NS; ++b) r = fmaf(Us[b * NS + a], v[b], r);
                    r = __fdividef(r, fmaf(0.5f * tau, lams[a], 1.f));
                    float z[NS];
#pragma unroll
                    for (int b = 0; b < NS; ++b) z[b] = __shfl_sync(gmask, r, lead + b);
                    r = 0.f;
#pragma unroll
                    for (int b = 0; b < NS; ++b) r = fmaf(Us[a * NS + b], z[b], r);
                    th = rsqrtf(fmaf(2.f * gamma, tau, 1.f));
                    tau *= th;
                    sigma /= th;
                } else {
#pragma unroll
                    for (int b = 0; b < NS; ++b) r = fmaf(Ss[a * NS + b], v[b], r);
                }
#pragma unroll
                for (int b = 0; b < NS; ++b) pn[b] = __shfl_sync(gmask, r, lead + b);
            } else if (accel) {
                // (I + tau M/2)^-1 v = U diag(1 / (1 + tau lam / 2)) U^T v
                float z[NS];
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    float s = 0.f;
#pragma unroll
                    for (int b = 0; b < NS; ++b) s = fmaf(Us[b * NS + a], v[b], s);
                    z[a] = __fdividef(s, fmaf(0.5f * tau, lams[a], 1.f));
                }
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    float s = 0.f;
#pragma unroll
                    for (int b = 0; b < NS; ++b) s = fmaf(Us[a * NS + b], z[b], s);
                    pn[a] = s;
                }
                th = rsqrtf(fmaf(2.f * gamma, tau, 1.f));
                tau *= th;
                sigma /= th;
            } else {
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    float s = 0.f;
#pragma unroll
                    for (int b = 0; b < NS; ++b) s = fmaf(Ss[a * NS + b], v[b], s);
                    pn[a] = s;
                }
            }
#pragma unroll
            for (int j = 0; j < NS; ++j) {
                pb[j] = fmaf(th, pn[j] - p[j], pn[j]);
                p[j] = pn[j];
            }
            if (park) {
                // save the point after this full step and take a new one
                int slot = 0;
                if (q == 0) slot = atomicAdd(prm.out_count, 1);
                slot = __shfl_sync(gmask, slot, lead);
                float *cy = prm.out_y + (size_t)slot * N * MS;
                for (int i = q; i < N; i += TPP)
#pragma unroll
                    for (int c = 0; c < MS; ++c) cy[(size_t)i * MS + c] = ys[i * MS + c];
                if (q == 0) {
                    float *st = prm.out_st + (size_t)slot * CARRY_W;
#pragma unroll
                    for (int j = 0; j < NS; ++j) {
                        st[j] = p[j];
                        st[16 + j] = pb[j];
                    }
                    st[32] = tau;
                    st[33] = sigma;
                    st[34] = __int_as_float(it_pt);
                    prm.out_list[slot] = pt;
                }
                __syncwarp(gmask);
                fetch();
            } else if (((wit + 1) % g) == 0) {
                float dq = 1.f;
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    float s = 0.f;
#pragma unroll
                    for (int b = 0; b < NS; ++b) s = fmaf(Vs[a * NS + b], x0[b] - acc[b], s);
                    dq = fmaf(-(x0[a] - acc[a]), s, dq);
                }
                Dprev = dq;
                have_D = true;
            }
        }
        fresh = false;
    }
}

// Host launcher: picks the instantiation for (NS, m); TPP = 4.
int small_supported_ns(int n) { return (n + 1) & ~1; }

cudaError_t launch_pdhg_small(int NS, int m, int tpp, int grid, int threads, size_t smem, cudaStream_t s,
                              const float *inst, const SolveParams &prm, int ys_stride, const float *x,
                              const float *p_init, float *phi, float *pstar, float *gap, int *iters,
                              int *status, int *counter) {
    void (*fn)(const float *, SolveParams, int, const float *, const float *, float *, float *, float *,
               int *, int *, int *) = nullptr;
#define HOPF_CASE(NSV)                                                                           \
    case NSV:                                                                                    \
        if (tpp == 32) fn = (m == 1) ? pdhg_small_kernel<NSV, 1, 32> : pdhg_small_kernel<NSV, 2, 32>; \
        else fn = (m == 1) ? pdhg_small_kernel<NSV, 1, 4> : pdhg_small_kernel<NSV, 2, 4>;        \
        break;
    switch (NS) {
        HOPF_CASE(2) HOPF_CASE(4) HOPF_CASE(6) HOPF_CASE(8)
        HOPF_CASE(10) HOPF_CASE(12) HOPF_CASE(14) HOPF_CASE(16)
        default: return cudaErrorInvalidValue;
    }
#undef HOPF_CASE
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, threads, smem, s>>>(inst, prm, ys_stride, x, p_init, phi, pstar, gap, iters, status, counter);
    return cudaGetLastError();
}

}  // namespace hopf
