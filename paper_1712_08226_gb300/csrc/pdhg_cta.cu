// Latency kernel of the small-state float32 solve: one thread block per query
// point, one (or two) quadrature nodes per thread.  It finishes the points that
// the throughput kernel (pdhg_small.cu, 4 lanes per point) parked after
// carry_cap iterations: few points, many iterations each, so the time per
// iteration matters more than the work per iteration.
//
// Same iteration, certificate and stopping rule as pdhg_small.cu (§III
// Eq. 15, Eq. 22, Eq. 23, Eq. 37; accelerated steps for a strongly convex G).
// Per iteration:
//   * every thread forms sigma K_i pbar, projects y_i onto w_i U and adds its
//     K_i^T y_i to a private copy of K^T y; its node rows K_i stay in registers
//     for the life of the block and pbar is read from shared memory;
//   * the NS partial sums of each warp are combined by a reduce-scatter of
//     shuffles (16 shuffles for up to 16 values), then across warps through
//     shared memory;
//   * thread j < NS computes row j of the n x n prox product.
#include "common.cuh"

namespace hopf {

constexpr int CTA_THREADS = 256;        // nodes per thread NPT: 1 (N <= 256) or 2 (N <= 512)

// Warp reduce-scatter of 16 values: afterwards lane L holds the warp sum of
// value index ((L>>4)&1)*8 + ((L>>3)&1)*4 + ((L>>2)&1)*2 + ((L>>1)&1).
__device__ __forceinline__ float reduce_scatter16(float (&v)[16], int lane) {
    float a[8], b[4], c[2], d;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const bool hi = lane & 16;
        float send = hi ? v[k] : v[k + 8];
        float keep = hi ? v[k + 8] : v[k];
        a[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool hi = lane & 8;
        float send = hi ? a[k] : a[k + 4];
        float keep = hi ? a[k + 4] : a[k];
        b[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const bool hi = lane & 4;
        float send = hi ? b[k] : b[k + 2];
        float keep = hi ? b[k + 2] : b[k];
        c[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool hi = lane & 2;
        float send = hi ? c[0] : c[1];
        float keep = hi ? c[1] : c[0];
        d = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return d + __shfl_xor_sync(0xffffffffu, d, 1);
}

__device__ __forceinline__ int scatter_index(int lane) {
    return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

template <int NS, int MS, int CTA_NPT>
__global__ void __launch_bounds__(CTA_THREADS)
pdhg_cta_kernel(const float *__restrict__ inst, SolveParams prm, const float *__restrict__ x,
                float *__restrict__ phi, float *__restrict__ pstar, float *__restrict__ gap_out,
                int *__restrict__ iters, int *__restrict__ status, int *__restrict__ counter) {
    constexpr int KU = MS * NS;                   // used entries of a node row
    constexpr int NW = CTA_THREADS / 32;
    const int n = prm.n, N = prm.N;
    const InstanceLayout L = InstanceLayout::make(n, prm.m, N);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    __shared__ float s_S[NS * NS], s_M[NS * NS], s_V[NS * NS], s_U[NS * NS], s_lam[NS];
    __shared__ float s_pb[NS], s_x0[NS], s_v[NS], s_r[NS], s_red[NW][16], s_hs[NW];
    __shared__ int s_pt, s_slot, s_done;
    __shared__ float s_Dprev;

    for (int e = tid; e < NS * NS; e += CTA_THREADS) {
        int a = e / NS, b = e % NS;
        bool in = a < n && b < n;
        s_S[e] = in ? inst[L.S + a * n + b] : (a == b ? 1.f : 0.f);
        s_M[e] = in ? inst[L.M + a * n + b] : 0.f;
        s_V[e] = in ? inst[L.V + a * n + b] : 0.f;
        s_U[e] = in ? inst[L.U + a * n + b] : (a == b ? 1.f : 0.f);
    }
    for (int e = tid; e < NS; e += CTA_THREADS) s_lam[e] = e < n ? inst[L.lam + e] : 0.f;
    // this thread's node rows, kept in registers
    float kr[CTA_NPT][KU], wr[CTA_NPT];
#pragma unroll
    for (int k = 0; k < CTA_NPT; ++k) {
        const int i = tid + k * CTA_THREADS;
        const bool ok = i < N;
        wr[k] = ok ? inst[L.w + i] : 0.f;
#pragma unroll
        for (int c = 0; c < MS; ++c)
#pragma unroll
            for (int j = 0; j < NS; ++j)
                kr[k][c * NS + j] = (ok && j < n) ? inst[L.K + ((size_t)i * MS + c) * n + j] : 0.f;
    }
    const float gamma = inst[L.sc + SC_GAMMA];
    const bool accel = prm.accel != 0;
    const bool ball = prm.ctrl_kind == HOPF_BALL;
    const float tol = (float)prm.tol_gap;
    const int g = prm.gap_every;
    const int n_carry = *prm.in_count;
    __syncthreads();

    for (;;) {
        // ---- take a parked point
        if (tid == 0) {
            int nx = atomicAdd(counter, 1);
            s_slot = nx;
            s_pt = nx < n_carry ? prm.in_list[nx] : -1;
        }
        __syncthreads();
        const int pt = s_pt, slot = s_slot;
        if (pt < 0) break;
        const float *st = prm.in_st + (size_t)slot * CARRY_W;
        float p = 0.f;                            // thread j < NS owns p_j
        if (tid < NS) {
            p = st[tid];
            s_pb[tid] = st[16 + tid];
            s_x0[tid] = tid < n ? x[(size_t)pt * n + tid] : 0.f;
        }
        float tau = st[32], sigma = st[33];
        int it_pt = __float_as_int(st[34]);
        float y[CTA_NPT][MS];
        const float *cy = prm.in_y + (size_t)slot * N * MS;
#pragma unroll
        for (int k = 0; k < CTA_NPT; ++k) {
            const int i = tid + k * CTA_THREADS;
#pragma unroll
            for (int c = 0; c < MS; ++c) y[k][c] = i < N ? cy[(size_t)i * MS + c] : 0.f;
        }
        if (tid == 0) {
            s_done = 0;
            s_Dprev = 0.f;
        }
        bool have_D = false;
        __syncthreads();

        for (int wit = 1;; ++wit) {
            ++it_pt;
            const bool check = (wit % g) == 0;
            float pb[NS];
#pragma unroll
            for (int j = 0; j < NS; ++j) pb[j] = s_pb[j];
            float acc[16], hs = 0.f;
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0.f;
#pragma unroll
            for (int k = 0; k < CTA_NPT; ++k) {
                float u[MS], tn = 0.f, un = 0.f;
#pragma unroll
                for (int c = 0; c < MS; ++c) {
                    float t0 = 0.f, t1 = 0.f;
#pragma unroll
                    for (int j = 0; j < NS; j += 2) {
                        t0 = fmaf(kr[k][c * NS + j], pb[j], t0);
                        if (j + 1 < NS) t1 = fmaf(kr[k][c * NS + j + 1], pb[j + 1], t1);
                    }
                    const float t = t0 + t1;
                    tn = ball ? fmaf(t, t, tn) : tn + fabsf(t);
                    u[c] = fmaf(sigma, t, y[k][c]);
                    un = fmaf(u[c], u[c], un);
                }
                const float wi = wr[k];
                hs = fmaf(wi, ball ? sqrtf(tn) : tn, hs);
                if (ball) {
                    float scale = (un > wi * wi) ? wi * rsqrtf(un) : 1.f;
#pragma unroll
                    for (int c = 0; c < MS; ++c) u[c] *= scale;
                } else {
#pragma unroll
                    for (int c = 0; c < MS; ++c) u[c] = fminf(fmaxf(u[c], -wi), wi);
                }
#pragma unroll
                for (int c = 0; c < MS; ++c) {
                    y[k][c] = u[c];
#pragma unroll
                    for (int j = 0; j < NS; ++j) acc[j] = fmaf(kr[k][c * NS + j], u[c], acc[j]);
                }
            }
            // K^T y over the block
            const float part = reduce_scatter16(acc, lane);
            if ((lane & 1) == 0) {
                const int idx = scatter_index(lane);
                s_red[warp][idx] = part;
            }
            if (check) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) hs += __shfl_xor_sync(0xffffffffu, hs, o);
                if (lane == 0) s_hs[warp] = hs;
            }
            __syncthreads();
            float accj = 0.f;
            if (tid < NS) {
#pragma unroll
                for (int w = 0; w < NW; ++w) accj += s_red[w][tid];
            }
            if (check && tid == 0 && have_D) {
                // certificate at (pbar of the previous step, y of the previous step)
                float H = 0.f;
#pragma unroll
                for (int w = 0; w < NW; ++w) H += s_hs[w];
                float quad = 1.f;
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    float s = 0.f;
#pragma unroll
                    for (int b = 0; b < NS; ++b) s = fmaf(s_M[a * NS + b], pb[b], s);
                    quad = fmaf(pb[a], fmaf(0.25f, s, -s_x0[a]), quad);
                }
                const float Pc = quad + H, Dc = s_Dprev;
                const float gc = rel_gap(Pc, Dc);
                const bool bad = !isfinite(Pc) || !isfinite(Dc);
                const float scl = fmaxf(1.f, fmaxf(fabsf(Pc), fabsf(Dc)));
                const bool conv = gc + gap_allowance(quad, H, Dc, scl) <= tol;
                if (bad || conv || it_pt - 1 >= prm.max_iter) {
                    phi[pt] = -Pc;
                    gap_out[pt] = gc;
                    iters[pt] = it_pt - 1;
                    status[pt] = bad ? HOPF_NONFINITE : (conv ? HOPF_OK : HOPF_MAXITER);
                    s_done = 1;
                }
            }
            if (check) {
                __syncthreads();
                if (s_done) {
                    if (tid < n) pstar[(size_t)pt * n + tid] = s_pb[tid];
                    __syncthreads();
                    break;
                }
            }
            // prox of G, one row per thread j < NS
            if (tid < NS) s_v[tid] = fmaf(-tau, accj, fmaf(tau, s_x0[tid], p));
            __syncthreads();
            float th = 1.f, pn = 0.f;
            if (accel) {
                float z = 0.f;
                if (tid < NS) {
                    for (int b = 0; b < NS; ++b) z = fmaf(s_U[b * NS + tid], s_v[b], z);
                    z = __fdividef(z, fmaf(0.5f * tau, s_lam[tid], 1.f));
                }
                __syncthreads();
                if (tid < NS) s_v[tid] = z;
                __syncthreads();
                if (tid < NS)
                    for (int b = 0; b < NS; ++b) pn = fmaf(s_U[tid * NS + b], s_v[b], pn);
                th = rsqrtf(fmaf(2.f * gamma, tau, 1.f));
                tau *= th;
                sigma /= th;
            } else if (tid < NS) {
                for (int b = 0; b < NS; ++b) pn = fmaf(s_S[tid * NS + b], s_v[b], pn);
            }
            if (tid < NS) {
                s_pb[tid] = fmaf(th, pn - p, pn);
                p = pn;
            }
            if (((wit + 1) % g) == 0) {
                // D(y) = 1 - r^T V r with r = x0 - K^T y, for the next check
                if (tid < NS) s_r[tid] = s_x0[tid] - accj;
                __syncthreads();
                if (tid == 0) {
                    float dq = 1.f;
#pragma unroll
                    for (int a = 0; a < NS; ++a) {
                        float s = 0.f;
#pragma unroll
                        for (int b = 0; b < NS; ++b) s = fmaf(s_V[a * NS + b], s_r[b], s);
                        dq = fmaf(-s_r[a], s, dq);
                    }
                    s_Dprev = dq;
                }
                have_D = true;
            }
            __syncthreads();
        }
    }
}

cudaError_t launch_pdhg_cta(int NS, int m, int grid, cudaStream_t s, const float *inst, const SolveParams &prm,
                            const float *x, float *phi, float *pstar, float *gap, int *iters, int *status,
                            int *counter) {
    void (*fn)(const float *, SolveParams, const float *, float *, float *, float *, int *, int *, int *) = nullptr;
#define HOPF_CASE(NSV)                                                                               \
    case NSV:                                                                                        \
        if (prm.N <= CTA_THREADS) fn = (m == 1) ? pdhg_cta_kernel<NSV, 1, 1> : pdhg_cta_kernel<NSV, 2, 1>; \
        else fn = (m == 1) ? pdhg_cta_kernel<NSV, 1, 2> : pdhg_cta_kernel<NSV, 2, 2>;                 \
        break;
    switch (NS) {
        HOPF_CASE(2) HOPF_CASE(4) HOPF_CASE(6) HOPF_CASE(8)
        HOPF_CASE(10) HOPF_CASE(12) HOPF_CASE(14) HOPF_CASE(16)
        default: return cudaErrorInvalidValue;
    }
#undef HOPF_CASE
    fn<<<grid, CTA_THREADS, 0, s>>>(inst, prm, x, phi, pstar, gap, iters, status, counter);
    return cudaGetLastError();
}

}  // namespace hopf
