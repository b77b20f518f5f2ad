// Chambolle-Pock iteration (§III, Eq. 15 with theta = 1; prox of Eq. 22-23
// and Eq. 37) for large state dimensions (16 < n <= 256, m <= 16), one node
// table shared by every point, float32.
//
// The per-iteration work of a point is two products with the stacked table,
// K pbar (G = N m rows) and K^T y, i.e. 4 G n flops on 2 G n table entries.
// Warp-per-point reads the whole table from L2 for every point and iteration;
// here a persistent block keeps a tile of 32 or 64 point slots and streams
// node blocks of K through shared memory once per iteration for the whole
// tile, so each table entry read feeds 2 x (tile) fused multiply-adds.
//
// Block layout: 8 warps.  In the K pbar product warp w owns npt consecutive
// nodes of the node block (rw = npt mp rows of K) and lane l owns slots l and
// l + 32; the m dot products of a (node, slot) pair end in one thread, which
// then does the dual step and the projection onto w_i U in registers (ball:
// radial scaling, box: clipping).  In the K^T y product warp w owns the state
// quads q = w, w + 8, ... and accumulates them over all node blocks in
// registers.  The dual variables of the slots live in a per-block global
// buffer [row][slot] (coalesced across lanes); p and x0 of the slots in
// per-block buffers [state][slot]; pbar in shared memory.
//
// Certificate (every gap_every iterations): P at the pbar the dual step used
// (P = pbar^T M pbar / 4 + 1 - <x0, pbar> + sum_i w_i |K_i pbar|_*, the norm
// sum taken from the dual step's products) and the Fenchel dual D at the new
// feasible y, D = 1 - u^T V u with u = x0 - K^T y; both are bounds for any p
// and any feasible y, so phi lies in [-P, -D].  A point stops when
// (P - D)/max(1,|P|,|D|) plus the float rounding allowance is <= tol_gap.
// For large n the float32 evaluation of P and D (quadratic forms over n^2
// terms, K^T y over G rows, with cancellation when |phi| is large) can be off
// by about 1e-5 relative, so a point that passes in float32 is re-certified:
// P(pbar) and D(y) are evaluated once more in float64 from the float64 table
// (y shrunk by 4e-7 so that float32 rounding cannot leave w_i U).  Only a
// point whose float64 gap passes is accepted (phi = -P in float64); otherwise
// it iterates on with its float32 acceptance threshold halved.  The slot of an
// accepted point takes the next point from a global queue.
//
// Time-to-reach sign mode (prm.sign_mode): a point also stops once the sign
// of phi is certified, P < 0 (phi > 0) or D > 0 (phi < 0); a float32 margin of
// the slot's tolerance nominates it and the float64 evaluation decides.  P
// and D of every finished point go to Pout / Dout when given.
//
// Fixed-step rule (prm.fx_nk set): the table covers [0, t_max]; a slot uses
// the first fx_nk nodes of its point (the last weighted fx_wl) and its own
// dual step fx_sig; a block streams only the node blocks its slots need.
#include "common.cuh"

namespace hopf {

namespace {

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc))));
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NG>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(NG) : "memory"); }

__device__ __forceinline__ float comp(const float4 &v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

// one-off: zero-padded float32 copies of K ([chunks cr][n4], row i mp + c for
// node i and control component c), of the symmetric S, M, V and of the
// eigenvectors U of M and their transpose ([n][n4] each, contiguous from Sp)
__global__ void tile_pad_kernel(const float *__restrict__ inst, int n, int m, int N, TileGeom g,
                                float *__restrict__ Kp, float *__restrict__ Sp, float *__restrict__ Mp,
                                float *__restrict__ Vp) {
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    const long long nk = (long long)g.chunks * g.cr * g.n4;
    const long long nm = (long long)n * g.n4;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nk + 5 * nm; e += stride) {
        if (e < nk) {
            const long long row = e / g.n4;
            const int j = (int)(e % g.n4);
            const long long i = row / g.mp;
            const int c = (int)(row % g.mp);
            Kp[e] = (i < N && c < m && j < n) ? inst[L.K + (i * m + c) * n + j] : 0.f;
        } else {
            const long long f = e - nk;
            const int which = (int)(f / nm);
            const long long r = f % nm;
            const int b = (int)(r / g.n4), a = (int)(r % g.n4);
            float v = 0.f;
            if (a < n) {
                if (which == 4) v = inst[L.U + (long long)a * n + b];           // U^T
                else v = inst[(which == 0 ? L.S : which == 1 ? L.M : which == 2 ? L.V : L.U) + (long long)b * n + a];
            }
            Sp[(long long)which * nm + r] = v;
        }
    }
}

}  // namespace

__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < TILE_WARPS; ++w) t += red[w];
    return t;
}

template <int MP, int PPT>
__global__ void __launch_bounds__(TILE_WARPS * 32, 1)
pdhg_tile_kernel(const float *__restrict__ inst, const double *__restrict__ inst64, const float *__restrict__ Kp,
                 const float *__restrict__ Sp,
                 const float *__restrict__ Mp, const float *__restrict__ Vp, SolveParams prm,
                 const float *__restrict__ x, const float *__restrict__ p_init, float *__restrict__ phi,
                 float *__restrict__ pstar, float *__restrict__ gap_out, int *__restrict__ iters,
                 int *__restrict__ status, float *__restrict__ slot_p, float *__restrict__ slot_x,
                 float *__restrict__ slot_y, int *__restrict__ queue, int dbuf, float *__restrict__ Pout,
                 float *__restrict__ Dout) {
    constexpr int NPT = MP >= 8 ? 1 : 8 / MP;
    constexpr int RW = NPT * MP;
    constexpr int PT = 32 * PPT;
    constexpr int NQW = 8;                          // n <= 256: at most 8 quads per warp
    const int n = prm.n, m = prm.m, N = prm.N, P = prm.P;
    const TileGeom g = tile_geom(n, m, N, PPT);
    const int n4 = g.n4, nq = g.nq, CR = g.cr, NC = g.nc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    const float *wv = inst + L.w;
    const float *sc = inst + L.sc;
    const bool ball = prm.ctrl_kind == HOPF_BALL;

    if (sc[SC_ZERO] != 0.f) {
        // T = 0: phi = J_x(x) = x^T V x - 1 (V = W^-1), p* = 2 V x
        const float *V = inst + L.V;
        for (int k = blockIdx.x * blockDim.x + tid; k < P; k += gridDim.x * blockDim.x) {
            const float *xk = x + (long long)k * n;
            float J = -1.f;
            for (int a = 0; a < n; ++a) {
                float s = 0.f;
                for (int b = 0; b < n; ++b) s = fmaf(V[a * n + b], xk[b], s);
                pstar[(long long)k * n + a] = 2.f * s;
                J = fmaf(xk[a], s, J);
            }
            phi[k] = J;
            gap_out[k] = 0.f;
            iters[k] = 0;
            status[k] = HOPF_OK;
        }
        return;
    }
    const float gamma = sc[SC_GAMMA];
    const float *lam = inst + L.lam;
    const float *Up = Sp + 3LL * n * n4, *Utp = Sp + 4LL * n * n4;   // U and U^T, padded

    extern __shared__ float4 smem4[];
    float *Kbuf0 = reinterpret_cast<float *>(smem4);               // [max(cr, pt)][n4]
    float *Kbuf1 = Kbuf0 + (long long)(CR > PT ? CR : PT) * n4;    // [cr][n4] when double-buffered
    float *Pb = Kbuf1 + (dbuf ? (long long)CR * n4 : 0LL);         // [nq][pt][4]
    float *Ks = Kbuf0;
    float *VB = Pb + (long long)n4 * PT;                           // [n4][pt]
    float *Ys = VB + (long long)n4 * PT;                           // [cr][pt]
    float *Hs = Ys + (long long)CR * PT;                           // [pt]
    float *Qs = Hs + PT, *Ds = Qs + PT;
    __shared__ int sl_pt[PT], sl_cnt[PT], sl_fresh[PT], sl_done[PT];
    __shared__ float sl_tol[PT], sl_tau[PT], sl_sig[PT];
    __shared__ int s_check, s_active, s_verify, s_park, s_nch;
    __shared__ int sl_park[PT], sl_nk[PT];
    __shared__ float sl_wl[PT], sl_mg[PT];
    const bool fx = prm.fx_nk != nullptr;
    __shared__ double red[TILE_WARPS];

    float *ps = slot_p + (long long)blockIdx.x * n4 * PT;          // [n4][pt]
    float *xs = slot_x + (long long)blockIdx.x * n4 * PT;
    float *Yg = slot_y + (long long)blockIdx.x * g.chunks * CR * PT;  // [chunks cr][pt]
    auto pb_at = [&](int j, int s) -> float & { return Pb[((j >> 2) * PT + s) * 4 + (j & 3)]; };

    // the queue walks points 0..P-1, or list[0 .. *list_count) when given
    const int Pq = prm.list ? *prm.list_count : P;
    auto take = [&]() -> int {
        for (;;) {
            const int q = atomicAdd(queue, 1);
            if (q >= Pq) return -1;
            const int k = prm.list ? prm.list[q] : q;
            if (!fx || prm.fx_nk[k] >= 0) return k;     // out-of-range horizons are skipped
        }
    };
    // per-slot node count, last weight and dual step of its point
    auto slot_rule = [&](int s) {
        const int k = sl_pt[s];
        const bool f = fx && k >= 0;
        sl_nk[s] = f ? prm.fx_nk[k] : N;
        sl_wl[s] = f ? (float)prm.fx_wl[k] : 0.f;
        sl_sig[s] = f ? (float)prm.fx_sig[k] : sc[SC_SIGMA];
    };
    // fill every slot from the queue
    if (tid < PT) {
        sl_pt[tid] = take();
        sl_cnt[tid] = 0;
        sl_fresh[tid] = 1;
        sl_done[tid] = 0;
        sl_tol[tid] = (float)prm.tol_gap;
        sl_mg[tid] = (float)prm.tol_gap;
        sl_tau[tid] = (float)prm.tau;
        slot_rule(tid);
    }
    __syncthreads();
    for (int e = tid; e < n4 * PT; e += blockDim.x) {
        const int j = e / PT, s = e % PT;
        const int k = sl_pt[s];
        float xv = 0.f, pv = 0.f;
        if (k >= 0 && j < n) {
            xv = x[(long long)k * n + j];
            pv = prm.warm ? p_init[(long long)k * n + j] : xv;
        }
        xs[j * PT + s] = xv;
        ps[j * PT + s] = pv;
        pb_at(j, s) = pv;
    }
    __syncthreads();

    for (int git = 1;; ++git) {
        if (tid < PT) {
            Hs[tid] = 0.f;
            Qs[tid] = 0.f;
            Ds[tid] = 0.f;
            if (sl_pt[tid] >= 0) ++sl_cnt[tid];
        }
        __syncthreads();
        if (tid == 0) {
            int chk = (git % prm.gap_every) == 0, act = 0, nmax = 0;
            for (int s = 0; s < PT; ++s)
                if (sl_pt[s] >= 0) {
                    ++act;
                    if (sl_cnt[s] > prm.max_iter) chk = 1;
                    nmax = max(nmax, sl_nk[s]);
                }
            s_check = chk;
            s_active = act;
            s_nch = fx ? (nmax + NC - 1) / NC : g.chunks;      // node blocks the slots need
        }
        __syncthreads();
        if (s_active == 0) break;
        const bool check = s_check != 0;
        const int nch = s_nch;

        float4 R[PPT][NQW];
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp)
#pragma unroll
            for (int k = 0; k < NQW; ++k) R[pp][k] = make_float4(0.f, 0.f, 0.f, 0.f);
        float hpart[PPT];
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp) hpart[pp] = 0.f;

        // node block c of K into shared memory (asynchronous copies; with two
        // buffers block c + 1 is in flight while block c is used)
        auto load_block = [&](int c, float *dstf) {
            const float4 *src = reinterpret_cast<const float4 *>(Kp + (long long)c * CR * n4);
            float4 *dst = reinterpret_cast<float4 *>(dstf);
            for (int e = tid; e < CR * nq; e += blockDim.x) cp_async16(dst + e, src + e);
            cp_async_commit();
        };
        if (dbuf) load_block(0, Kbuf0);
        for (int c = 0; c < nch; ++c) {
            if (dbuf) {
                Ks = (c & 1) ? Kbuf1 : Kbuf0;
                if (c + 1 < nch) {
                    load_block(c + 1, (c & 1) ? Kbuf0 : Kbuf1);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
            } else {
                load_block(c, Kbuf0);
                cp_async_wait<0>();
            }
            __syncthreads();
            // this block's dual variables, loaded before the products so the
            // global-memory latency overlaps them
            float ypre[PPT][RW];
#pragma unroll
            for (int t = 0; t < NPT; ++t) {
                const int i = c * NC + warp * NPT + t;
                const bool node_ok = i < N;
                const long long grow = (long long)c * CR + warp * RW + t * MP;
#pragma unroll
                for (int pp = 0; pp < PPT; ++pp) {
                    const int s = lane + 32 * pp;
                    const bool ld = node_ok && i < sl_nk[s] && sl_pt[s] >= 0 && !sl_fresh[s];
#pragma unroll
                    for (int cc = 0; cc < MP; ++cc) ypre[pp][t * MP + cc] = ld ? Yg[(grow + cc) * PT + s] : 0.f;
                }
            }
            // K pbar for this warp's rows and this lane's slots
            float acc[PPT][RW];
#pragma unroll
            for (int pp = 0; pp < PPT; ++pp)
#pragma unroll
                for (int r = 0; r < RW; ++r) acc[pp][r] = 0.f;
            {
                const float4 *Kw = reinterpret_cast<const float4 *>(Ks) + (long long)warp * RW * nq;
                const float4 *P4 = reinterpret_cast<const float4 *>(Pb);
#pragma unroll 2
                for (int q = 0; q < nq; ++q) {
                    float4 pv[PPT];
#pragma unroll
                    for (int pp = 0; pp < PPT; ++pp) pv[pp] = P4[q * PT + lane + 32 * pp];
#pragma unroll
                    for (int r = 0; r < RW; ++r) {
                        const float4 kv = Kw[r * nq + q];
#pragma unroll
                        for (int pp = 0; pp < PPT; ++pp) acc[pp][r] = dot4(kv, pv[pp], acc[pp][r]);
                    }
                }
            }
            // dual step and projection, one (node, slot) pair per thread
#pragma unroll
            for (int t = 0; t < NPT; ++t) {
                const int i = c * NC + warp * NPT + t;
                const bool node_ok = i < N;
                const float wtab = node_ok ? __ldg(wv + i) : 0.f;
                const int row = warp * RW + t * MP;
                const long long grow = (long long)c * CR + row;
#pragma unroll
                for (int pp = 0; pp < PPT; ++pp) {
                    const int s = lane + 32 * pp;
                    float yn[MP];
                    if (node_ok && sl_pt[s] >= 0) {
                        // weight of node i for this slot's horizon
                        const int nks = sl_nk[s];
                        const float wi = !fx ? wtab : (i < nks - 1 ? wtab : (i == nks - 1 ? sl_wl[s] : 0.f));
                        float nt = 0.f;
#pragma unroll
                        for (int cc = 0; cc < MP; ++cc) {
                            const float z = acc[pp][t * MP + cc];
                            nt += ball ? z * z : fabsf(z);
                        }
                        if (check) hpart[pp] = fmaf(wi, ball ? sqrtf(nt) : nt, hpart[pp]);
                        float yo[MP];
                        if (!sl_fresh[s]) {
#pragma unroll
                            for (int cc = 0; cc < MP; ++cc) yo[cc] = ypre[pp][t * MP + cc];
                        } else if (!prm.warm) {     // y0 = K p0 (§VI), unprojected
#pragma unroll
                            for (int cc = 0; cc < MP; ++cc) yo[cc] = acc[pp][t * MP + cc];
                        } else {                    // y0 = w_i argmax_{c in U} <c, K_i p0>
                            const float scl = nt > 0.f ? wi * rsqrtf(nt) : 0.f;
#pragma unroll
                            for (int cc = 0; cc < MP; ++cc) {
                                const float z = acc[pp][t * MP + cc];
                                yo[cc] = ball ? z * scl : (cc < m ? (z >= 0.f ? wi : -wi) : 0.f);
                            }
                        }
                        float nu = 0.f;
                        const float sigma = sl_sig[s];
#pragma unroll
                        for (int cc = 0; cc < MP; ++cc) {
                            yn[cc] = fmaf(sigma, acc[pp][t * MP + cc], yo[cc]);
                            nu = fmaf(yn[cc], yn[cc], nu);
                        }
                        if (ball) {
                            const float scl = (nu > wi * wi) ? wi * rsqrtf(nu) : 1.f;
#pragma unroll
                            for (int cc = 0; cc < MP; ++cc) yn[cc] *= scl;
                        } else {
#pragma unroll
                            for (int cc = 0; cc < MP; ++cc) yn[cc] = cc < m ? fminf(fmaxf(yn[cc], -wi), wi) : 0.f;
                        }
#pragma unroll
                        for (int cc = 0; cc < MP; ++cc) Yg[(grow + cc) * PT + s] = yn[cc];
                    } else {
#pragma unroll
                        for (int cc = 0; cc < MP; ++cc) yn[cc] = 0.f;
                    }
#pragma unroll
                    for (int cc = 0; cc < MP; ++cc) Ys[(row + cc) * PT + s] = yn[cc];
                }
            }
            __syncthreads();
            // K^T y over this node block: warp w, quads w, w + 8, ...
            {
                const float4 *K4 = reinterpret_cast<const float4 *>(Ks);
#pragma unroll 2
                for (int r = 0; r < CR; ++r) {
                    float yv[PPT];
#pragma unroll
                    for (int pp = 0; pp < PPT; ++pp) yv[pp] = Ys[r * PT + lane + 32 * pp];
#pragma unroll
                    for (int k = 0; k < NQW; ++k) {
                        const int q = warp + 8 * k;
                        if (q < nq) {
                            const float4 kv = K4[r * nq + q];
#pragma unroll
                            for (int pp = 0; pp < PPT; ++pp) {
                                R[pp][k].x = fmaf(kv.x, yv[pp], R[pp][k].x);
                                R[pp][k].y = fmaf(kv.y, yv[pp], R[pp][k].y);
                                R[pp][k].z = fmaf(kv.z, yv[pp], R[pp][k].z);
                                R[pp][k].w = fmaf(kv.w, yv[pp], R[pp][k].w);
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (check) {
#pragma unroll
            for (int pp = 0; pp < PPT; ++pp) atomicAdd(&Hs[lane + 32 * pp], hpart[pp]);
        }
        // v = p - tau K^T y + tau x0 (argument of the prox of Eq. 37) and, on
        // certificate iterations, u = x0 - K^T y (in the first K block buffer,
        // free: no copy is in flight after the last block)
        float *UB = Kbuf0;
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp) {
            const int s = lane + 32 * pp;
            const float tau = sl_tau[s];
#pragma unroll
            for (int k = 0; k < NQW; ++k) {
                const int q = warp + 8 * k;
                if (q < nq) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j = 4 * q + e;
                        const float xv = xs[j * PT + s], pv = ps[j * PT + s], r = comp(R[pp][k], e);
                        VB[j * PT + s] = fmaf(tau, xv - r, pv);
                        if (check) UB[j * PT + s] = xv - r;
                    }
                }
            }
        }
        __syncthreads();
        if (check) {
            // pbar^T (M pbar / 4 - x0) and u^T V u, this warp's share of the state
            float qp[PPT], dp[PPT];
#pragma unroll
            for (int pp = 0; pp < PPT; ++pp) qp[pp] = dp[pp] = 0.f;
#pragma unroll
            for (int k = 0; k < NQW; ++k) {
                const int q = warp + 8 * k;
                if (q >= nq) break;
                float4 mq[PPT], vq[PPT];
#pragma unroll
                for (int pp = 0; pp < PPT; ++pp) mq[pp] = vq[pp] = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int b = 0; b < n; ++b) {
                    const float4 m4 = __ldg(reinterpret_cast<const float4 *>(Mp + (long long)b * n4) + q);
                    const float4 v4 = __ldg(reinterpret_cast<const float4 *>(Vp + (long long)b * n4) + q);
#pragma unroll
                    for (int pp = 0; pp < PPT; ++pp) {
                        const int s = lane + 32 * pp;
                        const float pb = pb_at(b, s), uv = UB[b * PT + s];
                        mq[pp].x = fmaf(m4.x, pb, mq[pp].x);
                        mq[pp].y = fmaf(m4.y, pb, mq[pp].y);
                        mq[pp].z = fmaf(m4.z, pb, mq[pp].z);
                        mq[pp].w = fmaf(m4.w, pb, mq[pp].w);
                        vq[pp].x = fmaf(v4.x, uv, vq[pp].x);
                        vq[pp].y = fmaf(v4.y, uv, vq[pp].y);
                        vq[pp].z = fmaf(v4.z, uv, vq[pp].z);
                        vq[pp].w = fmaf(v4.w, uv, vq[pp].w);
                    }
                }
#pragma unroll
                for (int pp = 0; pp < PPT; ++pp) {
                    const int s = lane + 32 * pp;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int a = 4 * q + e;
                        qp[pp] = fmaf(pb_at(a, s), fmaf(0.25f, comp(mq[pp], e), -xs[a * PT + s]), qp[pp]);
                        dp[pp] = fmaf(UB[a * PT + s], comp(vq[pp], e), dp[pp]);
                    }
                }
            }
#pragma unroll
            for (int pp = 0; pp < PPT; ++pp) {
                atomicAdd(&Qs[lane + 32 * pp], qp[pp]);
                atomicAdd(&Ds[lane + 32 * pp], dp[pp]);
            }
            __syncthreads();
        }
        // stop decisions, one thread per slot
        if (tid < PT) {
            const int s = tid, k = sl_pt[s];
            sl_done[s] = 0;
            if (k >= 0) {
                const int cnt = sl_cnt[s];
                if (check && (cnt >= 2 || cnt > prm.max_iter)) {
                    const float quad = Qs[s] + 1.f, H = Hs[s];
                    const float Pv = quad + H, Dv = 1.f - Ds[s];
                    const float gp = rel_gap(Pv, Dv);
                    const float scl = fmaxf(1.f, fmaxf(fabsf(Pv), fabsf(Dv)));
                    int st = -1;
                    if (!isfinite(Pv) || !isfinite(Dv)) st = HOPF_NONFINITE;
                    else if (gp + gap_allowance(quad, H, Dv, scl) <= sl_tol[s]) st = HOPF_OK;
                    else if (prm.sign_mode && (-Pv > sl_mg[s] * scl || Dv > sl_mg[s] * scl)) st = HOPF_OK;
                    else if (cnt > prm.max_iter) st = HOPF_MAXITER;
                    if (st == HOPF_OK) {
                        sl_done[s] = 2;             // float64 re-certification below
                    } else if (st >= 0) {
                        phi[k] = -Pv;
                        gap_out[k] = gp;
                        iters[k] = cnt - 1;
                        status[k] = st;
                        if (Pout) Pout[k] = Pv;
                        if (Dout) Dout[k] = Dv;
                        sl_done[s] = 1;
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            int v = 0;
            for (int s = 0; s < PT; ++s) v |= sl_done[s] == 2;
            s_verify = v;
        }
        __syncthreads();
        if (s_verify) {
            const double *K64 = inst64 + L.K, *M64 = inst64 + L.M, *V64 = inst64 + L.V, *w64 = inst64 + L.w;
            double *ub = reinterpret_cast<double *>(Ys);            // n doubles (dual block is free here)
            for (int s = 0; s < PT; ++s) {
                if (sl_done[s] != 2) continue;                        // uniform: shared memory
                const int nks = sl_nk[s];
                const double wl64 = fx ? prm.fx_wl[sl_pt[s]] : 0.0;
                // H = sum_i w_i |K_i pbar|_*
                double hp = 0.0;
                for (int i = tid; i < nks; i += blockDim.x) {
                    double nt = 0.0;
                    for (int c = 0; c < m; ++c) {
                        const double *Kr = K64 + ((long long)i * m + c) * n;
                        double z = 0.0;
                        for (int j = 0; j < n; ++j) z = fma(Kr[j], (double)pb_at(j, s), z);
                        nt += ball ? z * z : fabs(z);
                    }
                    hp = fma((fx && i == nks - 1) ? wl64 : w64[i], ball ? sqrt(nt) : nt, hp);
                }
                const double H64 = block_sum(hp, red);
                // u = x0 - K^T y (y shrunk into w_i U), then D = 1 - u^T V u
                for (int j = tid; j < n; j += blockDim.x) {
                    double r = 0.0;
                    for (int i = 0; i < nks; ++i)
                        for (int c = 0; c < m; ++c)
                            r = fma(K64[((long long)i * m + c) * n + j],
                                    (double)Yg[((long long)i * MP + c) * PT + s], r);
                    ub[j] = (double)xs[j * PT + s] - (1.0 - 4e-7) * r;
                }
                __syncthreads();
                double qp = 0.0, dp = 0.0;
                for (int a = tid; a < n; a += blockDim.x) {
                    double mq = 0.0, vq = 0.0;
                    for (int b = 0; b < n; ++b) {
                        mq = fma(M64[(long long)a * n + b], (double)pb_at(b, s), mq);
                        vq = fma(V64[(long long)a * n + b], ub[b], vq);
                    }
                    qp = fma((double)pb_at(a, s), 0.25 * mq - (double)xs[a * PT + s], qp);
                    dp = fma(ub[a], vq, dp);
                }
                const double quad64 = block_sum(qp, red) + 1.0;
                const double D64 = 1.0 - block_sum(dp, red);
                const double P64 = quad64 + H64;
                const double g64 = rel_gap(P64, D64);
                const double scl = fmax(1.0, fmax(fabs(P64), fabs(D64)));
                if (tid == 0) {
                    if (g64 + gap_allowance(quad64, H64, D64, scl) <= prm.tol_gap ||
                        (prm.sign_mode && (P64 < 0.0 || D64 > 0.0))) {
                        const int k = sl_pt[s];
                        phi[k] = (float)(-P64);
                        gap_out[k] = (float)g64;
                        iters[k] = sl_cnt[s] - 1;
                        status[k] = HOPF_OK;
                        if (Pout) Pout[k] = (float)P64;
                        if (Dout) Dout[k] = (float)D64;
                        sl_done[s] = 1;
                    } else {
                        sl_done[s] = 0;
                        sl_tol[s] *= 0.5f;           // stricter float32 gap,
                        sl_mg[s] *= 2.f;             // wider float32 sign margin
                    }
                }
                __syncthreads();
            }
        }
        // p* of finished slots (the pbar of the certificate), then the prox
        // S v of Eq. 37 for every slot
        for (int e = tid; e < n * PT; e += blockDim.x) {
            const int s = e / n, a = e % n;
            if (sl_done[s]) pstar[(long long)sl_pt[s] * n + a] = pb_at(a, s);
        }
        float4 pn[PPT][NQW];
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp)
#pragma unroll
            for (int k = 0; k < NQW; ++k) pn[pp][k] = make_float4(0.f, 0.f, 0.f, 0.f);
        // plain step: p_new = S v.  Accelerated step (tau changes every
        // iteration): p_new = U diag(1 / (1 + tau lam / 2)) U^T v, the product
        // U^T v going through the u buffer (free after the certificate).
        const float *P1 = prm.accel ? Up : Sp;
#pragma unroll
        for (int k = 0; k < NQW; ++k) {
            const int q = warp + 8 * k;
            if (q >= nq) break;
            for (int b = 0; b < n; ++b) {
                const float4 s4 = __ldg(reinterpret_cast<const float4 *>(P1 + (long long)b * n4) + q);
#pragma unroll
                for (int pp = 0; pp < PPT; ++pp) {
                    const float v = VB[b * PT + lane + 32 * pp];
                    pn[pp][k].x = fmaf(s4.x, v, pn[pp][k].x);
                    pn[pp][k].y = fmaf(s4.y, v, pn[pp][k].y);
                    pn[pp][k].z = fmaf(s4.z, v, pn[pp][k].z);
                    pn[pp][k].w = fmaf(s4.w, v, pn[pp][k].w);
                }
            }
        }
        if (prm.accel) {
            __syncthreads();                       // every product of v done before U^T v is stored
#pragma unroll
            for (int pp = 0; pp < PPT; ++pp) {
                const int s = lane + 32 * pp;
                const float ht = 0.5f * sl_tau[s];
#pragma unroll
                for (int k = 0; k < NQW; ++k) {
                    const int q = warp + 8 * k;
                    if (q < nq) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int j = 4 * q + e;
                            UB[j * PT + s] = j < n ? comp(pn[pp][k], e) / fmaf(ht, __ldg(lam + j), 1.f) : 0.f;
                        }
                    }
                    pn[pp][k] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < NQW; ++k) {
                const int q = warp + 8 * k;
                if (q >= nq) break;
                for (int b = 0; b < n; ++b) {
                    const float4 s4 = __ldg(reinterpret_cast<const float4 *>(Utp + (long long)b * n4) + q);
#pragma unroll
                    for (int pp = 0; pp < PPT; ++pp) {
                        const float v = UB[b * PT + lane + 32 * pp];
                        pn[pp][k].x = fmaf(s4.x, v, pn[pp][k].x);
                        pn[pp][k].y = fmaf(s4.y, v, pn[pp][k].y);
                        pn[pp][k].z = fmaf(s4.z, v, pn[pp][k].z);
                        pn[pp][k].w = fmaf(s4.w, v, pn[pp][k].w);
                    }
                }
            }
        }
        __syncthreads();
        // p <- S v, pbar <- 2 p_new - p_old for the slots that go on
#pragma unroll
        for (int pp = 0; pp < PPT; ++pp) {
            const int s = lane + 32 * pp;
            if (sl_pt[s] < 0 || sl_done[s]) continue;
            // theta = 1 (Eq. 15) or 1 / sqrt(1 + 2 gamma tau) (accelerated)
            const float th = prm.accel ? rsqrtf(fmaf(2.f * gamma, sl_tau[s], 1.f)) : 1.f;
#pragma unroll
            for (int k = 0; k < NQW; ++k) {
                const int q = warp + 8 * k;
                if (q < nq) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j = 4 * q + e;
                        const float pnew = comp(pn[pp][k], e);
                        const float pold = ps[j * PT + s];
                        ps[j * PT + s] = pnew;
                        pb_at(j, s) = fmaf(th, pnew - pold, pnew);
                    }
                }
            }
        }
        __syncthreads();
        // finished slots take the next point
        if (tid < PT) {
            const int s = tid;
            if (sl_done[s]) {
                sl_pt[s] = take();
                sl_cnt[s] = 0;
                sl_fresh[s] = 1;
                sl_tol[s] = (float)prm.tol_gap;
                sl_mg[s] = (float)prm.tol_gap;
                sl_tau[s] = (float)prm.tau;
                slot_rule(s);
            } else {
                sl_fresh[s] = 0;
                if (prm.accel && sl_pt[s] >= 0) {
                    const float th = rsqrtf(fmaf(2.f * gamma, sl_tau[s], 1.f));
                    sl_tau[s] *= th;
                    sl_sig[s] /= th;
                }
            }
        }
        __syncthreads();
        for (int e = tid; e < n4 * PT; e += blockDim.x) {
            const int j = e / PT, s = e % PT;
            if (!sl_done[s]) continue;
            const int k = sl_pt[s];
            float xv = 0.f, pv = 0.f;
            if (k >= 0 && j < n) {
                xv = x[(long long)k * n + j];
                pv = prm.warm ? p_init[(long long)k * n + j] : xv;
            }
            xs[j * PT + s] = xv;
            ps[j * PT + s] = pv;
            pb_at(j, s) = pv;
        }
        __syncthreads();
        // drain: with the queue empty, a block down to a quarter of its slots
        // costs as much per iteration as a full one.  It parks the points it
        // still holds (pbar, p, step sizes, counts; the dual rows stay in this
        // block's buffer) for the one-block-per-point tail kernel and leaves.
        if (prm.carry_cap > 0) {
            if (tid == 0) {
                int act = 0, fresh = 0;
                for (int s = 0; s < PT; ++s)
                    if (sl_pt[s] >= 0) {
                        ++act;
                        fresh |= sl_fresh[s];
                    }
                const int q = *reinterpret_cast<volatile int *>(queue);
                s_park = (act > 0 && !fresh && q >= Pq && 4 * act <= PT) ? 1 : 0;
            }
            __syncthreads();
            if (s_park) {
                const int CW = 2 * n4 + 4;
                if (tid < PT) {
                    const int s = tid;
                    sl_park[s] = -1;
                    if (sl_pt[s] >= 0) {
                        const int e = atomicAdd(prm.out_count, 1);
                        sl_park[s] = e;
                        prm.out_list[2 * e] = sl_pt[s];
                        prm.out_list[2 * e + 1] = blockIdx.x * PT + s;
                        float *st = prm.out_st + (long long)e * CW + 2 * n4;
                        st[0] = sl_tau[s];
                        st[1] = sl_sig[s];
                        st[2] = (float)sl_cnt[s];
                        st[3] = sl_tol[s];
                    }
                }
                __syncthreads();
                for (int e = tid; e < n4 * PT; e += blockDim.x) {
                    const int j = e / PT, s = e % PT;
                    const int slot = sl_park[s];
                    if (slot < 0) continue;
                    prm.out_st[(long long)slot * CW + j] = pb_at(j, s);
                    prm.out_st[(long long)slot * CW + n4 + j] = ps[j * PT + s];
                }
                return;
            }
        }
    }
}

// Tail of the tiled solve: one 256-thread block per parked point, the same
// iteration (Eq. 15 or the accelerated steps) with the node table read from
// L2 (the padded float32 copy the tiled kernel used) instead of shared memory.
// A point alone on an SM then needs about 2 x (rows x n4 x 4 B) of L2 reads
// per iteration instead of a whole tile's arithmetic.  Its dual variables
// come from the tiled kernel's per-block buffer and stay in shared memory;
// the certificate and the float64 re-certification are the tiled kernel's.
__global__ void __launch_bounds__(256)
pdhg_tile_tail_kernel(const float *__restrict__ inst, const double *__restrict__ inst64,
                      const float *__restrict__ Kp, const float *__restrict__ Sp, SolveParams prm, int ppt,
                      const float *__restrict__ x, float *__restrict__ phi, float *__restrict__ pstar,
                      float *__restrict__ gap_out, int *__restrict__ iters, int *__restrict__ status,
                      const float *__restrict__ slot_y, int *__restrict__ queue2, float *__restrict__ Pout,
                      float *__restrict__ Dout) {
    const int n = prm.n, m = prm.m, N = prm.N;
    const TileGeom g = tile_geom(n, m, N, ppt);
    const int n4 = g.n4, nq = g.nq, MPd = g.mp, PT = g.pt;
    const int G = g.chunks * g.cr;                    // padded rows of the table
    const int CW = 2 * n4 + 4;
    const int tid = threadIdx.x, nt = blockDim.x;
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    const float *wv = inst + L.w;
    const float gamma = inst[L.sc + SC_GAMMA];
    const float *lam = inst + L.lam;
    const float *Mp = Sp + (long long)n * n4, *Vp = Sp + 2LL * n * n4;
    const float *Up = Sp + 3LL * n * n4, *Utp = Sp + 4LL * n * n4;
    const bool ball = prm.ctrl_kind == HOPF_BALL;
    extern __shared__ float4 tsm4[];
    float *pb = reinterpret_cast<float *>(tsm4);       // [n4] each
    float *pp = pb + n4, *x0 = pp + n4, *vb = x0 + n4, *ub = vb + n4;
    float *ys = ub + n4;                                // [G]
    __shared__ double red[TILE_WARPS];
    __shared__ float fred[3][TILE_WARPS];
    __shared__ int s_e;
    auto fsum3 = [&](float a, float b, float c, float &A, float &B, float &C) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        __syncthreads();
        if ((tid & 31) == 0) {
            fred[0][tid >> 5] = a;
            fred[1][tid >> 5] = b;
            fred[2][tid >> 5] = c;
        }
        __syncthreads();
        A = B = C = 0.f;
        for (int w = 0; w < TILE_WARPS; ++w) {
            A += fred[0][w];
            B += fred[1][w];
            C += fred[2][w];
        }
    };
    const int total = *prm.out_count;
    for (;;) {
        if (tid == 0) s_e = atomicAdd(queue2, 1);
        __syncthreads();
        const int e = s_e;
        __syncthreads();
        if (e >= total) break;
        const int k = prm.out_list[2 * e], loc = prm.out_list[2 * e + 1];
        const float *Yp = slot_y + (long long)(loc / PT) * G * PT + (loc % PT);
        const float *st = prm.out_st + (long long)e * CW;
        // node count and last weight of this point's horizon (fixed-step rule)
        const int nkv = prm.fx_nk ? prm.fx_nk[k] : N;
        const int Gk = nkv * MPd;                      // table rows in use
        const double wl64 = prm.fx_nk ? prm.fx_wl[k] : 0.0;
        auto wt = [&](int i) -> float {
            return (prm.fx_nk && i == nkv - 1) ? (float)wl64 : __ldg(wv + i);
        };
        for (int j = tid; j < n4; j += nt) {
            pb[j] = st[j];
            pp[j] = st[n4 + j];
            x0[j] = j < n ? x[(long long)k * n + j] : 0.f;
        }
        for (int r = tid; r < G; r += nt) ys[r] = r < Gk ? Yp[(long long)r * PT] : 0.f;
        float tau = st[2 * n4], sigma = st[2 * n4 + 1], tol = st[2 * n4 + 3];
        float mg = (float)prm.tol_gap * ((float)prm.tol_gap / fmaxf(tol, 1e-30f));   // sign margin: doubles as tol halves
        int cnt = (int)st[2 * n4 + 2];
        __syncthreads();
        for (;;) {
            ++cnt;
            const bool check = (cnt % prm.gap_every) == 0 || cnt > prm.max_iter;
            // dual step, threads over nodes
            float hp = 0.f;
            for (int i = tid; i < nkv; i += nt) {
                const float wi = wt(i);
                float z[16];
                float nz = 0.f;
                for (int c = 0; c < m; ++c) {
                    const float4 *Kr = reinterpret_cast<const float4 *>(Kp + ((long long)i * MPd + c) * n4);
                    const float4 *P4 = reinterpret_cast<const float4 *>(pb);
                    float a = 0.f;
                    for (int q = 0; q < nq; ++q) a = dot4(__ldg(Kr + q), P4[q], a);
                    z[c] = a;
                    nz += ball ? a * a : fabsf(a);
                }
                if (check) hp = fmaf(wi, ball ? sqrtf(nz) : nz, hp);
                float nu = 0.f;
                for (int c = 0; c < m; ++c) {
                    const float v = fmaf(sigma, z[c], ys[i * MPd + c]);
                    z[c] = v;
                    nu = fmaf(v, v, nu);
                }
                const float scl = (ball && nu > wi * wi) ? wi * rsqrtf(nu) : 1.f;
                for (int c = 0; c < m; ++c) ys[i * MPd + c] = ball ? z[c] * scl : fminf(fmaxf(z[c], -wi), wi);
            }
            __syncthreads();
            // K^T y, threads over state components
            for (int j = tid; j < n4; j += nt) {
                float r = 0.f;
                for (int row = 0; row < Gk; ++row) r = fmaf(__ldg(Kp + (long long)row * n4 + j), ys[row], r);
                vb[j] = fmaf(tau, x0[j] - r, pp[j]);
                ub[j] = x0[j] - r;
            }
            __syncthreads();
            bool done = false;
            if (check) {
                float qp = 0.f, dp = 0.f;
                for (int a = tid; a < n; a += nt) {
                    float mq = 0.f, vq = 0.f;
                    for (int b = 0; b < n; ++b) {
                        mq = fmaf(__ldg(Mp + (long long)b * n4 + a), pb[b], mq);
                        vq = fmaf(__ldg(Vp + (long long)b * n4 + a), ub[b], vq);
                    }
                    qp = fmaf(pb[a], fmaf(0.25f, mq, -x0[a]), qp);
                    dp = fmaf(ub[a], vq, dp);
                }
                float H, Q, Dd;
                fsum3(hp, qp, dp, H, Q, Dd);
                const float quad = Q + 1.f, Pv = quad + H, Dv = 1.f - Dd;
                const float gp = rel_gap(Pv, Dv);
                const float scl = fmaxf(1.f, fmaxf(fabsf(Pv), fabsf(Dv)));
                int stt = -1;
                if (!isfinite(Pv) || !isfinite(Dv)) stt = HOPF_NONFINITE;
                else if (gp + gap_allowance(quad, H, Dv, scl) <= tol) stt = HOPF_OK;
                else if (prm.sign_mode && (-Pv > mg * scl || Dv > mg * scl)) stt = HOPF_OK;
                else if (cnt > prm.max_iter) stt = HOPF_MAXITER;
                if (stt == HOPF_OK) {
                    // float64 re-certification
                    const double *K64 = inst64 + L.K, *M64 = inst64 + L.M, *V64 = inst64 + L.V;
                    const double *w64 = inst64 + L.w;
                    double h64 = 0.0;
                    for (int i = tid; i < nkv; i += nt) {
                        double nz = 0.0;
                        for (int c = 0; c < m; ++c) {
                            const double *Kr = K64 + ((long long)i * m + c) * n;
                            double z = 0.0;
                            for (int j = 0; j < n; ++j) z = fma(Kr[j], (double)pb[j], z);
                            nz += ball ? z * z : fabs(z);
                        }
                        h64 = fma((prm.fx_nk && i == nkv - 1) ? wl64 : w64[i], ball ? sqrt(nz) : nz, h64);
                    }
                    const double H64 = block_sum(h64, red);
                    double q64 = 0.0, d64 = 0.0;
                    // u = x0 - K^T (shrunk y) in float64, one component per thread, kept
                    // after the dual rows in shared memory
                    for (int j = tid; j < n; j += nt) {
                        double r = 0.0;
                        for (int i = 0; i < nkv; ++i)
                            for (int c = 0; c < m; ++c)
                                r = fma(K64[((long long)i * m + c) * n + j], (double)ys[i * MPd + c], r);
                        reinterpret_cast<double *>(ys + G)[j] = (double)x0[j] - (1.0 - 4e-7) * r;
                    }
                    __syncthreads();
                    const double *u64s = reinterpret_cast<const double *>(ys + G);
                    for (int a = tid; a < n; a += nt) {
                        double mq = 0.0, vq = 0.0;
                        for (int b = 0; b < n; ++b) {
                            mq = fma(M64[(long long)a * n + b], (double)pb[b], mq);
                            vq = fma(V64[(long long)a * n + b], u64s[b], vq);
                        }
                        q64 = fma((double)pb[a], 0.25 * mq - (double)x0[a], q64);
                        d64 = fma(u64s[a], vq, d64);
                    }
                    const double quad64 = block_sum(q64, red) + 1.0;
                    const double D64 = 1.0 - block_sum(d64, red);
                    const double P64 = quad64 + H64;
                    const double g64 = rel_gap(P64, D64);
                    const double s64 = fmax(1.0, fmax(fabs(P64), fabs(D64)));
                    if (g64 + gap_allowance(quad64, H64, D64, s64) <= prm.tol_gap ||
                        (prm.sign_mode && (P64 < 0.0 || D64 > 0.0))) {
                        if (tid == 0) {
                            phi[k] = (float)(-P64);
                            gap_out[k] = (float)g64;
                            iters[k] = cnt - 1;
                            status[k] = HOPF_OK;
                            if (Pout) Pout[k] = (float)P64;
                            if (Dout) Dout[k] = (float)D64;
                        }
                        done = true;
                    } else {
                        tol *= 0.5f;
                        mg *= 2.f;
                        if (cnt > prm.max_iter) stt = HOPF_MAXITER;
                    }
                    __syncthreads();
                }
                if (!done && stt >= 0 && stt != HOPF_OK) {
                    if (tid == 0) {
                        phi[k] = -Pv;
                        gap_out[k] = gp;
                        iters[k] = cnt - 1;
                        status[k] = stt;
                        if (Pout) Pout[k] = Pv;
                        if (Dout) Dout[k] = Dv;
                    }
                    done = true;
                }
            }
            if (done) {
                for (int a = tid; a < n; a += nt) pstar[(long long)k * n + a] = pb[a];
                __syncthreads();
                break;
            }
            // prox of Eq. 37 (plain) or through the eigenvectors of M (accelerated)
            float pn = 0.f;
            const int a = tid;
            if (!prm.accel) {
                if (a < n4)
                    for (int b = 0; b < n; ++b) pn = fmaf(__ldg(Sp + (long long)b * n4 + a), vb[b], pn);
            } else {
                float w = 0.f;
                if (a < n4)
                    for (int b = 0; b < n; ++b) w = fmaf(__ldg(Up + (long long)b * n4 + a), vb[b], w);
                __syncthreads();
                if (a < n4) ub[a] = a < n ? w / fmaf(0.5f * tau, __ldg(lam + a), 1.f) : 0.f;
                __syncthreads();
                if (a < n4)
                    for (int b = 0; b < n; ++b) pn = fmaf(__ldg(Utp + (long long)b * n4 + a), ub[b], pn);
            }
            const float th = prm.accel ? rsqrtf(fmaf(2.f * gamma, tau, 1.f)) : 1.f;
            __syncthreads();
            if (a < n4) {
                pb[a] = fmaf(th, pn - pp[a], pn);
                pp[a] = pn;
            }
            if (prm.accel) {
                tau *= th;
                sigma /= th;
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------ host side
bool tile_plan(int n, int m, int N, int P, int sms, size_t smem_limit, int *ppt, int *grid, size_t *smem,
               int *dbuf) {
    if (n < 1 || n > 256 || m < 1 || m > 16 || N < 1 || P < 1) return false;
    for (int cand = 2; cand >= 1; --cand) {
        const TileGeom g = tile_geom(n, m, N, cand);
        const int tiles = (P + g.pt - 1) / g.pt;
        if (cand == 2 && tiles < sms) continue;     // prefer more blocks over wider tiles
        for (int db = 1; db >= 0; --db) {
            const size_t bytes = (size_t)tile_smem_floats(g, db != 0) * sizeof(float);
            if (bytes > smem_limit) continue;
            *ppt = cand;
            *grid = tiles < sms ? tiles : sms;
            *smem = bytes;
            *dbuf = db;
            return true;
        }
    }
    return false;
}

// workspace floats: padded K, S, M, V; per-block p, x0 and dual buffers
long long tile_workspace_floats(int n, int m, int N, int ppt, int grid) {
    const TileGeom g = tile_geom(n, m, N, ppt);
    return (long long)g.chunks * g.cr * g.n4 + 5LL * n * g.n4 + 2LL * grid * g.n4 * g.pt +
           (long long)grid * g.chunks * g.cr * g.pt + 16;
}

template <int MP, int PPT>
static cudaError_t launch_tile_t(const float *inst, const double *inst64, const float *Kp, const float *Sp, const float *Mp,
                                 const float *Vp, const SolveParams &prm, const float *x, const float *p_init,
                                 float *phi, float *pstar, float *gap, int *iters, int *status, float *sp,
                                 float *sx, float *sy, int *queue, int grid, size_t smem, int dbuf, float *Pout,
                                 float *Dout, cudaStream_t s) {
    auto kern = pdhg_tile_kernel<MP, PPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, TILE_WARPS * 32, smem, s>>>(inst, inst64, Kp, Sp, Mp, Vp, prm, x, p_init, phi, pstar, gap, iters,
                                             status, sp, sx, sy, queue, dbuf, Pout, Dout);
    return cudaGetLastError();
}

// the tail kernel's dynamic shared memory: pbar, p, x0, v, u [n4], the dual
// rows [chunks cr] and the float64 u of the re-certification [n]
size_t tile_tail_smem(int n, int m, int N, int ppt) {
    const TileGeom g = tile_geom(n, m, N, ppt);
    return sizeof(float) * ((size_t)7 * g.n4 + (size_t)g.chunks * g.cr);
}

// parked-point state: pbar, p [n4] and tau, sigma, count, tolerance
long long tile_carry_floats(int n, int m, int N, int ppt, int P) {
    const TileGeom g = tile_geom(n, m, N, ppt);
    return (long long)P * (2 * g.n4 + 4);
}

// queue: 3 device ints (the tiled kernel's queue, the tail's queue, the
// parked count).  carry_st / carry_list (tile_carry_floats, 2 P ints) enable
// parking and the tail kernel; null runs the tiled kernel alone.
cudaError_t launch_pdhg_tile(const float *inst, const double *inst64, const SolveParams &prm_in, const float *x,
                             const float *p_init, float *phi, float *pstar, float *gap, int *iters, int *status,
                             float *ws, int *queue, int ppt, int grid, size_t smem, int dbuf, float *carry_st,
                             int *carry_list, cudaStream_t s, float *Pout, float *Dout) {
    const int n = prm_in.n, m = prm_in.m, N = prm_in.N;
    const TileGeom g = tile_geom(n, m, N, ppt);
    const size_t tsmem = tile_tail_smem(n, m, N, ppt);
    SolveParams prm = prm_in;
    prm.carry_cap = (carry_st && carry_list && tsmem <= 200 * 1024) ? 1 : 0;
    prm.out_st = carry_st;
    prm.out_list = carry_list;
    prm.out_count = queue + 2;
    float *Kp = ws;
    float *Sp = Kp + (long long)g.chunks * g.cr * g.n4;
    float *Mp = Sp + (long long)n * g.n4;
    float *Vp = Mp + (long long)n * g.n4;
    float *sp = Vp + 3LL * n * g.n4;             // after V come U and U^T
    float *sx = sp + (long long)grid * g.n4 * g.pt;
    float *sy = sx + (long long)grid * g.n4 * g.pt;
    cudaError_t e = cudaMemsetAsync(queue, 0, 3 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    tile_pad_kernel<<<256, 256, 0, s>>>(inst, n, m, N, g, Kp, Sp, Mp, Vp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
#define TILE_CASE(MPV)                                                                                        \
    case MPV:                                                                                                 \
        e = ppt == 2 ? launch_tile_t<MPV, 2>(inst, inst64, Kp, Sp, Mp, Vp, prm, x, p_init, phi, pstar, gap, iters, \
                                             status, sp, sx, sy, queue, grid, smem, dbuf, Pout, Dout, s)        \
                     : launch_tile_t<MPV, 1>(inst, inst64, Kp, Sp, Mp, Vp, prm, x, p_init, phi, pstar, gap, iters, \
                                             status, sp, sx, sy, queue, grid, smem, dbuf, Pout, Dout, s);       \
        break;
    switch (g.mp) {
        TILE_CASE(1)
        TILE_CASE(2)
        TILE_CASE(3)
        TILE_CASE(4)
        TILE_CASE(5)
        TILE_CASE(6)
        TILE_CASE(8)
        TILE_CASE(10)
        TILE_CASE(12)
        TILE_CASE(16)
        default:
            return cudaErrorInvalidValue;
    }
#undef TILE_CASE
    if (e != cudaSuccess || !prm.carry_cap) return e;
    if (tsmem > 48 * 1024) {
        e = cudaFuncSetAttribute(pdhg_tile_tail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem);
        if (e != cudaSuccess) return e;
    }
    pdhg_tile_tail_kernel<<<4 * grid, 256, tsmem, s>>>(inst, inst64, Kp, Sp, prm, ppt, x, phi, pstar, gap, iters,
                                                        status, sy, queue + 1, Pout, Dout);
    return cudaGetLastError();
}

// Tail of another solver: the padded float32 table (the tiled layout) and
// one 256-thread block per point parked in prm.out_* (state records of
// 2 n4 + 4 floats: pbar, p, tau, sigma, iteration count, threshold; dual rows
// in park_y at [e / 32][row][e % 32], the tiled layout with 32 slots).  ws
// holds tile_pad_floats(n, m, N) floats; queue2 is a zeroed device int.
long long tile_pad_floats(int n, int m, int N) {
    const TileGeom g = tile_geom(n, m, N, 1);
    return (long long)g.chunks * g.cr * g.n4 + 5LL * n * g.n4;
}

cudaError_t launch_tile_tail_parked(const float *inst, const double *inst64, const SolveParams &prm, const float *x,
                                    float *phi, float *pstar, float *gap, int *iters, int *status, float *ws,
                                    const float *park_y, int *queue2, int grid, cudaStream_t s) {
    const int n = prm.n, m = prm.m, N = prm.N;
    const TileGeom g = tile_geom(n, m, N, 1);
    const size_t tsmem = tile_tail_smem(n, m, N, 1);
    if (tsmem > 200 * 1024) return cudaErrorInvalidValue;
    float *Kp = ws;
    float *Sp = Kp + (long long)g.chunks * g.cr * g.n4;
    float *Mp = Sp + (long long)n * g.n4;
    float *Vp = Mp + (long long)n * g.n4;
    tile_pad_kernel<<<256, 256, 0, s>>>(inst, n, m, N, g, Kp, Sp, Mp, Vp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (tsmem > 48 * 1024) {
        e = cudaFuncSetAttribute(pdhg_tile_tail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem);
        if (e != cudaSuccess) return e;
    }
    pdhg_tile_tail_kernel<<<grid, 256, tsmem, s>>>(inst, inst64, Kp, Sp, prm, 1, x, phi, pstar, gap, iters, status,
                                                   park_y, queue2, nullptr, nullptr);
    return cudaGetLastError();
}

}  // namespace hopf
