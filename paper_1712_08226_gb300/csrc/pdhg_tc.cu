// Chambolle-Pock iteration (§III, Eq. 15 with theta = 1; prox of Eq. 22-23
// and Eq. 37) for large states on the tensor cores: one node table shared by
// every point, terminal-time variables with a diagonal target matrix W (so
// M' = W, V' = W^-1 and S' = (I + tau W/2)^-1 are diagonal), float32 state.
//
// A persistent block owns 128 point slots, one per tensor-memory lane (and
// per thread of its four slot warps).  Per iteration the two node-table products run as
// tcgen05.mma contractions over node blocks of 64 rows of the stacked table:
//   GEMM1  D1[128 x 64]  = Pbar[128 x n] . K_b^T        (K_b pbar for every slot)
//   GEMM2  D2[128 x n2] += Y_b[128 x 64] . (K_b^T)^T    (K^T y accumulated over blocks)
// with float32 accumulators in tensor memory.  Operands are float32 values
// split into two tf32 parts, x = hi + lo (hi, lo rounded to nearest tf32), and
// each product takes three passes (hi.hi + lo.hi + hi.lo), which carries about
// 22 bits; a single tf32 pass leaves the iteration stuck near a relative gap
// of 1e-5.  Between the two contractions of a node block the thread of each
// slot reads its row of D1, does the dual step and the projection onto w_i U
// (Eq. 23) and writes the new dual block as the A operand of GEMM2; after the
// last block it reads its row of D2 = K^T y and does the diagonal primal prox
// (Eq. 37) and the extrapolation.  Operand chunks (pbar, K blocks, K^T blocks,
// pre-split into tf32 hi/lo and laid out as shared-memory core-matrix images)
// stream through a shared-memory ring of up to four stages with bulk copies
// while the tensor core works on earlier chunks (roles below).
//
// Certificate (every gap_every iterations per slot): P at the pbar the dual
// step used and D at the new feasible y (both diagonal quadratic forms here,
// summed with compensation); a slot that passes in float32 is re-certified by
// the whole block with products evaluated in double-float32 arithmetic from a
// float32 hi/lo split of the float64 table (about 44 bits), P and D formed in
// float64.  An accepted point reports phi = -P, its slot takes the next point
// from a queue; a point that fails the re-check iterates on.
#include "common.cuh"
#include "tc.cuh"

namespace hopf {

// the tiled kernel's tail, reused for the points this kernel parks (pdhg_tile.cu)
long long tile_pad_floats(int n, int m, int N);
size_t tile_tail_smem(int n, int m, int N, int ppt);
cudaError_t launch_tile_tail_parked(const float *inst, const double *inst64, const SolveParams &prm, const float *x,
                                    float *phi, float *pstar, float *gap, int *iters, int *status, float *ws,
                                    const float *park_y, int *queue2, int grid, cudaStream_t s);

constexpr int TC_PTS = 128;                 // slots = tensor-memory lanes = threads
constexpr int TC_NB = 64;                   // rows of the stacked table per node block (GEMM1 N)
constexpr int TC_KC = 32;                   // GEMM1 contraction chunk (state components)
constexpr int TC_RC = 32;                   // GEMM2 contraction chunk (table rows)
constexpr int TC_YBYTES = 2 * 2 * TC_PTS * TC_RC * 4;   // dual block: 2 chunks x hi/lo
constexpr uint32_t TC_D1_COL = 256;         // tensor memory: D2 in [0, n2), two D1 in [256, 384)

struct TcGeom {
    int n, m, N, mp, npb, nblk, n1, nch1, n2;
    long long rows;
};

// rows reserved per node inside a block: 2, 4, 8, 10 or 16 (extra rows are zero)
__host__ __device__ inline int tc_mpad(int m) { return m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : m <= 10 ? 10 : 16; }

__host__ __device__ inline TcGeom tc_geom(int n, int m, int N) {
    TcGeom g;
    g.n = n;
    g.m = m;
    g.N = N;
    g.mp = tc_mpad(m);
    g.npb = TC_NB / g.mp;
    g.nblk = (N + g.npb - 1) / g.npb;
    g.n1 = (n + 7) & ~7;
    g.nch1 = (g.n1 + TC_KC - 1) / TC_KC;
    g.n2 = (n + 15) & ~15;
    g.rows = (long long)g.nblk * TC_NB;
    return g;
}
__host__ __device__ inline int tc_kcw(const TcGeom &g, int kc) {
    const int w = g.n1 - kc * TC_KC;
    return w < TC_KC ? w : TC_KC;
}

// float32 -> nearest tf32 (low 13 mantissa bits cleared, ties to even), the
// value the tensor core reads from a float32 container
__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) != 0x7f800000u) u += 0x0fffu + ((u >> 13) & 1u);
    return __uint_as_float(u & 0xffffe000u);
}
__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
    hi = tf32_rn(x);
    lo = tf32_rn(x - hi);
}

// ---------------------------------------------------------------- layouts
// element offset (floats) inside a core-matrix image of rows x kw floats
__device__ __forceinline__ int core_idx(int row, int k, int kw) { return (int)(tc::core_offset(row, k, kw * 4, 4) >> 2); }

struct TcImages {
    float *K1, *K2, *Kh, *Kl, *KTh, *KTl, *d32;
    double *d64;
};
__host__ __device__ inline long long tc_k1_floats(const TcGeom &g) { return (long long)g.nblk * g.nch1 * 2 * TC_NB * TC_KC; }
__host__ __device__ inline long long tc_k2_floats(const TcGeom &g) { return (long long)g.nblk * 2 * 2 * g.n2 * TC_RC; }
__host__ __device__ inline long long tc_slot_floats(const TcGeom &g) {
    // pbar image, x0, p, pbar (two buffers), dual variables
    return (long long)g.nch1 * 2 * TC_PTS * TC_KC + 4LL * TC_PTS * g.n1 + (long long)TC_PTS * g.rows;
}

// padded row R of node block b, local row r: node i = b npb + r / mp, control c = r % mp
__device__ __forceinline__ bool tc_row(const TcGeom &g, long long R, int &i, int &c) {
    const int b = (int)(R / TC_NB), r = (int)(R % TC_NB);
    const int t = r / g.mp;
    c = r % g.mp;
    i = b * g.npb + t;
    return t < g.npb && c < g.m && i < g.N;
}

// one-off: tensor-core operand images and the re-certification copies of the
// float64 table, diagonal of M', V', S'
__global__ void tc_prep_kernel(const double *__restrict__ inst64, int n, int m, int N, TcGeom g, TcImages im) {
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    const double *K = inst64 + L.K;
    const long long nk1 = tc_k1_floats(g), nk2 = tc_k2_floats(g), nkd = g.rows * g.n1, nkt = (long long)n * g.rows;
    const long long total = nk1 + nk2 + nkd + nkt + 3LL * g.n1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; e0 < total; e0 += stride) {
        long long e = e0;
        if (e < nk1) {
            // K1: [b][kc][h] chunks of 64 rows x kcw, core-matrix image
            const long long chunk = e / (TC_NB * TC_KC);
            const int off = (int)(e % (TC_NB * TC_KC));
            const int h = (int)(chunk & 1);
            const int kc = (int)((chunk >> 1) % g.nch1);
            const int b = (int)((chunk >> 1) / g.nch1);
            const int kw = tc_kcw(g, kc);
            if (off >= TC_NB * kw) continue;
            // invert the core layout: off -> (row, k)
            const int cm = off >> 5, within = off & 31;             // core matrix index, element in it
            const int kgroups = kw >> 2;
            const int rg = cm / kgroups, kg = cm % kgroups;
            const int row = rg * 8 + (within >> 2), k = kg * 4 + (within & 3);
            const int j = kc * TC_KC + k;
            int i, c;
            float v = 0.f;
            if (j < n && tc_row(g, (long long)b * TC_NB + row, i, c)) {
                float hi, lo;
                tf32_split((float)K[((long long)i * m + c) * n + j], hi, lo);
                const double rest = K[((long long)i * m + c) * n + j] - (double)hi;
                lo = tf32_rn((float)rest);
                v = h ? lo : hi;
            }
            im.K1[e] = v;
        } else if ((e -= nk1) < nk2) {
            // K2: [b][rc][h] chunks of n2 rows (state) x 32 (table rows), core-matrix image
            const long long chunk = e / ((long long)g.n2 * TC_RC);
            const int off = (int)(e % ((long long)g.n2 * TC_RC));
            const int h = (int)(chunk & 1);
            const int rc = (int)((chunk >> 1) & 1);
            const int b = (int)(chunk >> 2);
            const int cm = off >> 5, within = off & 31;
            const int rg = cm / (TC_RC / 4), kg = cm % (TC_RC / 4);
            const int j = rg * 8 + (within >> 2), k = kg * 4 + (within & 3);
            int i, c;
            float v = 0.f;
            if (j < n && tc_row(g, (long long)b * TC_NB + rc * TC_RC + k, i, c)) {
                const double kv = K[((long long)i * m + c) * n + j];
                const float hi = tf32_rn((float)kv);
                v = h ? tf32_rn((float)(kv - (double)hi)) : hi;
            }
            im.K2[e] = v;
        } else if ((e -= nk2) < nkd) {
            // Kh/Kl: [rows][n1] float32 hi/lo split of the float64 table (re-certification)
            const long long R = e / g.n1;
            const int j = (int)(e % g.n1);
            int i, c;
            double kv = 0.0;
            if (j < n && tc_row(g, R, i, c)) kv = K[((long long)i * m + c) * n + j];
            const float hi = (float)kv;
            im.Kh[e] = hi;
            im.Kl[e] = (float)(kv - (double)hi);
        } else if ((e -= nkd) < nkt) {
            // KTh/KTl: [n][rows]
            const int j = (int)(e / g.rows);
            const long long R = e % g.rows;
            int i, c;
            double kv = 0.0;
            if (tc_row(g, R, i, c)) kv = K[((long long)i * m + c) * n + j];
            const float hi = (float)kv;
            im.KTh[e] = hi;
            im.KTl[e] = (float)(kv - (double)hi);
        } else {
            e -= nkt;
            const int which = (int)(e / g.n1), j = (int)(e % g.n1);
            const double *D = inst64 + (which == 0 ? L.M : which == 1 ? L.V : L.S);
            const double v = j < n ? D[(long long)j * n + j] : 0.0;
            im.d64[e] = v;
            im.d32[e] = (float)v;
        }
    }
}

// --------------------------------------------------- compensated arithmetic
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, float b) {
    const float s = a.hi + b;
    const float bb = s - a.hi;
    const float err = (a.hi - (s - bb)) + (b - bb);
    DF r;
    r.hi = s;
    r.lo = a.lo + err;
    return r;
}
// a += (kh + kl) * x, with the product error of kh * x kept
__device__ __forceinline__ DF df_fma(DF a, float kh, float kl, float x) {
    const float p = kh * x;
    const float pe = fmaf(kh, x, -p);
    a = df_add(a, p);
    a.lo += fmaf(kl, x, pe);
    return a;
}
__device__ __forceinline__ DF df_shfl_sum(DF a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, a.hi, o), l = __shfl_xor_sync(0xffffffffu, a.lo, o);
        a = df_add(a, h);
        a.lo += l;
    }
    return a;
}
__device__ __forceinline__ void kahan(float &s, float &c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

__device__ __forceinline__ double tc_block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    const double t = red[0] + red[1] + red[2] + red[3];
    __syncthreads();
    return t;
}

// ------------------------------------------------------------------ kernel
// Thread roles: warps 0-3 own the 128 slots (tensor-memory lanes 32 w ..
// 32 w + 31, the dual and primal steps, certificates); lane 0 of warp 5
// streams the operand chunks of every iteration with bulk copies
// (cp.async.bulk, completion counted in bytes on an mbarrier) into an
// S-stage ring; lane 0 of warp 4 issues the MMAs in the order
//   G1(0), G1(1), G2(0), G1(2), G2(1), ..., G1(nblk-1), G2(nblk-2), G2(nblk-1)
// so that the dual step of block b (on the slot warps) overlaps GEMM1 of
// block b + 1 (two D1 accumulators in tensor memory).  Handshakes, all
// mbarriers: ring full/empty per stage, D1 full/empty per accumulator, dual
// block full/empty, D2 full once per iteration.  Every wait is bounded; a
// wait that runs out sets a shared failure flag, after which no thread waits
// or issues work any more and the block leaves at the end of the iteration.
constexpr int TC_THREADS = TC_PTS + 64;
constexpr int TC_MAX_STAGES = 4;
constexpr int TC_YOFF_LO = TC_PTS * TC_RC * 4;           // bytes: lo half of a dual chunk image
constexpr int TC_G1_ALO = TC_PTS * TC_KC * 4;            // offsets inside a ring stage (GEMM1 chunk)
constexpr int TC_G1_BHI = 2 * TC_PTS * TC_KC * 4;
constexpr int TC_G1_BLO = TC_G1_BHI + TC_NB * TC_KC * 4;

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(tc::smem_u32(mbar))
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(mbar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(mbar)) : "memory");
}
// barrier of the 128 slot threads only (named barrier 1)
__device__ __forceinline__ void slots_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// bounded wait; false (and the failure flag set) when it runs out or another
// thread has failed already
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, volatile int *fail) {
    for (long long i = 0; i < (1LL << 26); ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && *fail) return false;
    }
    *fail = 1;
    return false;
}

__device__ __forceinline__ double slots_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    slots_sync();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    slots_sync();
    const double t = red[0] + red[1] + red[2] + red[3];
    slots_sync();
    return t;
}

// three tf32 passes (hi.hi, lo.hi, hi.lo) over KS k-steps of 8; a descriptor's
// start address advances 256 bytes (16 units) per k-step
template <int KS>
__device__ __forceinline__ void mma3(uint32_t d, uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl, uint32_t idesc,
                                     bool first) {
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) tc::mma_tf32(d, ah + 16u * ks, bh + 16u * ks, idesc, (first && ks == 0) ? 0u : 1u);
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) tc::mma_tf32(d, al + 16u * ks, bh + 16u * ks, idesc, 1u);
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) tc::mma_tf32(d, ah + 16u * ks, bl + 16u * ks, idesc, 1u);
}

// position k of an iteration's chunk sequence: GEMM1 (g1 = true) or GEMM2
// chunk q of node block b
__device__ __forceinline__ void tc_chunk(const TcGeom &g, int k, bool &g1, int &b, int &q) {
    const int per = g.nch1 + 2;
    if (k < g.nch1) {
        g1 = true;
        b = 0;
        q = k;
        return;
    }
    const int k2 = k - g.nch1;
    const int st = 1 + k2 / per, r = k2 % per;
    if (st < g.nblk && r < g.nch1) {
        g1 = true;
        b = st;
        q = r;
    } else {
        g1 = false;
        b = st - 1;
        q = st < g.nblk ? r - g.nch1 : r;
    }
}

template <int MP>
__global__ void __launch_bounds__(TC_THREADS, 1)
pdhg_tc_kernel(TcGeom g, TcImages im, const float *__restrict__ inst, const double *__restrict__ inst64,
               SolveParams prm, const float *__restrict__ x, const float *__restrict__ p_init,
               float *__restrict__ phi, float *__restrict__ pstar, float *__restrict__ gap_out,
               int *__restrict__ iters, int *__restrict__ status, float *__restrict__ slots, int *queue, int *err,
               int stages, int stage_bytes, float *__restrict__ park_st, int *__restrict__ park_list,
               int *park_count, float *__restrict__ park_y) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t mb_full[TC_MAX_STAGES], mb_empty[TC_MAX_STAGES];
    __shared__ __align__(8) uint64_t mb_d1f[2], mb_d1e[2], mb_yf, mb_ye, mb_d2f;
    __shared__ uint32_t s_taddr;
    __shared__ int s_flag[TC_PTS];
    __shared__ volatile int s_fail;
    __shared__ int s_park;
    __shared__ double red[4];

    const int tid = threadIdx.x, warp = tid >> 5;
    const bool slot_thread = tid < TC_PTS;
    const int n = g.n, m = g.m, N = g.N, P = prm.P;
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    const float *sc = inst + L.sc;
    const float *wv = inst + L.w;
    const double *w64 = inst64 + L.w;
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

    const int n1 = g.n1, nch1 = g.nch1, n2 = g.n2, nblk = g.nblk;
    const long long rows = g.rows;
    const float tau = (float)prm.tau;
    const float sigma = sc[SC_SIGMA];
    const float *Md = im.d32, *Vd = im.d32 + n1, *Sd = im.d32 + 2 * n1;
    const double *Md64 = im.d64, *Vd64 = im.d64 + n1;

    // per-block slot storage (global, L2 resident)
    float *base = slots + (long long)blockIdx.x * tc_slot_floats(g);
    float *Pimg = base;                                             // [kc][h][128 x 32] core images
    float *xs = Pimg + (long long)nch1 * 2 * TC_PTS * TC_KC;        // [n1][slot]
    float *ps = xs + (long long)TC_PTS * n1;
    float *pbs = ps + (long long)TC_PTS * n1;                       // [2][n1][slot]
    float *ys = pbs + 2LL * TC_PTS * n1;                            // [rows][slot]
    // slot-minor layouts: a warp's accesses to one component or row coalesce
    const int sl = slot_thread ? tid : 0;
    float *xrow = xs + sl, *prow = ps + sl, *yrow = ys + sl;       // element j at [j * TC_PTS]

    if (warp == 0) tc::tmem_alloc(&s_taddr, 512);
    if (tid == 0) {
        for (int s = 0; s < TC_MAX_STAGES; ++s) {
            tc::mbar_init(&mb_full[s], 1);
            tc::mbar_init(&mb_empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&mb_d1f[s], 1);
            tc::mbar_init(&mb_d1e[s], TC_PTS);
        }
        tc::mbar_init(&mb_yf, TC_PTS);
        tc::mbar_init(&mb_ye, 1);
        tc::mbar_init(&mb_d2f, 1);
        s_fail = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = s_taddr;
    const uint32_t t_lane = taddr + ((uint32_t)((warp & 3) * 32) << 16);
    unsigned char *Ysm = tsm + (size_t)stages * stage_bytes;

    // slot state (thread tid < 128 owns slot tid)
    int pt = -1, cnt = 0, fresh = 0, par = 0, last_check = -1000000;
    const int Pq = prm.list ? *prm.list_count : P;

    // tf32 hi/lo image of pbar components j .. j + 3 of this slot (GEMM1 A operand)
    auto store_pbar_img4 = [&](int j, float4 v) {
        const int kc = j / TC_KC, k = j % TC_KC;
        const int kw = tc_kcw(g, kc);
        float4 h4, l4;
        tf32_split(v.x, h4.x, l4.x);
        tf32_split(v.y, h4.y, l4.y);
        tf32_split(v.z, h4.z, l4.z);
        tf32_split(v.w, h4.w, l4.w);
        float *img = Pimg + (long long)kc * 2 * TC_PTS * TC_KC;
        const int o = core_idx(tid, k, kw);
        *reinterpret_cast<float4 *>(img + o) = h4;
        *reinterpret_cast<float4 *>(img + TC_PTS * TC_KC + o) = l4;
    };
    auto take_point = [&]() {
        int k = -1;
        const int q = atomicAdd(queue, 1);
        if (q < Pq) k = prm.list ? prm.list[q] : q;
        pt = k;
        cnt = 0;
        fresh = k >= 0;
        last_check = -1000000;
        float *pbn = pbs + (long long)(par ^ 1) * TC_PTS * n1 + tid;
        for (int j = 0; j < n1; j += 4) {
            float xv[4], pv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                xv[e] = pv[e] = 0.f;
                if (k >= 0 && j + e < n) {
                    xv[e] = x[(long long)k * n + j + e];
                    pv[e] = prm.warm ? p_init[(long long)k * n + j + e] : xv[e];
                }
            }
            const float4 p4 = make_float4(pv[0], pv[1], pv[2], pv[3]);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                xrow[(j + e) * TC_PTS] = xv[e];
                prow[(j + e) * TC_PTS] = pv[e];
                pbn[(j + e) * TC_PTS] = pv[e];
            }
            store_pbar_img4(j, p4);
        }
    };
    if (slot_thread) {
        par = 1;          // take_point fills buffer par ^ 1 = 0, the first iteration's pbar
        take_point();
        par = 0;
        // the pbar images are read by bulk copies (async proxy)
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    __syncthreads();

    const int J = nblk * (nch1 + 2);
    const uint32_t idesc1 = tc::make_idesc(128, TC_NB, tc::FMT_TF32);
    const uint32_t idesc2 = tc::make_idesc(128, n2, tc::FMT_TF32);

    for (int it = 0;; ++it) {
        if (warp >= 4) {
            if (tid == TC_PTS + 32) {
                // ================= loader: bulk copies of this iteration's chunks
                const long long kbase = (long long)it * J;
                for (int k = 0; k < J && !s_fail; ++k) {
                    const long long kg = kbase + k;
                    const int st = (int)(kg % stages);
                    const long long use = kg / stages;
                    if (use >= 1 && !tc_wait(&mb_empty[st], (uint32_t)((use - 1) & 1), &s_fail)) break;
                    unsigned char *dst = tsm + (size_t)st * stage_bytes;
                    bool g1;
                    int b, q;
                    tc_chunk(g, k, g1, b, q);
                    if (g1) {
                        // pbar image chunk (hi, lo 16 KB further on) and the K block chunk
                        // (hi, lo 8 KB further on), each as one copy
                        const int kw = tc_kcw(g, q);
                        const uint32_t ab = (uint32_t)(TC_G1_ALO + TC_PTS * kw * 4);
                        const uint32_t bb = (uint32_t)(TC_NB * TC_KC * 4 + TC_NB * kw * 4);
                        mbar_expect_tx(&mb_full[st], ab + bb);
                        bulk_g2s(dst, Pimg + (long long)q * 2 * TC_PTS * TC_KC, ab, &mb_full[st]);
                        bulk_g2s(dst + TC_G1_BHI, im.K1 + ((long long)b * nch1 + q) * 2 * TC_NB * TC_KC, bb,
                                 &mb_full[st]);
                    } else {
                        const uint32_t bb = (uint32_t)(2 * n2 * TC_RC * 4);
                        mbar_expect_tx(&mb_full[st], bb);
                        bulk_g2s(dst, im.K2 + ((long long)b * 2 + q) * 2 * n2 * TC_RC, bb, &mb_full[st]);
                    }
                }
            } else if (tid == TC_PTS) {
                // ================= tensor-core issuer
                const long long kbase = (long long)it * J;
                for (int k = 0; k < J && !s_fail; ++k) {
                    const long long kg = kbase + k;
                    const int st = (int)(kg % stages);
                    bool g1;
                    int b, q;
                    tc_chunk(g, k, g1, b, q);
                    const long long gb = (long long)it * nblk + b;
                    // dependencies: the D1 accumulator free again (GEMM1), the
                    // dual block written (GEMM2), the operands landed
                    if (g1 && q == 0 && gb >= 2 &&
                        !tc_wait(&mb_d1e[gb & 1], (uint32_t)(((gb >> 1) - 1) & 1), &s_fail))
                        break;
                    if (!g1 && q == 0 && !tc_wait(&mb_yf, (uint32_t)(gb & 1), &s_fail)) break;
                    if (!tc_wait(&mb_full[st], (uint32_t)((kg / stages) & 1), &s_fail)) break;
                    tc::fence_after_sync();
                    const uint32_t src = tc::smem_u32(tsm + (size_t)st * stage_bytes);
                    if (g1) {
                        const int kw = tc_kcw(g, q);
                        const uint32_t sbo = (uint32_t)(kw / 4) * 128u;
                        const uint32_t d1 = taddr + TC_D1_COL + (uint32_t)(gb & 1) * TC_NB;
                        const uint64_t ah = tc::make_desc(src, 128u, sbo), al = tc::make_desc(src + TC_G1_ALO, 128u, sbo);
                        const uint64_t bh = tc::make_desc(src + TC_G1_BHI, 128u, sbo);
                        const uint64_t bl = tc::make_desc(src + TC_G1_BLO, 128u, sbo);
                        switch (kw / 8) {
                            case 1: mma3<1>(d1, ah, al, bh, bl, idesc1, q == 0); break;
                            case 2: mma3<2>(d1, ah, al, bh, bl, idesc1, q == 0); break;
                            case 3: mma3<3>(d1, ah, al, bh, bl, idesc1, q == 0); break;
                            default: mma3<4>(d1, ah, al, bh, bl, idesc1, q == 0); break;
                        }
                        tc::mma_commit(&mb_empty[st]);
                        if (q == nch1 - 1) tc::mma_commit(&mb_d1f[gb & 1]);
                    } else {
                        const uint32_t y_hi = tc::smem_u32(Ysm) + (uint32_t)q * 2 * TC_YOFF_LO;
                        const uint32_t sbo = (uint32_t)(TC_RC / 4) * 128u;
                        const uint64_t ah = tc::make_desc(y_hi, 128u, sbo), al = tc::make_desc(y_hi + TC_YOFF_LO, 128u, sbo);
                        const uint64_t bh = tc::make_desc(src, 128u, sbo);
                        const uint64_t bl = tc::make_desc(src + (uint32_t)(n2 * TC_RC * 4), 128u, sbo);
                        mma3<TC_RC / 8>(taddr, ah, al, bh, bl, idesc2, b == 0 && q == 0);
                        tc::mma_commit(&mb_empty[st]);
                        if (q == 1) {
                            tc::mma_commit(&mb_ye);
                            if (b == nblk - 1) tc::mma_commit(&mb_d2f);
                        }
                    }
                }
            }
        } else {
            // ================= slot threads: dual step per node block
            if (pt >= 0) ++cnt;
            float H = 0.f, Hc = 0.f;   // sum_i w_i |K_i pbar|_* of this iteration, compensated
            const float *pbo = pbs + (long long)par * TC_PTS * n1 + tid;   // pbar used by this iteration
            float *pbn = pbs + (long long)(par ^ 1) * TC_PTS * n1 + tid;
            for (int b = 0; b < nblk; ++b) {
                const long long gb = (long long)it * nblk + b;
                // this block's dual rows first: their global-memory latency
                // overlaps the wait for the K pbar product
                float yv[TC_NB];
                const long long R0 = (long long)b * TC_NB;
                if (pt >= 0 && !fresh) {
#pragma unroll
                    for (int e = 0; e < TC_NB; ++e) yv[e] = yrow[(R0 + e) * TC_PTS];
                }
                tc_wait(&mb_d1f[gb & 1], (uint32_t)((gb >> 1) & 1), &s_fail);
                tc::fence_after_sync();
                float z[TC_NB];
#pragma unroll
                for (int c0 = 0; c0 < TC_NB; c0 += 16) {
                    float v[16];
                    tc::tmem_ld16(t_lane + TC_D1_COL + (uint32_t)(gb & 1) * TC_NB + (uint32_t)c0, v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) z[c0 + e] = v[e];
                }
                tc::fence_before_sync();
                mbar_arrive(&mb_d1e[gb & 1]);             // GEMM1 of block b + 2 may overwrite it
                constexpr int NPB = TC_NB / MP;
#pragma unroll
                for (int t = 0; t < NPB; ++t) {
                    const int i = b * NPB + t;
                    const bool ok = pt >= 0 && i < N;
                    const float wi = ok ? __ldg(wv + i) : 0.f;
                    float nt = 0.f;
#pragma unroll
                    for (int c = 0; c < MP; ++c) {
                        const float zz = c < m ? z[t * MP + c] : 0.f;
                        nt += ball ? zz * zz : fabsf(zz);
                    }
                    if (ok) kahan(H, Hc, wi * (ball ? sqrtf(nt) : nt));
                    float nu = 0.f;
#pragma unroll
                    for (int c = 0; c < MP; ++c) {
                        const int r = t * MP + c;
                        float yo;
                        if (!ok || c >= m) yo = 0.f;
                        else if (!fresh) yo = yv[r];
                        else if (!prm.warm) yo = z[r];                        // y0 = K p0 (§VI), unprojected
                        else if (ball) yo = nt > 0.f ? z[r] * wi * rsqrtf(nt) : 0.f;   // w_i argmax <c, K_i p0>
                        else yo = z[r] >= 0.f ? wi : -wi;
                        const float yn = (ok && c < m) ? fmaf(sigma, z[r], yo) : 0.f;
                        yv[r] = yn;
                        nu = fmaf(yn, yn, nu);
                    }
                    if (ok) {
                        if (ball) {
                            const float scl = (nu > wi * wi) ? wi * rsqrtf(nu) : 1.f;
#pragma unroll
                            for (int c = 0; c < MP; ++c) yv[t * MP + c] *= scl;
                        } else {
#pragma unroll
                            for (int c = 0; c < MP; ++c) yv[t * MP + c] = fminf(fmaxf(yv[t * MP + c], -wi), wi);
                        }
                    }
                }
#pragma unroll
                for (int r = NPB * MP; r < TC_NB; ++r) yv[r] = 0.f;
                if (pt >= 0) {
#pragma unroll
                    for (int e = 0; e < TC_NB; ++e) yrow[(R0 + e) * TC_PTS] = yv[e];
                }
                // the previous dual block has been consumed by GEMM2
                if (gb >= 1) tc_wait(&mb_ye, (uint32_t)((gb - 1) & 1), &s_fail);
                // dual block as the A operand of GEMM2 (tf32 hi/lo, core-matrix images)
                float *Yf = reinterpret_cast<float *>(Ysm);
#pragma unroll
                for (int rc = 0; rc < 2; ++rc) {
#pragma unroll
                    for (int k = 0; k < TC_RC; k += 4) {
                        float4 h4, l4;
                        tf32_split(yv[rc * TC_RC + k], h4.x, l4.x);
                        tf32_split(yv[rc * TC_RC + k + 1], h4.y, l4.y);
                        tf32_split(yv[rc * TC_RC + k + 2], h4.z, l4.z);
                        tf32_split(yv[rc * TC_RC + k + 3], h4.w, l4.w);
                        const int o = core_idx(tid, k, TC_RC);
                        *reinterpret_cast<float4 *>(Yf + rc * 2 * TC_PTS * TC_RC + o) = h4;
                        *reinterpret_cast<float4 *>(Yf + rc * 2 * TC_PTS * TC_RC + TC_PTS * TC_RC + o) = l4;
                    }
                }
                tc::fence_smem_to_async();
                mbar_arrive(&mb_yf);
            }
            // ---- primal prox (diagonal S), extrapolation, certificate
            tc_wait(&mb_d2f, (uint32_t)(it & 1), &s_fail);
            tc::fence_after_sync();
            fresh = 0;
            const bool check = pt >= 0 && (cnt % prm.gap_every == 0 || cnt > prm.max_iter) &&
                               (cnt >= 2 || cnt > prm.max_iter);
            float qs = 0.f, qc = 0.f, ds = 0.f, dc = 0.f;
            for (int c0 = 0; c0 < n2; c0 += 16) {
                float u[16];
                tc::tmem_ld16(t_lane + (uint32_t)c0, u);
                if (pt < 0) continue;
#pragma unroll
                for (int e0 = 0; e0 < 16; e0 += 4) {
                    const int j0 = c0 + e0;
                    if (j0 >= n) break;
                    const float4 s4 = __ldg(reinterpret_cast<const float4 *>(Sd + j0));
                    float xa[4], pa[4], ba[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        xa[e] = xrow[(j0 + e) * TC_PTS];
                        pa[e] = prow[(j0 + e) * TC_PTS];
                        ba[e] = pbo[(j0 + e) * TC_PTS];
                    }
                    const float sa[4] = {s4.x, s4.y, s4.z, s4.w};
                    float pn[4], pbv[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float v = fmaf(tau, xa[e] - u[e0 + e], pa[e]);
                        pn[e] = j0 + e < n ? sa[e] * v : 0.f;
                        pbv[e] = 2.f * pn[e] - pa[e];
                        if (check && j0 + e < n) {
                            kahan(qs, qc, ba[e] * fmaf(0.25f * __ldg(Md + j0 + e), ba[e], -xa[e]));
                            const float r = xa[e] - u[e0 + e];
                            kahan(ds, dc, r * r * __ldg(Vd + j0 + e));
                        }
                    }
                    const float4 pb4 = make_float4(pbv[0], pbv[1], pbv[2], pbv[3]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        prow[(j0 + e) * TC_PTS] = pn[e];
                        pbn[(j0 + e) * TC_PTS] = pbv[e];
                    }
                    store_pbar_img4(j0, pb4);
                }
            }
            // stop decisions.  The float32 gap of the large chain-like problems
            // carries noise near 1e-5 (K^T y is accumulated over thousands of
            // table rows in float32), so it only nominates points; the
            // double-float32 re-check (which reads the whole table) decides: at
            // most once every 8 gap checks for a float32 gap within 1.5 tol, once
            // every 32 checks within 4 tol.
            int cand = 0;
            if (check) {
                const float quad = qs + 1.f;
                const float Pv = quad + H, Dv = 1.f - ds;
                const float gp = rel_gap(Pv, Dv);
                if (!isfinite(Pv) || !isfinite(Dv)) {
                    phi[pt] = -Pv;
                    gap_out[pt] = gp;
                    iters[pt] = cnt - 1;
                    status[pt] = HOPF_NONFINITE;
                    cand = 2;
                } else if ((gp <= 1.5f * (float)prm.tol_gap && cnt - last_check >= 8 * prm.gap_every) ||
                           (gp <= 4.f * (float)prm.tol_gap && cnt - last_check >= 32 * prm.gap_every)) {
                    cand = 1;
                    last_check = cnt;
                } else if (cnt > prm.max_iter) {
                    phi[pt] = -Pv;
                    gap_out[pt] = gp;
                    iters[pt] = cnt - 1;
                    status[pt] = HOPF_MAXITER;
                    for (int j = 0; j < n; ++j) pstar[(long long)pt * n + j] = pbo[j * TC_PTS];
                    cand = 2;
                }
            }
            s_flag[tid] = cand;
            slots_sync();
            // re-check of the nominated points, one slot at a time (whole slot
            // group), reading the float32 hi/lo split of the float64 table once
            // per product.  The ring stages are idle here (this iteration's
            // contractions are complete, the next one's copies wait for the
            // iteration barrier): the point's pbar, x0 and y are gathered there,
            // and the row products z_R = K_R pbar kept there in float64.
            float *stage_f = reinterpret_cast<float *>(tsm);
            float *pb_c = stage_f, *x_c = stage_f + n1, *y_c = stage_f + 2 * n1;
            double *z_c = reinterpret_cast<double *>(stage_f + ((2 * n1 + rows + 1) & ~1LL));
            for (int s = 0; s < TC_PTS; ++s) {
                if (s_flag[s] != 1) continue;                           // uniform (shared memory)
                const float *pb_s = pbs + (long long)par * TC_PTS * n1 + s;   // element j at [j * TC_PTS]
                for (int j = tid; j < n1; j += TC_PTS) {
                    pb_c[j] = j < n ? pb_s[j * TC_PTS] : 0.f;
                    x_c[j] = j < n ? xs[j * TC_PTS + s] : 0.f;
                }
                for (long long R = tid; R < rows; R += TC_PTS) y_c[R] = ys[R * TC_PTS + s] * (1.f - 4e-7f);
                // (y shrunk by 4e-7 so that float32 rounding cannot leave w_i U)
                slots_sync();
                // z_R = K_R pbar in double-float32, one thread per table row
                for (long long R = tid; R < rows; R += TC_PTS) {
                    DF a = {0.f, 0.f};
                    const float4 *kh4 = reinterpret_cast<const float4 *>(im.Kh + R * n1);
                    const float4 *kl4 = reinterpret_cast<const float4 *>(im.Kl + R * n1);
#pragma unroll 4
                    for (int q = 0; q < n1 / 4; ++q) {
                        const float4 h = kh4[q], l = kl4[q];
                        a = df_fma(a, h.x, l.x, pb_c[4 * q]);
                        a = df_fma(a, h.y, l.y, pb_c[4 * q + 1]);
                        a = df_fma(a, h.z, l.z, pb_c[4 * q + 2]);
                        a = df_fma(a, h.w, l.w, pb_c[4 * q + 3]);
                    }
                    z_c[R] = (double)a.hi + (double)a.lo;
                }
                slots_sync();
                // H = sum_i w_i |K_i pbar|_*
                double hp = 0.0;
                for (int i = tid; i < N; i += TC_PTS) {
                    const long long R = (long long)(i / g.npb) * TC_NB + (i % g.npb) * g.mp;
                    double nt = 0.0;
                    for (int c = 0; c < m; ++c) nt += ball ? z_c[R + c] * z_c[R + c] : fabs(z_c[R + c]);
                    hp += w64[i] * (ball ? sqrt(nt) : nt);
                }
                const double H64 = slots_sum(hp, red);
                // u = x0 - K^T y (threads over state components, rows read
                // coalesced), D = 1 - u^T V u, quad = pbar^T M pbar / 4 - <x0, pbar>
                double dq = 0.0, qq = 0.0;
                for (int j = tid; j < n; j += TC_PTS) {
                    DF a = {0.f, 0.f};
                    const float *kh = im.Kh + j, *kl = im.Kl + j;
#pragma unroll 8
                    for (int R = 0; R < (int)rows; ++R) a = df_fma(a, kh[(long long)R * n1], kl[(long long)R * n1], y_c[R]);
                    const double u = (double)x_c[j] - ((double)a.hi + (double)a.lo);
                    dq += u * u * Vd64[j];
                    const double pb = (double)pb_c[j];
                    qq += pb * (0.25 * Md64[j] * pb - (double)x_c[j]);
                }
                const double D64 = 1.0 - slots_sum(dq, red);
                const double P64 = 1.0 + slots_sum(qq, red) + H64;
                if (tid == s) {
                    const double gp = (P64 - D64) / fmax(1.0, fmax(fabs(P64), fabs(D64)));
                    if (gp <= prm.tol_gap) {
                        phi[pt] = (float)(-P64);
                        gap_out[pt] = (float)gp;
                        iters[pt] = cnt - 1;
                        status[pt] = HOPF_OK;
                        for (int j = 0; j < n; ++j) pstar[(long long)pt * n + j] = pbo[j * TC_PTS];
                        cand = 2;
                    } else {
                        cand = 0;
                    }
                }
            }
            // finished slots take the next point; pbar images go to the bulk copies
            if (cand == 2) take_point();
            par ^= 1;
            // generic writes (pbar images, gathered re-check operands in the ring)
            // before the next iteration's bulk copies
            asm volatile("fence.proxy.async;" ::: "memory");
        }
        // iteration boundary, all threads (every copy and product of the
        // iteration is complete here)
        const int any = __syncthreads_or(slot_thread && pt >= 0);
        if (any == 0 || s_fail) break;
        // drain: the queue is empty and at most a quarter of the slots are
        // busy.  A block-iteration costs the same with 1 or 128 busy slots, so
        // the remaining points are parked (pbar, p, step sizes, count; the dual
        // rows converted to the tiled layout) for the one-block-per-point tail
        // kernel, which iterates a point with the table read from L2.
        if (park_y) {
            const int act = __syncthreads_count(slot_thread && pt >= 0);
            const int fr = __syncthreads_or(slot_thread && pt >= 0 && fresh);
            if (tid == 0)
                s_park = (!fr && 4 * act <= TC_PTS && *reinterpret_cast<volatile int *>(queue) >= Pq) ? 1 : 0;
            __syncthreads();
            if (s_park) {
                if (slot_thread && pt >= 0) {
                    const TileGeom tg = tile_geom(n, m, N, 1);
                    const int n4 = tg.n4, CW = 2 * n4 + 4, G = tg.chunks * tg.cr;
                    const int e = atomicAdd(park_count, 1);
                    park_list[2 * e] = pt;
                    park_list[2 * e + 1] = e;
                    float *st = park_st + (long long)e * CW;
                    const float *pbc = pbs + (long long)par * TC_PTS * n1 + tid;     // the next iteration's pbar
                    for (int j = 0; j < n4; ++j) {
                        st[j] = j < n ? pbc[j * TC_PTS] : 0.f;
                        st[n4 + j] = j < n ? prow[j * TC_PTS] : 0.f;
                    }
                    st[2 * n4] = tau;
                    st[2 * n4 + 1] = sigma;
                    st[2 * n4 + 2] = (float)cnt;
                    st[2 * n4 + 3] = (float)prm.tol_gap;
                    float *yd = park_y + (long long)(e / 32) * G * 32 + (e % 32);
                    for (int i = 0; i < N; ++i) {
                        const long long R = (long long)(i / g.npb) * TC_NB + (i % g.npb) * g.mp;
                        for (int c = 0; c < tg.mp; ++c)
                            yd[(long long)(i * tg.mp + c) * 32] = c < m ? yrow[(R + c) * TC_PTS] : 0.f;
                    }
                }
                break;
            }
        }
    }
    if (s_fail) {
        if (tid == 0) atomicExch(err, 1);
        if (slot_thread && pt >= 0) status[pt] = HOPF_MAXITER;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

// ------------------------------------------------------------------ host
// ring stage: a GEMM1 chunk (pbar and K block, hi/lo: 48 KB) or a GEMM2 chunk
// (K^T block, hi/lo: 256 n2 bytes), whichever is larger
static int tc_stage_bytes(const TcGeom &g) {
    const int g1 = TC_G1_BLO + TC_NB * TC_KC * 4, g2 = 2 * g.n2 * TC_RC * 4;
    return ((g1 > g2 ? g1 : g2) + 1023) & ~1023;
}
static int tc_stages(const TcGeom &g, size_t smem_limit) {
    const long long room = (long long)smem_limit - TC_YBYTES - 4096;
    const long long s = room / tc_stage_bytes(g);
    return s >= TC_MAX_STAGES ? TC_MAX_STAGES : (int)s;
}

bool tc_plan(int n, int m, int N, int P, int sms, size_t smem_limit, int *grid) {
    if (n < 16 || n > 256 || m < 1 || m > 16 || N < 1 || P < 1) return false;
    const TcGeom g = tc_geom(n, m, N);
    const int stages = tc_stages(g, smem_limit);
    if (stages < 2) return false;
    // the re-check gathers pbar, x0, y and keeps the row products (float64) in the ring
    if ((2LL * g.n1 + 3LL * g.rows + 2) * 4 > (long long)stages * tc_stage_bytes(g)) return false;
    const int tiles = (P + TC_PTS - 1) / TC_PTS;
    *grid = tiles < sms ? tiles : sms;
    return true;
}

// points parked by the drain, for the tail kernel (the tiled kernel's layouts):
// padded table, state records, [count, tail queue, -, -] + point list, dual rows
static long long tc_park_floats(int n, int m, int N, int grid) {
    const TileGeom tg = tile_geom(n, m, N, 1);
    const long long cap = 32LL * grid;
    return tile_pad_floats(n, m, N) + 64 + cap * (2 * tg.n4 + 4) + 64 + 4 + 2 * cap + 64 +
           cap * (long long)tg.chunks * tg.cr + 64;
}

long long tc_workspace_floats(int n, int m, int N, int grid) {
    const TcGeom g = tc_geom(n, m, N);
    return tc_k1_floats(g) + tc_k2_floats(g) + 4LL * g.rows * g.n1 + 3LL * g.n1 + 6LL * g.n1 + 64 +
           (long long)grid * tc_slot_floats(g) + 64 + tc_park_floats(n, m, N, grid);
}

template <int MP>
static cudaError_t launch_tc_t(const TcGeom &g, const TcImages &im, const float *inst, const double *inst64,
                               const SolveParams &prm, const float *x, const float *p_init, float *phi, float *pstar,
                               float *gap, int *iters, int *status, float *slots, int *queue, int grid,
                               float *park_st, int *park_list, int *park_count, float *park_y, cudaStream_t s) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int stages = tc_stages(g, (size_t)optin - 2048), sb = tc_stage_bytes(g);
    const int smem = stages * sb + TC_YBYTES;
    e = cudaFuncSetAttribute(pdhg_tc_kernel<MP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    pdhg_tc_kernel<MP><<<grid, TC_THREADS, smem, s>>>(g, im, inst, inst64, prm, x, p_init, phi, pstar, gap, iters,
                                                       status, slots, queue, queue + 1, stages, sb, park_st, park_list,
                                                       park_count, park_y);
    return cudaGetLastError();
}

cudaError_t launch_pdhg_tc(const float *inst, const double *inst64, const SolveParams &prm, const float *x,
                           const float *p_init, float *phi, float *pstar, float *gap, int *iters, int *status, float *ws,
                           int *queue, int grid, cudaStream_t s) {
    const int n = prm.n, m = prm.m, N = prm.N;
    const TcGeom g = tc_geom(n, m, N);
    TcImages im;
    float *p = ws;
    im.K1 = p;  p += tc_k1_floats(g);
    im.K2 = p;  p += tc_k2_floats(g);
    im.Kh = p;  p += g.rows * g.n1;
    im.Kl = p;  p += g.rows * g.n1;
    im.KTh = p; p += (long long)n * g.rows;
    im.KTl = p; p += (long long)n * g.rows;
    p += g.rows * g.n1 * 2 - 2LL * n * g.rows;          // keep the carve of tc_workspace_floats
    im.d32 = p; p += 3LL * g.n1;
    p = reinterpret_cast<float *>(((uintptr_t)p + 63) & ~(uintptr_t)63);
    im.d64 = reinterpret_cast<double *>(p);
    p += 6LL * g.n1;
    p = reinterpret_cast<float *>(((uintptr_t)p + 255) & ~(uintptr_t)255);
    float *slots = p;
    p += (long long)grid * tc_slot_floats(g);
    // drain parking (tail kernel in the tiled layout), when its shared memory fits
    const TileGeom tg = tile_geom(n, m, N, 1);
    const bool park = tile_tail_smem(n, m, N, 1) <= 200 * 1024;
    const long long cap = 32LL * grid;
    p = reinterpret_cast<float *>(((uintptr_t)p + 255) & ~(uintptr_t)255);
    float *tile_ws = p;
    p += tile_pad_floats(n, m, N);
    p = reinterpret_cast<float *>(((uintptr_t)p + 255) & ~(uintptr_t)255);
    float *park_st = p;
    p += cap * (2 * tg.n4 + 4);
    p = reinterpret_cast<float *>(((uintptr_t)p + 255) & ~(uintptr_t)255);
    int *park_ctr = reinterpret_cast<int *>(p);          // [0] parked count, [1] tail queue
    int *park_list = park_ctr + 4;
    p += 4 + 2 * cap;
    p = reinterpret_cast<float *>(((uintptr_t)p + 255) & ~(uintptr_t)255);
    float *park_y = p;
    cudaError_t e = cudaMemsetAsync(queue, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(park_ctr, 0, 4 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    tc_prep_kernel<<<512, 256, 0, s>>>(inst64, n, m, N, g, im);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float *pst = park ? park_st : nullptr, *py = park ? park_y : nullptr;
    int *pl = park ? park_list : nullptr;
    switch (g.mp) {
        case 2: e = launch_tc_t<2>(g, im, inst, inst64, prm, x, p_init, phi, pstar, gap, iters, status, slots, queue, grid, pst, pl, park_ctr, py, s); break;
        case 4: e = launch_tc_t<4>(g, im, inst, inst64, prm, x, p_init, phi, pstar, gap, iters, status, slots, queue, grid, pst, pl, park_ctr, py, s); break;
        case 8: e = launch_tc_t<8>(g, im, inst, inst64, prm, x, p_init, phi, pstar, gap, iters, status, slots, queue, grid, pst, pl, park_ctr, py, s); break;
        case 10: e = launch_tc_t<10>(g, im, inst, inst64, prm, x, p_init, phi, pstar, gap, iters, status, slots, queue, grid, pst, pl, park_ctr, py, s); break;
        default: e = launch_tc_t<16>(g, im, inst, inst64, prm, x, p_init, phi, pstar, gap, iters, status, slots, queue, grid, pst, pl, park_ctr, py, s); break;
    }
    if (e != cudaSuccess || !park) return e;
    // the parked points: one 256-thread block each (up to four per SM)
    SolveParams pt = prm;
    pt.carry_cap = 0;
    pt.out_st = park_st;
    pt.out_list = park_list;
    pt.out_count = park_ctr;
    pt.list = nullptr;
    pt.list_count = nullptr;
    return launch_tile_tail_parked(inst, inst64, pt, x, phi, pstar, gap, iters, status, tile_ws, park_y, park_ctr + 1,
                                   4 * grid, s);
}

}  // namespace hopf
