// C ABI entry points (include/hopf.h): argument checks, workspace, launches.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <map>
#include <vector>

#include "common.cuh"

namespace hopf {
// host launchers (defined next to their kernels)
cudaError_t launch_build_instances(int grid, int threads, cudaStream_t s, const double *A, const double *B,
                                   const double *qd, const double *W, const double *Tv, const int *active,
                                   int n_inst, int n, int m, int N, int rule, double tau, double sigma_scale,
                                   double *out64, float *out32, double *scratch);
cudaError_t launch_horizons(int count, cudaStream_t s, const void *t, bool t_is_float, double *Tv);
template <typename R>
cudaError_t launch_pdhg_generic(const R *inst, const SolveParams &prm, const R *x, const R *p_init, R *phi,
                                R *pstar, R *gap, int *iters, int *status, R *Pv, R *Dv, R *y,
                                const int *active, cudaStream_t s);
bool tile_plan(int n, int m, int N, int P, int sms, size_t smem_limit, int *ppt, int *grid, size_t *smem,
               int *dbuf);
long long tile_workspace_floats(int n, int m, int N, int ppt, int grid);
cudaError_t launch_pdhg_tile(const float *inst, const double *inst64, const SolveParams &prm, const float *x,
                             const float *p_init, float *phi, float *pstar, float *gap, int *iters, int *status,
                             float *ws, int *queue, int ppt, int grid, size_t smem, int dbuf, float *carry_st,
                             int *carry_list, cudaStream_t s, float *Pout = nullptr, float *Dout = nullptr);
long long tile_carry_floats(int n, int m, int N, int ppt, int P);
bool tc_plan(int n, int m, int N, int P, int sms, size_t smem_limit, int *grid);
long long tc_workspace_floats(int n, int m, int N, int grid);
cudaError_t launch_pdhg_tc(const float *inst, const double *inst64, const SolveParams &prm, const float *x,
                           const float *p_init, float *phi, float *pstar, float *gap, int *iters, int *status, float *ws,
                           int *queue, int grid, cudaStream_t s);
cudaError_t launch_build_instances_opt(int grid, int threads, cudaStream_t s, const double *A, const double *B,
                                       const double *qd, const double *W, const double *Tv, const int *active,
                                       int n_inst, int n, int m, int N, int rule, double tau, double sigma_scale,
                                       double *out64, float *out32, double *scratch, int need_eig, int terminal,
                                       double *gram_snap, int snap);
int fixed_powers_count(int N);
cudaError_t launch_fixed_lam(const double *snaps, int nsnap, int n, double *lam, double *scratch, cudaStream_t s);
cudaError_t launch_fixed_powers(const double *A, int n, double dt, int J, double *Ep, double *Em, double *scratch,
                                cudaStream_t s);
template <typename R>
cudaError_t launch_fixed_prep(int P, const double *Tv, int t_stride, double t_max, double dt, int N, double tau,
                              double sigma_scale, const double *lam, int snap, const int *active, int *nk,
                              double *wl, double *sig, int n, R *phi, R *pstar, R *gap, int *iters, int *status,
                              cudaStream_t s);
template <typename R>
cudaError_t launch_fixed_map(int mode, int P, int n, const double *A, double anorm, const double *pw, int J,
                             const int *nk, const double *wl, const R *in, R *out, const int *active, int sms,
                             cudaStream_t s);
template <typename R>
cudaError_t launch_to_terminal(const double *inst64, int n, int m, int N, int inst_stride, int P, const R *x,
                               const R *p0, R *xq, R *q0, const int *active, cudaStream_t s);
template <typename R>
cudaError_t launch_from_terminal(const double *inst64, int n, int m, int N, int inst_stride, int P, const R *q,
                                 R *p, const int *active, cudaStream_t s);
cudaError_t launch_build_instances_wblocks(int grid, int threads, cudaStream_t s, const double *A, const double *B,
                                           const double *qd, const double *W, int w_count, const double *Tv,
                                           int n_inst, int n, int m, int N, int rule, double tau,
                                           double sigma_scale, double *out64, float *out32, double *scratch);
template <typename R>
cudaError_t launch_pdhg_stacked(const R *inst, const SolveParams &prm, int k, const R *x, const R *p_init, R *phi,
                                R *pstar, R *gap, int *iters, int *status, R *y, cudaStream_t s);
cudaError_t launch_tc_selftest(int N, int K, const float *A, const float *B, float *D, int *err, cudaStream_t s);
cudaError_t launch_pdhg_cta(int NS, int m, int grid, cudaStream_t s, const float *inst, const SolveParams &prm,
                            const float *x, float *phi, float *pstar, float *gap, int *iters, int *status,
                            int *counter);
cudaError_t launch_pdhg_small(int NS, int m, int tpp, int grid, int threads, size_t smem, cudaStream_t s,
                              const float *inst, const SolveParams &prm, int ys_stride, const float *x,
                              const float *p_init, float *phi, float *pstar, float *gap, int *iters,
                              int *status, int *counter);
template <typename R>
cudaError_t launch_ttr_init(int P, cudaStream_t s, const double *inst0, int n, int m, int N, const R *x,
                            const R *T_lo, const R *T_hi, double t_max, double *lo, double *hi, int *phase,
                            int *warm, int *st, double *Tfinal);
cudaError_t launch_ttr_newton_start(int P, cudaStream_t s, const double *hi, const int *phase, double *cand,
                                    int *active);
template <typename R>
cudaError_t launch_ttr_newton_update(int P, cudaStream_t s, int n, int m, int ctrl_kind, const double *A,
                                     const double *B, const double *qd, const R *x, double t_max, double tol_T,
                                     const R *Pv, const R *Dv, const R *pstar, double *cand, int *active, double *lo,
                                     double *hi, int *phase, int *st, double *Tfinal, int *remaining);
cudaError_t launch_ttr_candidates(int P, cudaStream_t s, const double *lo, const double *hi, const int *phase,
                                  double *cand, int *active);
template <typename R>
cudaError_t launch_ttr_update(int P, cudaStream_t s, double t_max, double tol_T, const double *cand,
                              const int *active, const R *Pv, const R *Dv, const int *sst, double *lo,
                              double *hi, int *phase, int *warm, int *st, double *Tfinal, int *remaining);
cudaError_t launch_ttr_cap(int P, cudaStream_t s, const double *hi, int *phase, int *st, double *Tfinal);
template <typename R>
cudaError_t launch_ttr_finish(int P, cudaStream_t s, const int *st, const int *fst, const double *Tfinal,
                              R *T_star, int *status);
template <typename R>
cudaError_t launch_trajectory(int grid, int threads, cudaStream_t s, const double *A, const double *B,
                              const double *qd, int n, int m, int ctrl_kind, int P, const R *x, const R *T,
                              const R *pstar, int S, R *xt, R *ut, double *scratch, const double *Eh_sh,
                              const double *G_sh);
template <typename R>
cudaError_t launch_traj_minmax(int P, const R *T, double *out, cudaStream_t s);
cudaError_t launch_traj_shared_expm(int threads, const double *A, int n, int S, const double *TT, double *Eh,
                                    double *G, double *scratch, cudaStream_t s);
long long mlp_param_count(int n_in, int h, int n_out);
long long mlp_scratch_floats(int n_in, int h, int n_out, int B, bool train);
cudaError_t mlp_forward(int n_in, int h, int n_out, const __nv_bfloat16 *wb, const float *w, const float *x_shift,
                        const float *x_scale, const float *y_shift, const float *y_scale, int B, const float *x,
                        float *y, float *scratch, bool keep_pre, cudaStream_t s);
cudaError_t mlp_forward_tc(int n_in, int h, int n_out, const __nv_bfloat16 *wb, const float *w,
                           const float *x_shift, const float *x_scale, const float *y_shift, const float *y_scale,
                           int B, const float *x, float *y, float *scratch, int *err, cudaStream_t s);
cudaError_t mlp_loss_grad(int n_in, int h, int n_out, const __nv_bfloat16 *wb, const float *w, const float *x_shift,
                          const float *x_scale, const float *y_shift, const float *y_scale, int B, const float *x,
                          const float *y, float *loss, float *grad, float *scratch, cudaStream_t s);
cudaError_t mlp_adam(long long count, float *w, __nv_bfloat16 *wb, const float *g, float *m, float *v, float lr,
                     float b1, float b2, float eps, int step, cudaStream_t s);
cudaError_t mlp_sync_bf16(long long count, const float *w, __nv_bfloat16 *wb, cudaStream_t s);

// Hardest-first order for the warm solve: points whose predicted p* is small
// take the most iterations (the relative gap then asks for a small absolute
// gap), so they are started first.  Buckets of |p_hat|^2 by powers of two,
// ascending; order within a bucket unspecified.
constexpr int ORDER_BUCKETS = 64;
__global__ void order_count_kernel(int P, int n, const float *phat, int *bucket, int *counts) {
    __shared__ int h[ORDER_BUCKETS];
    for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P) {
        float s = 0.f;
        for (int j = 0; j < n; ++j) {
            float v = phat[(long long)k * n + j];
            s = fmaf(v, v, s);
        }
        int e = 0;
        frexpf(s, &e);                         // s = f 2^e, f in [0.5, 1)
        int b = s > 0.f ? e + 32 : 0;
        b = b < 0 ? 0 : (b >= ORDER_BUCKETS ? ORDER_BUCKETS - 1 : b);
        bucket[k] = b;
        atomicAdd(&h[b], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x)
        if (h[i]) atomicAdd(&counts[i], h[i]);
}
__global__ void order_scan_kernel(int P, int hard, int *counts, int *total) {
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < ORDER_BUCKETS; ++i) {
            int c = counts[i];
            counts[i] = run;                   // exclusive prefix: cursor of bucket i
            run += c;
        }
        total[0] = P;                          // whole list
        total[1] = hard;                       // hardest points (latency kernel)
        total[2] = P - hard;                   // the rest (throughput kernel)
    }
}
__global__ void order_scatter_kernel(int P, const int *bucket, int *cursor, int *list) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P) list[atomicAdd(&cursor[bucket[k]], 1)] = k;
}

// list of the points whose status is not OK (order unspecified)
__global__ void failed_points_kernel(int P, const int *status, int *list, int *count) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P && status[k] != HOPF_OK) list[atomicAdd(count, 1)] = k;
}

// list of the active points (order unspecified)
__global__ void active_points_kernel(int P, const int *active, int *list, int *count) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P && active[k]) list[atomicAdd(count, 1)] = k;
}

// dst row k = src row k for the active points (all when active is null)
template <typename R>
__global__ void copy_rows_kernel(int P, int n, const int *active, const R *src, R *dst) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)P * n) return;
    const int k = (int)(e / n);
    if (!active || active[k]) dst[e] = src[e];
}
template <typename R>
cudaError_t launch_copy_rows(int P, int n, const int *active, const R *src, R *dst, cudaStream_t s) {
    const long long total = (long long)P * n;
    copy_rows_kernel<R><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(P, n, active, src, dst);
    return cudaGetLastError();
}
}  // namespace hopf

using namespace hopf;

namespace {

thread_local std::string g_err;
std::mutex g_mu;

struct Workspace {
    void *ptr = nullptr;
    size_t size = 0;
};
// one grow-only workspace per (device, stream): calls on one stream reuse it
// in stream order; calls on different streams may run concurrently
std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;


// events of the last profiled hopf_value call
struct Profile {
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    int device = -1;
    bool valid = false;
} g_prof;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                                \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(HOPF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// side stream and fork/join events per device (the warm solve runs its
// hardest points concurrently with the rest)
struct Side {
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
std::vector<Side> g_side;

int side_stream(int dev, Side **out) {
    if ((int)g_side.size() <= dev) g_side.resize(dev + 1);
    Side &sd = g_side[dev];
    if (!sd.stream) {
        CU(cudaStreamCreateWithFlags(&sd.stream, cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&sd.fork, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&sd.join, cudaEventDisableTiming));
    }
    *out = &sd;
    return HOPF_SUCCESS;
}

// Bump allocator over the device workspace; a first pass with base == nullptr
// only measures.
struct Arena {
    char *base;
    size_t off = 0;
    explicit Arena(void *b) : base((char *)b) {}
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

int ensure_workspace(size_t bytes, void **out, cudaStream_t stream) {
    int dev = 0;
    CU(cudaGetDevice(&dev));
    Workspace &w = g_ws[std::make_pair(dev, stream)];
    if (w.size < bytes) {
        if (w.ptr) {
            CU(cudaStreamSynchronize(stream));
            CU(cudaFree(w.ptr));
            w.ptr = nullptr;
            w.size = 0;
        }
        size_t want = bytes + bytes / 4 + (1 << 20);
        if (cudaMalloc(&w.ptr, want) != cudaSuccess) {
            cudaGetLastError();
            w.ptr = nullptr;
            return fail(HOPF_ENOMEM, "cudaMalloc of %zu bytes failed", want);
        }
        w.size = want;
    }
    *out = w.ptr;
    return HOPF_SUCCESS;
}

bool all_finite(const double *a, long long count) {
    for (long long i = 0; i < count; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

// Host-side argument check: W symmetric positive definite (Cholesky).
bool is_spd(const double *W, int n) {
    std::vector<double> L((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (std::fabs(W[i * n + j] - W[j * n + i]) > 1e-12 * (1.0 + std::fabs(W[i * n + j]))) return false;
    for (int j = 0; j < n; ++j) {
        double d = W[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (!(d > 0.0)) return false;
        L[j * n + j] = std::sqrt(d);
        for (int i = j + 1; i < n; ++i) {
            double s = W[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = s / L[j * n + j];
        }
    }
    return true;
}

int check_problem(const hopf_problem *pr, const hopf_opts *o, bool need_solver) {
    if (!pr || !o) return fail(HOPF_EINVAL, "null problem or options");
    if (pr->n < 1 || pr->m < 1 || pr->n > 4096 || pr->m > 16)
        return fail(HOPF_EINVAL, "unsupported sizes n=%d m=%d (1<=n<=4096, 1<=m<=16)", pr->n, pr->m);
    if (!pr->A || !pr->B || !pr->W) return fail(HOPF_EINVAL, "A, B and W are required");
    if (pr->ctrl_kind != HOPF_BALL && pr->ctrl_kind != HOPF_BOX)
        return fail(HOPF_EINVAL, "ctrl_kind must be HOPF_BALL or HOPF_BOX");
    if (pr->ctrl_kind == HOPF_BALL && !(pr->radius > 0.0 && std::isfinite(pr->radius)))
        return fail(HOPF_EINVAL, "ball radius must be positive and finite");
    if (pr->ctrl_kind == HOPF_BOX) {
        if (!pr->half_widths) return fail(HOPF_EINVAL, "box control needs half_widths");
        for (int c = 0; c < pr->m; ++c)
            if (!(pr->half_widths[c] > 0.0) || !std::isfinite(pr->half_widths[c]))
                return fail(HOPF_EINVAL, "half_widths must be positive and finite");
    }
    const long long n = pr->n, m = pr->m;
    if (!all_finite(pr->A, n * n) || !all_finite(pr->B, n * m) || !all_finite(pr->W, n * n))
        return fail(HOPF_ENONFINITE, "A, B or W has a non-finite entry");
    if (!is_spd(pr->W, pr->n)) return fail(HOPF_ENOTSPD, "W is not symmetric positive definite");
    if (o->precision != HOPF_FP64 && o->precision != HOPF_FP32) return fail(HOPF_EINVAL, "bad precision");
    if (need_solver) {
        if (o->rule != HOPF_LEFT_RIEMANN && o->rule != HOPF_TRAPEZOID && o->rule != HOPF_SIMPSON &&
            o->rule != HOPF_LEFT_FIXED)
            return fail(HOPF_EINVAL, "bad rule");
        if (o->N < 1 || (o->rule == HOPF_TRAPEZOID && o->N < 2) ||
            (o->rule == HOPF_SIMPSON && (o->N < 3 || o->N % 2 == 0)) || o->N > (1 << 20))
            return fail(HOPF_EINVAL, "bad node count N=%d", o->N);
        if (o->max_iter < 0 || o->gap_every < 1) return fail(HOPF_EINVAL, "bad max_iter or gap_every");
        if (!(o->tau > 0.0) || !(o->sigma_scale > 0.0) || !(o->sigma_scale <= 1.0))
            return fail(HOPF_EINVAL, "need tau > 0 and 0 < sigma_scale <= 1");
        if (!(o->tol_gap >= 0.0)) return fail(HOPF_EINVAL, "bad tol_gap");
        if (o->accel != 0 && o->accel != 1) return fail(HOPF_EINVAL, "accel must be 0 or 1");
        if (o->newton != 0 && o->newton != 1) return fail(HOPF_EINVAL, "newton must be 0 or 1");
        if (o->kernel != HOPF_KERNEL_AUTO && o->kernel != HOPF_KERNEL_GENERIC && o->kernel != HOPF_KERNEL_TENSOR &&
            o->kernel != HOPF_KERNEL_TILE)
            return fail(HOPF_EINVAL, "kernel must be one of HOPF_KERNEL_AUTO, _GENERIC, _TENSOR, _TILE");
        if (o->variables != HOPF_VARS_INITIAL && o->variables != HOPF_VARS_TERMINAL)
            return fail(HOPF_EINVAL, "variables must be HOPF_VARS_INITIAL or HOPF_VARS_TERMINAL");
        if (o->adaptive != 0 && o->adaptive != 1) return fail(HOPF_EINVAL, "adaptive must be 0 or 1");
        if (o->adaptive && o->accel) return fail(HOPF_EINVAL, "adaptive and accel exclude each other");
        if (o->rule == HOPF_LEFT_FIXED) {
            if (o->variables != HOPF_VARS_TERMINAL)
                return fail(HOPF_EINVAL, "the fixed-step rule needs terminal-time variables");
            if (!(o->t_max > 0.0) || !std::isfinite(o->t_max))
                return fail(HOPF_EINVAL, "the fixed-step rule needs a finite t_max > 0");
            if (o->adaptive) return fail(HOPF_EINVAL, "the fixed-step rule runs fixed step sizes (adaptive = 0)");
            if (pr->n > 512) return fail(HOPF_EINVAL, "the fixed-step rule supports n <= 512");
        }
    }
    return HOPF_SUCCESS;
}

struct Device {
    int id = 0, sms = 0;
    size_t smem_optin = 0;
};

int query_device(Device *d) {
    CU(cudaGetDevice(&d->id));
    CU(cudaDeviceGetAttribute(&d->sms, cudaDevAttrMultiProcessorCount, d->id));
    int v = 0;
    CU(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, d->id));
    d->smem_optin = (size_t)v;
    return HOPF_SUCCESS;
}

// Problem matrices on the device (float64), Q diagonal folded separately.
struct DevProblem {
    double *A, *B, *q, *W;
};

template <typename AR>
DevProblem take_problem(AR &a, int n, int m) {
    DevProblem d;
    d.A = a.template take<double>((size_t)n * n);
    d.B = a.template take<double>((size_t)n * m);
    d.q = a.template take<double>((size_t)m);
    d.W = a.template take<double>((size_t)n * n);
    return d;
}

int upload_problem(const DevProblem &d, const hopf_problem *pr, cudaStream_t s) {
    const int n = pr->n, m = pr->m;
    std::vector<double> q(m);
    for (int c = 0; c < m; ++c) q[c] = pr->ctrl_kind == HOPF_BALL ? pr->radius : pr->half_widths[c];
    CU(cudaMemcpyAsync(d.A, pr->A, sizeof(double) * n * n, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(d.B, pr->B, sizeof(double) * n * m, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(d.q, q.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(d.W, pr->W, sizeof(double) * n * n, cudaMemcpyHostToDevice, s));
    // the staging vector q lives until the copy has been issued from pageable
    // memory, which completes before cudaMemcpyAsync returns for pageable sources
    return HOPF_SUCCESS;
}

// one warp builds a small table (its block barriers are cheap); more threads for large n
int table_threads(int n) { return n <= 16 ? 32 : (n <= 32 ? 64 : 256); }

// ------------------------------------------------------------ small kernel
constexpr int SMALL_MAX_THREADS = 384;
// Multi-phase solve: a point moves on to the next (lower-latency) phase after
// this many iterations, or as soon as its phase has no new point left.
constexpr int SMALL_PARK_ITERS = 4096;

struct SmallPlan {
    bool ok = false;
    int NS = 0, pts = 0, threads = 0, ys_stride = 0, grid = 0, tpp = 4;
    size_t smem = 0;
};

SmallPlan plan_small(const Device &dev, int n, int m, int N, int P, int tpp = 4) {
    const int SMALL_TPP = tpp;
    SmallPlan sp;
    sp.tpp = tpp;
    if (n > 16 || m > 2) return sp;
    sp.NS = (n + 1) & ~1;
    const int KR = (m * sp.NS + 1 + 3) & ~3;
    int pad = 0;
    while ((((N + pad) * m) % 32) != ((SMALL_TPP * m) % 32)) ++pad;
    sp.ys_stride = (N + pad) * m;
    const size_t fixed = sizeof(float) * ((size_t)N * KR + 4 * sp.NS * sp.NS + ((sp.NS + 3) & ~3));
    const size_t per_pt = sizeof(float) * ((size_t)sp.ys_stride + sp.NS);
    const size_t budget = dev.smem_optin;
    if (fixed + 8 * per_pt > budget) return sp;
    int pts = (int)((budget - fixed) / per_pt);
    pts = std::min(pts, SMALL_MAX_THREADS / SMALL_TPP);
    pts -= pts % std::max(1, 32 / SMALL_TPP);
    if (pts < std::max(1, 32 / SMALL_TPP)) return sp;
    sp.pts = pts;
    sp.threads = pts * SMALL_TPP;
    sp.smem = fixed + (size_t)pts * per_pt;
    int want = (P + pts - 1) / pts;
    sp.grid = std::max(1, std::min(dev.sms, want));
    sp.ok = true;
    return sp;
}

struct CarryBufs {
    float *y = nullptr, *st = nullptr;
    int *list = nullptr, *count = nullptr;
};
struct CarryPair {
    CarryBufs a, b;
    int *ctr = nullptr;   // [3] point counters of the three phases
};

template <typename AR>
CarryPair take_carry(AR &ar, int P, int N, int m) {
    CarryPair cp;
    for (CarryBufs *cb : {&cp.a, &cp.b}) {
        cb->y = ar.template take<float>((size_t)P * N * m);
        cb->st = ar.template take<float>((size_t)P * CARRY_W);
        cb->list = ar.template take<int>(P);
        cb->count = ar.template take<int>(4);
    }
    cp.ctr = ar.template take<int>(4);
    return cp;
}

// Small-state float32 solve in up to three phases:
//   1. 4 lanes per point (throughput); points uncertified after park_iters
//      iterations are parked;
//   2. 32 lanes per point resumes them; points still uncertified after
//      4 park_iters more are parked again;
//   3. one 256-thread block per point (latency) finishes the rest.
int run_small_two_phase(const SmallPlan &sp, const SmallPlan &sp32, int m, const float *inst, SolveParams prm,
                        const float *x, const float *pinit, float *phi, float *pstar, float *gap, int *iters,
                        int *status, const CarryPair &cp, int park_iters, cudaStream_t s) {
    CU(cudaMemsetAsync(cp.ctr, 0, 3 * sizeof(int), s));
    CU(cudaMemsetAsync(cp.a.count, 0, sizeof(int), s));
    CU(cudaMemsetAsync(cp.b.count, 0, sizeof(int), s));
    const bool multi = sp32.ok && park_iters >= 0 && prm.N <= 512;
    const int cap = park_iters > 0 ? park_iters : SMALL_PARK_ITERS;
    prm.carry_cap = multi ? cap : 0;
    prm.carry_in = 0;
    prm.out_y = cp.a.y;
    prm.out_st = cp.a.st;
    prm.out_list = cp.a.list;
    prm.out_count = cp.a.count;
    CU(launch_pdhg_small(sp.NS, m, sp.tpp, sp.grid, sp.threads, sp.smem, s, inst, prm, sp.ys_stride, x, pinit, phi,
                         pstar, gap, iters, status, cp.ctr));
    if (!multi) return HOPF_SUCCESS;
    prm.carry_in = 1;
    prm.in_y = cp.a.y;
    prm.in_st = cp.a.st;
    prm.in_list = cp.a.list;
    prm.in_count = cp.a.count;
    prm.carry_cap = 5 * cap;
    prm.out_y = cp.b.y;
    prm.out_st = cp.b.st;
    prm.out_list = cp.b.list;
    prm.out_count = cp.b.count;
    CU(launch_pdhg_small(sp32.NS, m, sp32.tpp, sp32.grid, sp32.threads, sp32.smem, s, inst, prm, sp32.ys_stride, x,
                         pinit, phi, pstar, gap, iters, status, cp.ctr + 1));
    prm.carry_cap = 0;
    prm.in_y = cp.b.y;
    prm.in_st = cp.b.st;
    prm.in_list = cp.b.list;
    prm.in_count = cp.b.count;
    CU(launch_pdhg_cta(sp.NS, m, 2 * sp32.grid, s, inst, prm, x, phi, pstar, gap, iters, status, cp.ctr + 2));
    return HOPF_SUCCESS;
}

void fill_params(SolveParams &prm, const hopf_problem *pr, const hopf_opts *o, int P) {
    prm = SolveParams{};
    prm.n = pr->n;
    prm.m = pr->m;
    prm.N = o->N;
    prm.P = P;
    prm.ctrl_kind = pr->ctrl_kind;
    prm.max_iter = o->max_iter;
    prm.gap_every = o->gap_every;
    prm.warm = 0;
    prm.sign_mode = 0;
    prm.inst_stride = 0;
    prm.accel = o->accel;
    prm.adaptive = o->adaptive;
    prm.tau = o->tau;
    prm.tol_gap = o->tol_gap;
    prm.sign_floor = o->precision == HOPF_FP64 ? 1e-13 : 1e-6;
}

template <typename R>
int launch_generic(const R *inst, const SolveParams &prm, const R *x, const R *p_init, R *phi, R *pstar,
                   R *gap, int *iters, int *status, R *Pv, R *Dv, R *y, const int *active,
                   cudaStream_t s) {
    CU(launch_pdhg_generic<R>(inst, prm, x, p_init, phi, pstar, gap, iters, status, Pv, Dv, y, active, s));
    return HOPF_SUCCESS;
}

int launch_tables(const DevProblem &d, const hopf_problem *pr, const hopf_opts *o, const double *Tv,
                  const int *active, int n_inst, double *inst64, float *inst32, double *scratch, int grid,
                  cudaStream_t s) {
    CU(launch_build_instances_opt(grid, table_threads(pr->n), s, d.A, d.B, d.q, d.W, Tv, active, n_inst, pr->n,
                                  pr->m, o->N, o->rule, o->tau, o->sigma_scale, inst64, inst32, scratch,
                                  o->accel || o->adaptive, o->variables == HOPF_VARS_TERMINAL, nullptr, 0));
    return HOPF_SUCCESS;
}

int table_grid(const Device &dev, int n_inst) { return std::max(1, std::min(n_inst, 4 * dev.sms)); }

bool diagonal(const double *W, int n) {
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            if (a != b && W[a * n + b] != 0.0) return false;
    return true;
}

// The tensor-core kernel: float32, one shared table, terminal-time variables
// with a diagonal W (diagonal M', V', S'), plain steps (Eq. 15), 16 <= n <= 256.
// Chosen automatically when the batch fills at least half of the SMs with
// 128-point tiles; HOPF_KERNEL_TENSOR asks for it whenever it applies.
bool want_tc(const hopf_problem *pr, const hopf_opts *o, int t_stride, int P, const Device &dev, int *grid) {
    if (o->precision != HOPF_FP32 || t_stride != 0 || o->accel || o->variables != HOPF_VARS_TERMINAL) return false;
    if (o->kernel != HOPF_KERNEL_AUTO && o->kernel != HOPF_KERNEL_TENSOR) return false;
    if (o->kernel == HOPF_KERNEL_AUTO && (pr->n < 32 || P < 64 * dev.sms)) return false;
    if (!diagonal(pr->W, pr->n)) return false;
    return tc_plan(pr->n, pr->m, o->N, P, dev.sms, dev.smem_optin - 2048, grid);
}

// --------------------------------------------------------------- hopf_value
template <typename R>
int value_impl(const hopf_problem *pr, const hopf_opts *o, int P, const void *x_, const void *t_,
               int t_stride, const void *pinit_, void *phi_, void *pstar_, void *gap_, int *iters,
               int *status, cudaStream_t s) {
    const int n = pr->n, m = pr->m, N = o->N;
    const bool fp32 = o->precision == HOPF_FP32;
    const int n_inst = t_stride ? P : 1;
    Device dev;
    int rc = query_device(&dev);
    if (rc) return rc;
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    SmallPlan sp, sp32;
    if (fp32 && t_stride == 0 && o->kernel == HOPF_KERNEL_AUTO && !o->adaptive) {
        sp = plan_small(dev, n, m, N, P);
        sp32 = plan_small(dev, n, m, N, P, 32);
        sp32.grid = dev.sms;
    }
    // large states, one shared table: the tensor-core kernel or the tiled kernel
    int tc_grid = 0;
    const bool tcore = !sp.ok && !o->adaptive && want_tc(pr, o, t_stride, P, dev, &tc_grid);
    int tile_ppt = 0, tile_grid = 0, tile_dbuf = 0;
    size_t tile_smem = 0;
    const bool tile = fp32 && t_stride == 0 && !tcore && !sp.ok && !o->adaptive &&
                      (o->kernel == HOPF_KERNEL_AUTO || o->kernel == HOPF_KERNEL_TILE) &&
                      tile_plan(n, m, N, P, dev.sms, dev.smem_optin - 2048, &tile_ppt, &tile_grid, &tile_smem,
                                &tile_dbuf);
    const int tgrid = table_grid(dev, n_inst);
    const bool hio = o->host_io != 0;
    const bool term = o->variables == HOPF_VARS_TERMINAL;
    CarryPair cb;
    R *xq = nullptr, *q0 = nullptr, *qs = nullptr;

    auto plan = [&](Arena &a, DevProblem &d, double *&Tv, double *&i64, float *&i32, double *&tsc,
                    R *&dx, R *&dt, R *&dpi, R *&dphi, R *&dps, R *&dgap, int *&dit, int *&dst, R *&y,
                    int *&ctr, float *&tws, float *&tcs, int *&tcl) {
        xq = term ? a.template take<R>((size_t)P * n) : nullptr;
        q0 = (term && pinit_) ? a.template take<R>((size_t)P * n) : nullptr;
        qs = term ? a.template take<R>((size_t)P * n) : nullptr;
        d = take_problem(a, n, m);
        Tv = a.template take<double>(n_inst);
        i64 = a.template take<double>((size_t)n_inst * L.stride);
        i32 = fp32 ? a.template take<float>((size_t)n_inst * L.stride) : nullptr;
        tsc = a.template take<double>((size_t)tgrid * table_scratch_doubles(n, m));
        dx = hio ? a.template take<R>((size_t)P * n) : (R *)x_;
        dt = hio ? a.template take<R>((size_t)n_inst) : (R *)t_;
        dpi = (hio && pinit_) ? a.template take<R>((size_t)P * n) : (R *)pinit_;
        dphi = hio ? a.template take<R>(P) : (R *)phi_;
        dps = hio ? a.template take<R>((size_t)P * n) : (R *)pstar_;
        dgap = hio ? a.template take<R>(P) : (R *)gap_;
        dit = hio ? a.template take<int>(P) : iters;
        dst = hio ? a.template take<int>(P) : status;
        y = (sp.ok || tile || tcore) ? nullptr : a.template take<R>((size_t)P * N * m);
        ctr = a.template take<int>(4);
        tws = tile ? a.template take<float>((size_t)tile_workspace_floats(n, m, N, tile_ppt, tile_grid))
                   : (tcore ? a.template take<float>((size_t)tc_workspace_floats(n, m, N, tc_grid)) : nullptr);
        tcs = tile ? a.template take<float>((size_t)tile_carry_floats(n, m, N, tile_ppt, P)) : nullptr;
        tcl = tile ? a.template take<int>((size_t)2 * P) : nullptr;
        if (sp.ok) cb = take_carry(a, P, N, m);
    };
    DevProblem d;
    double *Tv, *i64, *tsc;
    float *i32;
    R *dx, *dt, *dpi, *dphi, *dps, *dgap, *y;
    int *dit, *dst, *ctr;
    float *tws, *tcs;
    int *tcl;
    Arena meas(nullptr);
    plan(meas, d, Tv, i64, i32, tsc, dx, dt, dpi, dphi, dps, dgap, dit, dst, y, ctr, tws, tcs, tcl);
    void *base = nullptr;
    rc = ensure_workspace(meas.off, &base, s);
    if (rc) return rc;
    Arena a(base);
    plan(a, d, Tv, i64, i32, tsc, dx, dt, dpi, dphi, dps, dgap, dit, dst, y, ctr, tws, tcs, tcl);

    rc = upload_problem(d, pr, s);
    if (rc) return rc;
    if (hio) {
        CU(cudaMemcpyAsync(dx, x_, sizeof(R) * P * n, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(dt, t_, sizeof(R) * n_inst, cudaMemcpyHostToDevice, s));
        if (pinit_) CU(cudaMemcpyAsync(dpi, pinit_, sizeof(R) * P * n, cudaMemcpyHostToDevice, s));
    }
    const bool prof = o->profile != 0;
    if (prof) {
        if (g_prof.device != dev.id) {
            for (auto &e : g_prof.ev)
                if (e) cudaEventDestroy(e);
            for (auto &e : g_prof.ev) CU(cudaEventCreate(&e));
            g_prof.device = dev.id;
        }
        g_prof.valid = false;
        CU(cudaEventRecord(g_prof.ev[0], s));
    }
    CU(launch_horizons(n_inst, s, dt, fp32, Tv));
    rc = launch_tables(d, pr, o, Tv, nullptr, n_inst, i64, i32, tsc, tgrid, s);
    if (rc) return rc;

    // terminal-time variables: the iteration sees e^{TA} x and e^{-TA^T} p_init
    // and returns q*, mapped back to p* = e^{TA^T} q* after the solve
    const R *sx = dx, *spi = dpi;
    R *sps = dps;
    if (term) {
        CU(launch_to_terminal<R>(i64, n, m, N, t_stride ? 1 : 0, P, dx, dpi, xq, q0, nullptr, s));
        sx = xq;
        spi = q0;
        sps = qs;
    }
    if (prof) CU(cudaEventRecord(g_prof.ev[1], s));
    SolveParams prm;
    fill_params(prm, pr, o, P);
    prm.warm = pinit_ != nullptr;
    prm.inst_stride = t_stride ? 1 : 0;
    const R *inst = fp32 ? (const R *)i32 : (const R *)i64;
    if (sp.ok) {
        rc = run_small_two_phase(sp, sp32, m, (const float *)inst, prm, (const float *)sx, (const float *)spi,
                                 (float *)dphi, (float *)sps, (float *)dgap, dit, dst, cb, o->park_iters, s);
        if (rc) return rc;
    } else if (tcore) {
        CU(launch_pdhg_tc((const float *)inst, i64, prm, (const float *)sx, (const float *)spi, (float *)dphi,
                          (float *)sps, (float *)dgap, dit, dst, tws, ctr, tc_grid, s));
    } else if (tile) {
        CU(launch_pdhg_tile((const float *)inst, i64, prm, (const float *)sx, (const float *)spi, (float *)dphi,
                            (float *)sps, (float *)dgap, dit, dst, tws, ctr, tile_ppt, tile_grid, tile_smem,
                            tile_dbuf, tcs, tcl, s));
    } else {
        rc = launch_generic<R>(inst, prm, sx, spi, dphi, sps, dgap, dit, dst, nullptr, nullptr, y, nullptr, s);
        if (rc) return rc;
    }
    if (prof) CU(cudaEventRecord(g_prof.ev[2], s));
    if (term) CU(launch_from_terminal<R>(i64, n, m, N, t_stride ? 1 : 0, P, qs, dps, nullptr, s));
    if (prof) g_prof.valid = true;
    if (hio) {
        CU(cudaMemcpyAsync(phi_, dphi, sizeof(R) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(pstar_, dps, sizeof(R) * P * n, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(gap_, dgap, sizeof(R) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(iters, dit, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(status, dst, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    return HOPF_SUCCESS;
}

// ------------------------------------------------------- hopf_value_stacked
__global__ void expand_horizons_kernel(const double *Tv, int nT, int k, double *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nT * k) out[i] = Tv[i / k];
}

template <typename R>
int stacked_impl(const hopf_stacked *sp, const hopf_opts *o, int P, const void *x_, const void *t_, int t_stride,
                 const void *pinit_, void *phi_, void *pstar_, void *gap_, int *iters, int *status,
                 cudaStream_t s) {
    const hopf_problem *pr = &sp->base;
    const int nb = pr->n, m = pr->m, N = o->N, k = sp->copies;
    if (o->variables != HOPF_VARS_INITIAL) return fail(HOPF_EINVAL, "stacked solve: variables must be HOPF_VARS_INITIAL");
    if (o->adaptive) return fail(HOPF_EINVAL, "stacked solve: adaptive steps are not supported");
    const bool fp32 = o->precision == HOPF_FP32;
    const int nT = t_stride ? P : 1;
    const int n_inst = nT * k;
    Device dev;
    int rc = query_device(&dev);
    if (rc) return rc;
    const InstanceLayout L = InstanceLayout::make(nb, m, N);
    const int tgrid = table_grid(dev, n_inst);
    DevProblem d;
    double *Wb, *Tv, *Tx, *i64, *tsc;
    float *i32;
    R *y;
    auto plan = [&](Arena &a) {
        d = take_problem(a, nb, m);
        Wb = a.template take<double>((size_t)k * nb * nb);
        Tv = a.template take<double>(nT);
        Tx = a.template take<double>(n_inst);
        i64 = a.template take<double>((size_t)n_inst * L.stride);
        i32 = fp32 ? a.template take<float>((size_t)n_inst * L.stride) : nullptr;
        tsc = a.template take<double>((size_t)tgrid * table_scratch_doubles(nb, m));
        y = a.template take<R>((size_t)P * N * m);
    };
    Arena meas(nullptr);
    plan(meas);
    void *base = nullptr;
    rc = ensure_workspace(meas.off, &base, s);
    if (rc) return rc;
    Arena a(base);
    plan(a);
    std::vector<double> q(m);
    for (int c = 0; c < m; ++c) q[c] = pr->ctrl_kind == HOPF_BALL ? pr->radius : pr->half_widths[c];
    CU(cudaMemcpyAsync(d.A, pr->A, sizeof(double) * nb * nb, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(d.B, pr->B, sizeof(double) * nb * m, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(d.q, q.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(Wb, sp->W_blocks, sizeof(double) * k * nb * nb, cudaMemcpyHostToDevice, s));
    CU(launch_horizons(nT, s, t_, fp32, Tv));
    expand_horizons_kernel<<<(n_inst + 255) / 256, 256, 0, s>>>(Tv, nT, k, Tx);
    CU(cudaGetLastError());
    CU(launch_build_instances_wblocks(tgrid, table_threads(nb), s, d.A, d.B, d.q, Wb, k, Tx, n_inst, nb, m, N,
                                      o->rule, o->tau, o->sigma_scale, i64, i32, tsc));
    SolveParams prm;
    fill_params(prm, pr, o, P);
    prm.warm = pinit_ != nullptr;
    prm.inst_stride = t_stride ? 1 : 0;
    const R *inst = fp32 ? (const R *)i32 : (const R *)i64;
    CU(launch_pdhg_stacked<R>(inst, prm, k, (const R *)x_, (const R *)pinit_, (R *)phi_, (R *)pstar_, (R *)gap_,
                              iters, status, y, s));
    return HOPF_SUCCESS;
}

// ------------------------------------------------------- hopf_time_to_reach
template <typename R>
int ttr_impl(const hopf_problem *pr, const hopf_opts *o, int P, const void *x_, const void *Tlo_,
             const void *Thi_, const void *pinit_, void *Tstar_, void *pstar_, void *gap_, int *status,
             int *steps_out, cudaStream_t s) {
    const int n = pr->n, m = pr->m, N = o->N;
    const bool fp32 = o->precision == HOPF_FP32;
    Device dev;
    int rc = query_device(&dev);
    if (rc) return rc;
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    const int tgrid = table_grid(dev, P);
    const bool hio = o->host_io != 0;
    const bool wb = Tlo_ && Thi_;

    struct Bufs {
        DevProblem d;
        double *Tz, *inst0, *i64, *tsc, *lo, *hi, *cand, *Tf;
        float *i32;
        int *phase, *warm, *st, *act, *sst, *fst, *its, *rem;
        R *Pv, *Dv, *phi, *gtmp, *ptmp, *y;
        R *dx, *dlo, *dhi, *dpi, *dTs, *dps, *dgap;
        R *xq, *q0, *qtmp;   // terminal-time variables: mapped point, warm start, solution
        int *dst;
    } b;
    const bool term = o->variables == HOPF_VARS_TERMINAL;
    auto plan = [&](Arena &a) {
        b.d = take_problem(a, n, m);
        b.Tz = a.template take<double>(1);
        b.inst0 = a.template take<double>(L.stride);
        b.i64 = a.template take<double>((size_t)P * L.stride);
        b.i32 = fp32 ? a.template take<float>((size_t)P * L.stride) : nullptr;
        b.tsc = a.template take<double>((size_t)tgrid * table_scratch_doubles(n, m));
        b.lo = a.template take<double>(P);
        b.hi = a.template take<double>(P);
        b.cand = a.template take<double>(P);
        b.Tf = a.template take<double>(P);
        b.phase = a.template take<int>(P);
        b.warm = a.template take<int>(P);
        b.st = a.template take<int>(P);
        b.act = a.template take<int>(P);
        b.sst = a.template take<int>(P);
        b.fst = a.template take<int>(P);
        b.its = a.template take<int>(P);
        b.rem = a.template take<int>(4);
        b.Pv = a.template take<R>(P);
        b.Dv = a.template take<R>(P);
        b.phi = a.template take<R>(P);
        b.gtmp = a.template take<R>(P);
        b.ptmp = a.template take<R>((size_t)P * n);
        b.y = a.template take<R>((size_t)P * N * m);
        b.dx = hio ? a.template take<R>((size_t)P * n) : (R *)x_;
        b.dlo = (hio && wb) ? a.template take<R>(P) : (R *)Tlo_;
        b.dhi = (hio && wb) ? a.template take<R>(P) : (R *)Thi_;
        b.dpi = (hio && pinit_) ? a.template take<R>((size_t)P * n) : (R *)pinit_;
        b.dTs = hio ? a.template take<R>(P) : (R *)Tstar_;
        b.dps = hio ? a.template take<R>((size_t)P * n) : (R *)pstar_;
        b.dgap = hio ? a.template take<R>(P) : (R *)gap_;
        b.dst = hio ? a.template take<int>(P) : status;
        b.xq = term ? a.template take<R>((size_t)P * n) : nullptr;
        b.q0 = term ? a.template take<R>((size_t)P * n) : nullptr;
        b.qtmp = term ? a.template take<R>((size_t)P * n) : nullptr;
    };
    Arena meas(nullptr);
    plan(meas);
    void *base = nullptr;
    rc = ensure_workspace(meas.off, &base, s);
    if (rc) return rc;
    Arena a(base);
    plan(a);
    // one solve of the points act (all if null) at the horizons of the current
    // instances, from p0 (null: cold start), solution into pout; in
    // terminal-time variables the point and p0 are mapped in and the
    // solution mapped back
    auto solve = [&](const SolveParams &pp, const R *inst_, const R *p0, R *pout, R *gout, int *sout,
                     const int *act) -> int {
        const R *sx = b.dx, *sp0 = p0;
        R *sout_p = pout;
        if (term) {
            CU(launch_to_terminal<R>(b.i64, n, m, N, 1, P, b.dx, p0, b.xq, p0 ? b.q0 : nullptr, act, s));
            sx = b.xq;
            sp0 = p0 ? b.q0 : nullptr;
            sout_p = b.qtmp;
        }
        SolveParams q = pp;
        q.warm = sp0 != nullptr;
        int r = launch_generic<R>(inst_, q, sx, sp0, b.phi, sout_p, gout, b.its, sout, b.Pv, b.Dv, b.y, act, s);
        if (r) return r;
        if (term) CU(launch_from_terminal<R>(b.i64, n, m, N, 1, P, b.qtmp, pout, act, s));
        return HOPF_SUCCESS;
    };

    rc = upload_problem(b.d, pr, s);
    if (rc) return rc;
    if (hio) {
        CU(cudaMemcpyAsync(b.dx, x_, sizeof(R) * P * n, cudaMemcpyHostToDevice, s));
        if (wb) {
            CU(cudaMemcpyAsync(b.dlo, Tlo_, sizeof(R) * P, cudaMemcpyHostToDevice, s));
            CU(cudaMemcpyAsync(b.dhi, Thi_, sizeof(R) * P, cudaMemcpyHostToDevice, s));
        }
        if (pinit_) CU(cudaMemcpyAsync(b.dpi, pinit_, sizeof(R) * P * n, cudaMemcpyHostToDevice, s));
    }
    CU(cudaMemsetAsync(b.Tz, 0, sizeof(double), s));
    rc = launch_tables(b.d, pr, o, b.Tz, nullptr, 1, b.inst0, nullptr, b.tsc, 1, s);
    if (rc) return rc;
    CU(launch_ttr_init<R>(P, s, b.inst0, n, m, N, b.dx, wb ? b.dlo : nullptr, wb ? b.dhi : nullptr, o->t_max,
                          b.lo, b.hi, b.phase, b.warm, b.st, b.Tf));

    SolveParams prm;
    fill_params(prm, pr, o, P);
    prm.warm = pinit_ != nullptr;
    prm.inst_stride = 1;
    const R *inst = fp32 ? (const R *)b.i32 : (const R *)b.i64;
    int steps = 0;
    const int max_steps = o->max_steps > 0 ? o->max_steps : 256;
    int remaining = 0;
    if (o->newton) {
        // hybrid Newton/bisection (§IV).  A candidate's solve stops as soon as
        // the sign of phi is certified (or at tol_gap); the step uses the
        // middle of the certified interval, so far from the root a loose
        // solve gives an inexact Newton step and near it the solve tightens
        // by itself.  After the first candidate every solve starts from the
        // previous candidate's p*.
        CU(launch_ttr_newton_start(P, s, b.hi, b.phase, b.cand, b.act));
        prm.sign_mode = 1;
        for (;;) {
            rc = launch_tables(b.d, pr, o, b.cand, b.act, P, b.i64, b.i32, b.tsc, tgrid, s);
            if (rc) return rc;
            const R *p0 = steps == 0 ? b.dpi : b.ptmp;
            rc = solve(prm, inst, p0, b.ptmp, b.gtmp, b.sst, b.act);
            if (rc) return rc;
            CU(cudaMemsetAsync(b.rem, 0, sizeof(int), s));
            CU(launch_ttr_newton_update<R>(P, s, n, m, pr->ctrl_kind, b.d.A, b.d.B, b.d.q, b.dx, o->t_max, o->tol_T,
                                           b.Pv, b.Dv, b.ptmp, b.cand, b.act, b.lo, b.hi, b.phase, b.st, b.Tf,
                                           b.rem));
            CU(cudaMemcpyAsync(&remaining, b.rem, sizeof(int), cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            ++steps;
            if (remaining == 0 || steps >= max_steps) break;
        }
        prm.warm = b.dpi != nullptr;
    }
    for (; !o->newton;) {
        CU(launch_ttr_candidates(P, s, b.lo, b.hi, b.phase, b.cand, b.act));
        rc = launch_tables(b.d, pr, o, b.cand, b.act, P, b.i64, b.i32, b.tsc, tgrid, s);
        if (rc) return rc;
        prm.sign_mode = 1;
        rc = solve(prm, inst, b.dpi, b.ptmp, b.gtmp, b.sst, b.act);
        if (rc) return rc;
        CU(cudaMemsetAsync(b.rem, 0, sizeof(int), s));
        CU(launch_ttr_update<R>(P, s, o->t_max, o->tol_T, b.cand, b.act, b.Pv, b.Dv, b.sst, b.lo, b.hi, b.phase,
                                b.warm, b.st, b.Tf, b.rem));
        CU(cudaMemcpyAsync(&remaining, b.rem, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        ++steps;
        if (remaining == 0 || steps >= max_steps) break;
    }
    // points the step cap stopped: T* = top of the bracket, status MAXITER
    if (remaining > 0) CU(launch_ttr_cap(P, s, b.hi, b.phase, b.st, b.Tf));
    // final certified solve at T* (T = 0 inside the target, t_max if unreachable)
    rc = launch_tables(b.d, pr, o, b.Tf, nullptr, P, b.i64, b.i32, b.tsc, tgrid, s);
    if (rc) return rc;
    prm.sign_mode = 0;
    rc = solve(prm, inst, b.dpi, b.dps, b.dgap, b.fst, nullptr);
    if (rc) return rc;
    CU(launch_ttr_finish<R>(P, s, b.st, b.fst, b.Tf, b.dTs, b.dst));
    if (hio) {
        CU(cudaMemcpyAsync(Tstar_, b.dTs, sizeof(R) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(pstar_, b.dps, sizeof(R) * P * n, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(gap_, b.dgap, sizeof(R) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(status, b.dst, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    if (steps_out) *steps_out = steps;
    return HOPF_SUCCESS;
}

// ------------------------------------------------- fixed-step quadrature rule
// One table on [0, t_max] in terminal-time variables (N nodes, step
// dt = t_max / N) serves every point and horizon: the node count, last weight
// and dual step of each point's horizon come from fixed_prep, the maps of
// the query point and of p from the binary powers of e^{+-dt A}.
struct FixedCtx {
    int N = 0, nsnap = 0, J = 0;
    double dt = 0.0, anorm = 0.0;
    double *Tm = nullptr, *i64 = nullptr, *tsc = nullptr, *snaps = nullptr, *lam = nullptr, *lsc = nullptr;
    double *Ep = nullptr, *Em = nullptr, *psc = nullptr, *wl = nullptr, *sig = nullptr;
    float *i32 = nullptr;
    int *nk = nullptr;
};

template <typename AR>
FixedCtx take_fixed(AR &a, int n, int m, int N, int P, bool fp32) {
    FixedCtx f;
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    f.N = N;
    f.nsnap = (N + FX_SNAP - 1) / FX_SNAP;
    f.J = fixed_powers_count(N);
    f.Tm = a.template take<double>(1);
    f.i64 = a.template take<double>((size_t)L.stride);
    f.i32 = fp32 ? a.template take<float>((size_t)L.stride) : nullptr;
    f.tsc = a.template take<double>((size_t)table_scratch_doubles(n, m));
    f.snaps = a.template take<double>((size_t)f.nsnap * n * n);
    f.lam = a.template take<double>((size_t)f.nsnap);
    f.lsc = a.template take<double>((size_t)f.nsnap * (2 * n + 8));
    f.Ep = a.template take<double>((size_t)f.J * n * n);
    f.Em = a.template take<double>((size_t)f.J * n * n);
    f.psc = a.template take<double>((size_t)2 * (2 * n * n + 8));
    f.nk = a.template take<int>((size_t)P);
    f.wl = a.template take<double>((size_t)P);
    f.sig = a.template take<double>((size_t)P);
    return f;
}

// the shared table at t_max with its prefix |K|^2 values, and the powers
int fixed_setup(FixedCtx &f, const DevProblem &d, const hopf_problem *pr, const hopf_opts *o, cudaStream_t s) {
    const int n = pr->n, m = pr->m;
    f.dt = o->t_max / (double)o->N;
    double r1 = 0.0, ri = 0.0;          // |A|_1 and |A|_inf bound the sub-steps of the remainder series
    for (int a = 0; a < n; ++a) {
        double cs = 0.0, rs = 0.0;
        for (int b = 0; b < n; ++b) {
            cs += std::fabs(pr->A[b * n + a]);
            rs += std::fabs(pr->A[a * n + b]);
        }
        r1 = std::max(r1, cs);
        ri = std::max(ri, rs);
    }
    f.anorm = std::max(r1, ri);
    CU(cudaMemcpyAsync(f.Tm, &o->t_max, sizeof(double), cudaMemcpyHostToDevice, s));
    CU(launch_build_instances_opt(1, table_threads(n), s, d.A, d.B, d.q, d.W, f.Tm, nullptr, 1, n, m, o->N,
                                  HOPF_LEFT_RIEMANN, o->tau, o->sigma_scale, f.i64, f.i32, f.tsc, o->accel, 1,
                                  f.snaps, FX_SNAP));
    CU(launch_fixed_lam(f.snaps, f.nsnap, n, f.lam, f.lsc, s));
    CU(launch_fixed_powers(d.A, n, f.dt, f.J, f.Ep, f.Em, f.psc, s));
    return HOPF_SUCCESS;
}

// tiled kernel for float32 states of 17..256 components, else the general one
bool fixed_tile(const hopf_problem *pr, const hopf_opts *o, int P, const Device &dev, int *ppt, int *grid,
                size_t *smem, int *dbuf) {
    return o->precision == HOPF_FP32 && pr->n > 16 && o->kernel != HOPF_KERNEL_GENERIC &&
           tile_plan(pr->n, pr->m, o->N, P, dev.sms, dev.smem_optin - 2048, ppt, grid, smem, dbuf);
}

template <typename R>
int value_fixed_impl(const hopf_problem *pr, const hopf_opts *o, int P, const void *x_, const void *t_,
                     int t_stride, const void *pinit_, void *phi_, void *pstar_, void *gap_, int *iters,
                     int *status, cudaStream_t s) {
    const int n = pr->n, m = pr->m, N = o->N;
    const bool fp32 = o->precision == HOPF_FP32;
    const bool hio = o->host_io != 0;
    const int nT = t_stride ? P : 1;
    Device dev;
    int rc = query_device(&dev);
    if (rc) return rc;
    int tile_ppt = 0, tile_grid = 0, tile_dbuf = 0;
    size_t tile_smem = 0;
    const bool tile = fixed_tile(pr, o, P, dev, &tile_ppt, &tile_grid, &tile_smem, &tile_dbuf);
    FixedCtx f;
    DevProblem d;
    double *Tv;
    R *dx, *dt, *dpi, *dphi, *dps, *dgap, *xq, *q0, *qs, *y;
    int *dit, *dst, *ctr, *tcl;
    float *tws, *tcs;
    auto plan = [&](Arena &a) {
        d = take_problem(a, n, m);
        f = take_fixed(a, n, m, N, P, fp32);
        Tv = a.template take<double>(nT);
        dx = hio ? a.template take<R>((size_t)P * n) : (R *)x_;
        dt = hio ? a.template take<R>((size_t)nT) : (R *)t_;
        dpi = (hio && pinit_) ? a.template take<R>((size_t)P * n) : (R *)pinit_;
        dphi = hio ? a.template take<R>(P) : (R *)phi_;
        dps = hio ? a.template take<R>((size_t)P * n) : (R *)pstar_;
        dgap = hio ? a.template take<R>(P) : (R *)gap_;
        dit = hio ? a.template take<int>(P) : iters;
        dst = hio ? a.template take<int>(P) : status;
        xq = a.template take<R>((size_t)P * n);
        q0 = pinit_ ? a.template take<R>((size_t)P * n) : nullptr;
        qs = a.template take<R>((size_t)P * n);
        y = tile ? nullptr : a.template take<R>((size_t)P * N * m);
        ctr = a.template take<int>(4);
        tws = tile ? a.template take<float>((size_t)tile_workspace_floats(n, m, N, tile_ppt, tile_grid)) : nullptr;
        tcs = tile ? a.template take<float>((size_t)tile_carry_floats(n, m, N, tile_ppt, P)) : nullptr;
        tcl = tile ? a.template take<int>((size_t)2 * P) : nullptr;
    };
    Arena meas(nullptr);
    plan(meas);
    void *base = nullptr;
    rc = ensure_workspace(meas.off, &base, s);
    if (rc) return rc;
    Arena a(base);
    plan(a);
    rc = upload_problem(d, pr, s);
    if (rc) return rc;
    if (hio) {
        CU(cudaMemcpyAsync(dx, x_, sizeof(R) * P * n, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(dt, t_, sizeof(R) * nT, cudaMemcpyHostToDevice, s));
        if (pinit_) CU(cudaMemcpyAsync(dpi, pinit_, sizeof(R) * P * n, cudaMemcpyHostToDevice, s));
    }
    CU(launch_horizons(nT, s, dt, fp32, Tv));
    rc = fixed_setup(f, d, pr, o, s);
    if (rc) return rc;
    CU(launch_fixed_prep<R>(P, Tv, t_stride, o->t_max, f.dt, N, o->tau, o->sigma_scale, f.lam, FX_SNAP, nullptr,
                            f.nk, f.wl, f.sig, n, dphi, dps, dgap, dit, dst, s));
    CU(launch_fixed_map<R>(0, P, n, d.A, f.anorm, f.Ep, f.J, f.nk, f.wl, dx, xq, nullptr, dev.sms, s));
    if (pinit_) CU(launch_fixed_map<R>(2, P, n, d.A, f.anorm, f.Em, f.J, f.nk, f.wl, dpi, q0, nullptr, dev.sms, s));
    SolveParams prm;
    fill_params(prm, pr, o, P);
    prm.warm = pinit_ != nullptr;
    prm.fx_nk = f.nk;
    prm.fx_wl = f.wl;
    prm.fx_sig = f.sig;
    if (tile) {
        CU(launch_pdhg_tile(f.i32, f.i64, prm, (const float *)xq, (const float *)q0, (float *)dphi, (float *)qs,
                            (float *)dgap, dit, dst, tws, ctr, tile_ppt, tile_grid, tile_smem, tile_dbuf, tcs, tcl,
                            s));
    } else {
        const R *inst = fp32 ? (const R *)f.i32 : (const R *)f.i64;
        rc = launch_generic<R>(inst, prm, xq, q0, dphi, qs, dgap, dit, dst, nullptr, nullptr, y, nullptr, s);
        if (rc) return rc;
    }
    CU(launch_fixed_map<R>(1, P, n, d.A, f.anorm, f.Ep, f.J, f.nk, f.wl, qs, dps, nullptr, dev.sms, s));
    if (hio) {
        CU(cudaMemcpyAsync(phi_, dphi, sizeof(R) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(pstar_, dps, sizeof(R) * P * n, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(gap_, dgap, sizeof(R) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(iters, dit, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(status, dst, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    return HOPF_SUCCESS;
}

template <typename R>
int ttr_fixed_impl(const hopf_problem *pr, const hopf_opts *o, int P, const void *x_, const void *Tlo_,
                   const void *Thi_, const void *pinit_, void *Tstar_, void *pstar_, void *gap_, int *status,
                   int *steps_out, cudaStream_t s) {
    const int n = pr->n, m = pr->m, N = o->N;
    const bool fp32 = o->precision == HOPF_FP32;
    const bool hio = o->host_io != 0;
    const bool wb = Tlo_ && Thi_;
    Device dev;
    int rc = query_device(&dev);
    if (rc) return rc;
    int tile_ppt = 0, tile_grid = 0, tile_dbuf = 0;
    size_t tile_smem = 0;
    const bool tile = fixed_tile(pr, o, P, dev, &tile_ppt, &tile_grid, &tile_smem, &tile_dbuf);
    FixedCtx f;
    struct Bufs {
        DevProblem d;
        double *lo, *hi, *cand, *Tf;
        int *phase, *warm, *st, *act, *sst, *fst, *its, *rem, *list, *ctr, *tcl;
        R *Pv, *Dv, *phi, *gtmp, *ptmp, *xq, *q0, *qlast, *qout, *y;
        R *dx, *dlo, *dhi, *dpi, *dTs, *dps, *dgap;
        int *dst;
        float *tws, *tcs;
    } b;
    auto plan = [&](Arena &a) {
        b.d = take_problem(a, n, m);
        f = take_fixed(a, n, m, N, P, fp32);
        b.lo = a.template take<double>(P);
        b.hi = a.template take<double>(P);
        b.cand = a.template take<double>(P);
        b.Tf = a.template take<double>(P);
        b.phase = a.template take<int>(P);
        b.warm = a.template take<int>(P);
        b.st = a.template take<int>(P);
        b.act = a.template take<int>(P);
        b.sst = a.template take<int>(P);
        b.fst = a.template take<int>(P);
        b.its = a.template take<int>(P);
        b.rem = a.template take<int>(4);
        b.list = a.template take<int>(P);
        b.ctr = a.template take<int>(4);
        b.Pv = a.template take<R>(P);
        b.Dv = a.template take<R>(P);
        b.phi = a.template take<R>(P);
        b.gtmp = a.template take<R>(P);
        b.ptmp = a.template take<R>((size_t)P * n);
        b.xq = a.template take<R>((size_t)P * n);
        b.q0 = pinit_ ? a.template take<R>((size_t)P * n) : nullptr;
        b.qlast = a.template take<R>((size_t)P * n);
        b.qout = a.template take<R>((size_t)P * n);
        b.y = tile ? nullptr : a.template take<R>((size_t)P * N * m);
        b.tws = tile ? a.template take<float>((size_t)tile_workspace_floats(n, m, N, tile_ppt, tile_grid)) : nullptr;
        b.tcs = tile ? a.template take<float>((size_t)tile_carry_floats(n, m, N, tile_ppt, P)) : nullptr;
        b.tcl = tile ? a.template take<int>((size_t)2 * P) : nullptr;
        b.dx = hio ? a.template take<R>((size_t)P * n) : (R *)x_;
        b.dlo = (hio && wb) ? a.template take<R>(P) : (R *)Tlo_;
        b.dhi = (hio && wb) ? a.template take<R>(P) : (R *)Thi_;
        b.dpi = (hio && pinit_) ? a.template take<R>((size_t)P * n) : (R *)pinit_;
        b.dTs = hio ? a.template take<R>(P) : (R *)Tstar_;
        b.dps = hio ? a.template take<R>((size_t)P * n) : (R *)pstar_;
        b.dgap = hio ? a.template take<R>(P) : (R *)gap_;
        b.dst = hio ? a.template take<int>(P) : status;
    };
    Arena meas(nullptr);
    plan(meas);
    void *base = nullptr;
    rc = ensure_workspace(meas.off, &base, s);
    if (rc) return rc;
    Arena a(base);
    plan(a);
    rc = upload_problem(b.d, pr, s);
    if (rc) return rc;
    if (hio) {
        CU(cudaMemcpyAsync(b.dx, x_, sizeof(R) * P * n, cudaMemcpyHostToDevice, s));
        if (wb) {
            CU(cudaMemcpyAsync(b.dlo, Tlo_, sizeof(R) * P, cudaMemcpyHostToDevice, s));
            CU(cudaMemcpyAsync(b.dhi, Thi_, sizeof(R) * P, cudaMemcpyHostToDevice, s));
        }
        if (pinit_) CU(cudaMemcpyAsync(b.dpi, pinit_, sizeof(R) * P * n, cudaMemcpyHostToDevice, s));
    }
    rc = fixed_setup(f, b.d, pr, o, s);
    if (rc) return rc;
    // V' = W^-1 of the shared table is the T = 0 test of the target (Eq. 34)
    CU(launch_ttr_init<R>(P, s, f.i64, n, m, N, b.dx, wb ? b.dlo : nullptr, wb ? b.dhi : nullptr, o->t_max, b.lo,
                          b.hi, b.phase, b.warm, b.st, b.Tf));
    SolveParams prm;
    fill_params(prm, pr, o, P);
    prm.fx_nk = f.nk;
    prm.fx_wl = f.wl;
    prm.fx_sig = f.sig;
    // one solve of the active points at the horizons Tv: the rule data of
    // each horizon, the query point mapped to e^{TA} x, solution q into qout
    // (copied to qlast), P and D into Pv, Dv.  The first solve starts from
    // the user's p_init mapped to q0 = e^{-TA^T} p_init (cold without it);
    // every later one from the point's last solution in qlast (zero for a
    // point inside the target, solved only at T = 0).
    bool first = true;
    CU(cudaMemsetAsync(b.qlast, 0, sizeof(R) * P * n, s));
    auto solve = [&](const double *Tv, const int *act, int sign_mode, R *gap_o, int *st_o) -> int {
        CU(launch_fixed_prep<R>(P, Tv, 1, o->t_max, f.dt, N, o->tau, o->sigma_scale, f.lam, FX_SNAP, act, f.nk, f.wl,
                                f.sig, n, (R *)nullptr, (R *)nullptr, (R *)nullptr, nullptr, nullptr, s));
        CU(launch_fixed_map<R>(0, P, n, b.d.A, f.anorm, f.Ep, f.J, f.nk, f.wl, b.dx, b.xq, act, dev.sms, s));
        const R *p0 = first ? nullptr : b.qlast;
        if (first && b.dpi) {
            CU(launch_fixed_map<R>(2, P, n, b.d.A, f.anorm, f.Em, f.J, f.nk, f.wl, b.dpi, b.q0, act, dev.sms, s));
            p0 = b.q0;
        }
        first = false;
        R *q_out = b.qout;
        SolveParams q = prm;
        q.warm = p0 != nullptr;
        q.sign_mode = sign_mode;
        if (tile) {
            CU(cudaMemsetAsync(b.ctr, 0, sizeof(int), s));
            if (act) {
                active_points_kernel<<<(P + 255) / 256, 256, 0, s>>>(P, act, b.list, b.ctr);
                CU(cudaGetLastError());
                q.list = b.list;
                q.list_count = b.ctr;
            }
            CU(launch_pdhg_tile(f.i32, f.i64, q, (const float *)b.xq, (const float *)p0, (float *)b.phi,
                                (float *)q_out, (float *)gap_o, b.its, st_o, b.tws, b.ctr + 1, tile_ppt, tile_grid,
                                tile_smem, tile_dbuf, b.tcs, b.tcl, s, (float *)b.Pv, (float *)b.Dv));
        } else {
            const R *inst = fp32 ? (const R *)f.i32 : (const R *)f.i64;
            int r = launch_generic<R>(inst, q, b.xq, p0, b.phi, q_out, gap_o, b.its, st_o, b.Pv, b.Dv, b.y, act, s);
            if (r) return r;
        }
        // the next solve starts from this one's solution
        CU(launch_copy_rows<R>(P, n, act, b.qout, b.qlast, s));
        return HOPF_SUCCESS;
    };
    int steps = 0;
    const int max_steps = o->max_steps > 0 ? o->max_steps : 256;
    int remaining = 0;
    if (o->newton) {
        // hybrid Newton/bisection of §IV; the derivative d phi / dT = -H_x
        // needs p* in the paper's variable: p = e^{T A^T} q
        CU(launch_ttr_newton_start(P, s, b.hi, b.phase, b.cand, b.act));
        for (;;) {
            rc = solve(b.cand, b.act, 1, b.gtmp, b.sst);
            if (rc) return rc;
            CU(launch_fixed_map<R>(1, P, n, b.d.A, f.anorm, f.Ep, f.J, f.nk, f.wl, b.qout, b.ptmp, b.act, dev.sms, s));
            CU(cudaMemsetAsync(b.rem, 0, sizeof(int), s));
            CU(launch_ttr_newton_update<R>(P, s, n, m, pr->ctrl_kind, b.d.A, b.d.B, b.d.q, b.dx, o->t_max, o->tol_T,
                                           b.Pv, b.Dv, b.ptmp, b.cand, b.act, b.lo, b.hi, b.phase, b.st, b.Tf,
                                           b.rem));
            CU(cudaMemcpyAsync(&remaining, b.rem, sizeof(int), cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            ++steps;
            if (remaining == 0 || steps >= max_steps) break;
        }
    } else {
        for (;;) {
            CU(launch_ttr_candidates(P, s, b.lo, b.hi, b.phase, b.cand, b.act));
            rc = solve(b.cand, b.act, 1, b.gtmp, b.sst);
            if (rc) return rc;
            CU(cudaMemsetAsync(b.rem, 0, sizeof(int), s));
            CU(launch_ttr_update<R>(P, s, o->t_max, o->tol_T, b.cand, b.act, b.Pv, b.Dv, b.sst, b.lo, b.hi,
                                    b.phase, b.warm, b.st, b.Tf, b.rem));
            CU(cudaMemcpyAsync(&remaining, b.rem, sizeof(int), cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            ++steps;
            if (remaining == 0 || steps >= max_steps) break;
        }
    }
    if (remaining > 0) CU(launch_ttr_cap(P, s, b.hi, b.phase, b.st, b.Tf));
    // final certified solve at T* (T = 0 inside the target, t_max if
    // unreachable), p* = e^{T* A^T} q*
    rc = solve(b.Tf, nullptr, 0, b.dgap, b.fst);
    if (rc) return rc;
    CU(launch_fixed_map<R>(1, P, n, b.d.A, f.anorm, f.Ep, f.J, f.nk, f.wl, b.qout, b.dps, nullptr, dev.sms, s));
    CU(launch_ttr_finish<R>(P, s, b.st, b.fst, b.Tf, b.dTs, b.dst));
    if (hio) {
        CU(cudaMemcpyAsync(Tstar_, b.dTs, sizeof(R) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(pstar_, b.dps, sizeof(R) * P * n, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(gap_, b.dgap, sizeof(R) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(status, b.dst, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    if (steps_out) *steps_out = steps;
    return HOPF_SUCCESS;
}

// --------------------------------------------------------- hopf_trajectory
template <typename R>
int traj_impl(const hopf_problem *pr, const hopf_opts *o, int P, const void *x_, const void *T_,
              const void *ps_, int S, void *xt_, void *ut_, cudaStream_t s) {
    const int n = pr->n, m = pr->m;
    Device dev;
    int rc = query_device(&dev);
    if (rc) return rc;
    const bool hio = o->host_io != 0;
    const int grid = std::max(1, std::min(P, 4 * dev.sms));
    const long long per = 5LL * n * n + 4LL * n + 4LL * n * m + 48;
    DevProblem d;
    double *sc, *shared, *mm;
    R *dx, *dT, *dps, *dxt, *dut;
    auto plan = [&](Arena &a) {
        d = take_problem(a, n, m);
        sc = a.template take<double>((size_t)grid * per);
        shared = a.template take<double>(4LL * n * n + 16);   // e^{hA}, e^{-hA}, expm scratch
        mm = a.template take<double>(2);
        dx = hio ? a.template take<R>((size_t)P * n) : (R *)x_;
        dT = hio ? a.template take<R>(P) : (R *)T_;
        dps = hio ? a.template take<R>((size_t)P * n) : (R *)ps_;
        dxt = hio ? a.template take<R>((size_t)P * (S + 1) * n) : (R *)xt_;
        dut = hio ? a.template take<R>((size_t)P * (S + 1) * m) : (R *)ut_;
    };
    Arena meas(nullptr);
    plan(meas);
    void *base = nullptr;
    rc = ensure_workspace(meas.off, &base, s);
    if (rc) return rc;
    Arena a(base);
    plan(a);
    rc = upload_problem(d, pr, s);
    if (rc) return rc;
    if (hio) {
        CU(cudaMemcpyAsync(dx, x_, sizeof(R) * P * n, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(dT, T_, sizeof(R) * P, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(dps, ps_, sizeof(R) * P * n, cudaMemcpyHostToDevice, s));
    }
    // one horizon for the whole batch (the common case): the step
    // exponentials are computed once instead of once per point
    double tmm[2] = {0.0, 1.0};
    CU(launch_traj_minmax<R>(P, dT, mm, s));
    CU(cudaMemcpyAsync(tmm, mm, sizeof tmm, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const double *Eh_sh = nullptr, *G_sh = nullptr;
    if (tmm[0] == tmm[1]) {
        double *Eh = shared, *G = shared + (long long)n * n;
        CU(launch_traj_shared_expm(table_threads(n), d.A, n, S, mm, Eh, G, shared + 2LL * n * n, s));
        Eh_sh = Eh;
        G_sh = G;
    }
    CU(launch_trajectory<R>(grid, table_threads(n), s, d.A, d.B, d.q, n, m, pr->ctrl_kind, P, dx, dT, dps, S,
                            dxt, dut, sc, Eh_sh, G_sh));
    if (hio) {
        CU(cudaMemcpyAsync(xt_, dxt, sizeof(R) * P * (S + 1) * n, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(ut_, dut, sizeof(R) * P * (S + 1) * m, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    return HOPF_SUCCESS;
}

// ------------------------------------------------------- hopf_node_table
int node_table_impl(const hopf_problem *pr, const hopf_opts *o, double T, double *K_, double *w_, cudaStream_t s) {
    const int n = pr->n, m = pr->m, N = o->N;
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    DevProblem d;
    double *Tv, *i64, *tsc;
    auto plan = [&](Arena &a) {
        d = take_problem(a, n, m);
        Tv = a.template take<double>(1);
        i64 = a.template take<double>((size_t)L.stride);
        tsc = a.template take<double>((size_t)table_scratch_doubles(n, m));
    };
    Arena meas(nullptr);
    plan(meas);
    void *base = nullptr;
    int rc = ensure_workspace(meas.off, &base, s);
    if (rc) return rc;
    Arena a(base);
    plan(a);
    rc = upload_problem(d, pr, s);
    if (rc) return rc;
    CU(cudaMemcpyAsync(Tv, &T, sizeof(double), cudaMemcpyHostToDevice, s));
    rc = launch_tables(d, pr, o, Tv, nullptr, 1, i64, nullptr, tsc, 1, s);
    if (rc) return rc;
    const cudaMemcpyKind kind = o->host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    CU(cudaMemcpyAsync(K_, i64 + L.K, sizeof(double) * (size_t)N * m * n, kind, s));
    CU(cudaMemcpyAsync(w_, i64 + L.w, sizeof(double) * (size_t)N, kind, s));
    if (o->host_io) CU(cudaStreamSynchronize(s));
    return HOPF_SUCCESS;
}

// network prediction: tensor cores when requested and the layers fit one MMA in N
int net_predict(const hopf_mlp *net, int B, const float *x, float *y, float *scratch, int *err, cudaStream_t s) {
    if (net->use_tc && net->hidden <= 256 && net->n_out <= 256) {
        CU(mlp_forward_tc(net->n_in, net->hidden, net->n_out, (const __nv_bfloat16 *)net->w_bf16, net->w, net->x_shift,
                          net->x_scale, net->y_shift, net->y_scale, B, x, y, scratch, err, s));
    } else {
        CU(mlp_forward(net->n_in, net->hidden, net->n_out, (const __nv_bfloat16 *)net->w_bf16, net->w, net->x_shift,
                       net->x_scale, net->y_shift, net->y_scale, B, x, y, scratch, false, s));
    }
    return HOPF_SUCCESS;
}

int check_mlp(const hopf_mlp *net) {
    if (!net) return fail(HOPF_EINVAL, "null network");
    if (net->n_in < 1 || net->hidden < 1 || net->n_out < 1 || net->hidden > 65536)
        return fail(HOPF_EINVAL, "bad network sizes");
    if (!net->w || !net->w_bf16 || !net->x_shift || !net->x_scale || !net->y_shift || !net->y_scale)
        return fail(HOPF_EINVAL, "network pointers must be set");
    return HOPF_SUCCESS;
}

int value_warm_impl(const hopf_problem *pr, const hopf_opts *o, const hopf_mlp *net, int P, const void *x_,
                    const void *t_, int t_stride, int max_iter_warm, void *phi_, void *pstar_, void *gap_,
                    int *iters, int *status, int *n_fallback, cudaStream_t s) {
    const int n = pr->n, m = pr->m, N = o->N;
    const int n_inst = t_stride ? P : 1;
    Device dev;
    int rc = query_device(&dev);
    if (rc) return rc;
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    SmallPlan sp, sp32;
    if (t_stride == 0) {
        sp = plan_small(dev, n, m, N, P);
        sp32 = plan_small(dev, n, m, N, P, 32);
        sp32.grid = dev.sms;
    }
    // large states, one shared table: the tensor-core or the tiled kernel
    // (warm solve and fallback)
    int tc_grid = 0;
    const bool tcore = !sp.ok && want_tc(pr, o, t_stride, P, dev, &tc_grid);
    int tile_ppt = 0, tile_grid = 0, tile_dbuf = 0;
    size_t tile_smem = 0;
    const bool tile = t_stride == 0 && !sp.ok && !tcore &&
                      tile_plan(n, m, N, P, dev.sms, dev.smem_optin - 2048, &tile_ppt, &tile_grid, &tile_smem,
                                &tile_dbuf);
    const int tgrid = table_grid(dev, n_inst);
    DevProblem d;
    double *Tv, *i64, *tsc;
    float *i32, *phat, *msc, *y, *tws, *tcs;
    int *tcl;
    int *list, *cnt, *ctr, *ord, *obucket, *ocount, *ototal;
    CarryPair cb;
    const bool hio = o->host_io != 0;
    const bool term = o->variables == HOPF_VARS_TERMINAL;
    float *dx, *dt, *dphi, *dps, *dgap;
    float *xq = nullptr, *qhat = nullptr, *qs = nullptr;
    int *dit, *dst;
    auto plan = [&](Arena &a) {
        d = take_problem(a, n, m);
        xq = term ? a.template take<float>((size_t)P * n) : nullptr;
        qhat = term ? a.template take<float>((size_t)P * n) : nullptr;
        qs = term ? a.template take<float>((size_t)P * n) : nullptr;
        dx = hio ? a.template take<float>((size_t)P * n) : (float *)x_;
        dt = hio ? a.template take<float>((size_t)n_inst) : (float *)t_;
        dphi = hio ? a.template take<float>(P) : (float *)phi_;
        dps = hio ? a.template take<float>((size_t)P * n) : (float *)pstar_;
        dgap = hio ? a.template take<float>(P) : (float *)gap_;
        dit = hio ? a.template take<int>(P) : iters;
        dst = hio ? a.template take<int>(P) : status;
        Tv = a.template take<double>(n_inst);
        i64 = a.template take<double>((size_t)n_inst * L.stride);
        i32 = a.template take<float>((size_t)n_inst * L.stride);
        tsc = a.template take<double>((size_t)tgrid * table_scratch_doubles(n, m));
        phat = a.template take<float>((size_t)P * n);
        msc = a.template take<float>((size_t)mlp_scratch_floats(net->n_in, net->hidden, net->n_out, P, false));
        list = a.template take<int>(P);
        cnt = a.template take<int>(4);
        ctr = a.template take<int>(4);
        ord = a.template take<int>(P);
        obucket = a.template take<int>(P);
        ocount = a.template take<int>(ORDER_BUCKETS);
        ototal = a.template take<int>(4);
        y = (sp.ok || tile || tcore) ? nullptr : a.template take<float>((size_t)P * N * m);
        tws = tile ? a.template take<float>((size_t)tile_workspace_floats(n, m, N, tile_ppt, tile_grid))
                   : (tcore ? a.template take<float>((size_t)tc_workspace_floats(n, m, N, tc_grid)) : nullptr);
        tcs = tile ? a.template take<float>((size_t)tile_carry_floats(n, m, N, tile_ppt, P)) : nullptr;
        tcl = tile ? a.template take<int>((size_t)2 * P) : nullptr;
        if (sp.ok) cb = take_carry(a, P, N, m);
    };
    Arena meas(nullptr);
    plan(meas);
    void *base = nullptr;
    rc = ensure_workspace(meas.off, &base, s);
    if (rc) return rc;
    Arena a(base);
    plan(a);
    rc = upload_problem(d, pr, s);
    if (rc) return rc;
    if (hio) {
        CU(cudaMemcpyAsync(dx, x_, sizeof(float) * P * n, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(dt, t_, sizeof(float) * n_inst, cudaMemcpyHostToDevice, s));
    }
    const bool prof = o->profile != 0;
    if (prof) {
        if (g_prof.device != dev.id) {
            for (auto &e : g_prof.ev)
                if (e) cudaEventDestroy(e);
            for (auto &e : g_prof.ev) CU(cudaEventCreate(&e));
            g_prof.device = dev.id;
        }
        g_prof.valid = false;
        CU(cudaEventRecord(g_prof.ev[0], s));
    }
    // the node table (side stream) and the network's prediction of p* with
    // the hardest-first ordering (caller's stream) are independent: overlap
    Side *tsd = nullptr;
    rc = side_stream(dev.id, &tsd);
    if (rc) return rc;
    CU(cudaEventRecord(tsd->fork, s));
    CU(cudaStreamWaitEvent(tsd->stream, tsd->fork, 0));
    CU(launch_horizons(n_inst, tsd->stream, dt, true, Tv));
    rc = launch_tables(d, pr, o, Tv, nullptr, n_inst, i64, i32, tsc, tgrid, tsd->stream);
    if (rc) return rc;
    CU(cudaEventRecord(tsd->join, tsd->stream));
    rc = net_predict(net, P, dx, phat, msc, ctr + 3, s);
    if (rc) return rc;
    SolveParams prm;
    fill_params(prm, pr, o, P);
    prm.inst_stride = t_stride ? 1 : 0;
    // in terminal-time variables the solves see e^{TA} x and q = e^{-TA^T} p
    const float *sx = term ? xq : dx;
    float *sps = term ? qs : dps;
    auto solve = [&](const SolveParams &pp, const float *pinit) -> int {
        if (sp.ok)
            return run_small_two_phase(sp, sp32, m, i32, pp, sx, pinit, dphi, sps, dgap, dit, dst, cb,
                                       o->park_iters, s);
        if (tcore) {
            CU(launch_pdhg_tc(i32, i64, pp, sx, pinit, dphi, sps, dgap, dit, dst, tws, ctr, tc_grid, s));
            return HOPF_SUCCESS;
        }
        if (tile) {
            CU(launch_pdhg_tile(i32, i64, pp, sx, pinit, dphi, sps, dgap, dit, dst, tws, ctr, tile_ppt, tile_grid,
                                tile_smem, tile_dbuf, tcs, tcl, s));
            return HOPF_SUCCESS;
        }
        return launch_generic<float>(i32, pp, sx, pinit, dphi, sps, dgap, dit, dst, nullptr, nullptr, y, nullptr, s);
    };
    // hardest-first order of the warm solve
    CU(cudaMemsetAsync(ocount, 0, sizeof(int) * ORDER_BUCKETS, s));
    order_count_kernel<<<(P + 255) / 256, 256, 0, s>>>(P, n, phat, obucket, ocount);
    order_scan_kernel<<<1, 32, 0, s>>>(P, 0, ocount, ototal);
    order_scatter_kernel<<<(P + 255) / 256, 256, 0, s>>>(P, obucket, ocount, ord);
    CU(cudaGetLastError());
    CU(cudaStreamWaitEvent(s, tsd->join, 0));
    if (term) CU(launch_to_terminal<float>(i64, n, m, N, t_stride ? 1 : 0, P, dx, phat, xq, qhat, nullptr, s));
    const float *pstart = term ? qhat : phat;
    if (prof) CU(cudaEventRecord(g_prof.ev[1], s));
    // warm solve, capped at max_iter_warm
    SolveParams pw = prm;
    pw.warm = 1;
    pw.max_iter = max_iter_warm;
    pw.list = ord;
    pw.list_count = ototal;
    rc = solve(pw, pstart);
    if (rc) return rc;
    // cold fallback for every point that the warm solve did not certify
    CU(cudaMemsetAsync(cnt, 0, sizeof(int), s));
    failed_points_kernel<<<(P + 255) / 256, 256, 0, s>>>(P, dst, list, cnt);
    CU(cudaGetLastError());
    SolveParams pc = prm;
    pc.warm = 0;
    pc.list = list;
    pc.list_count = cnt;
    rc = solve(pc, nullptr);
    if (rc) return rc;
    if (prof) {
        CU(cudaEventRecord(g_prof.ev[2], s));
        g_prof.valid = true;
    }
    if (term) CU(launch_from_terminal<float>(i64, n, m, N, t_stride ? 1 : 0, P, qs, dps, nullptr, s));
    if (n_fallback)
        CU(cudaMemcpyAsync(n_fallback, cnt, sizeof(int), hio ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    if (hio) {
        CU(cudaMemcpyAsync(phi_, dphi, sizeof(float) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(pstar_, dps, sizeof(float) * P * n, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(gap_, dgap, sizeof(float) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(iters, dit, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(status, dst, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    return HOPF_SUCCESS;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

void hopf_default_opts(hopf_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->rule = HOPF_LEFT_RIEMANN;
    o->N = 100;
    o->max_iter = 100000;
    o->gap_every = 8;
    o->precision = HOPF_FP32;
    o->host_io = 0;
    o->tau = 1.0;
    o->sigma_scale = 1.0;
    o->tol_gap = 1e-5;
    o->t_max = 10.0;
    o->tol_T = 1e-5;
}

int hopf_value(const hopf_problem *prob, const hopf_opts *opts, int P, const void *x, const void *t,
               int t_stride, const void *p_init, void *phi, void *p_star, void *gap, int *iters, int *status,
               void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    int rc = check_problem(prob, opts, true);
    if (rc) return rc;
    if (P < 0) return fail(HOPF_EINVAL, "P must be >= 0");
    if (P == 0) return HOPF_SUCCESS;
    if (t_stride != 0 && t_stride != 1) return fail(HOPF_EINVAL, "t_stride must be 0 or 1");
    if (!x || !t || !phi || !p_star || !gap || !iters || !status) return fail(HOPF_EINVAL, "null array");
    cudaStream_t s = (cudaStream_t)stream;
    if (opts->rule == HOPF_LEFT_FIXED) {
        if (opts->precision == HOPF_FP64)
            return value_fixed_impl<double>(prob, opts, P, x, t, t_stride, p_init, phi, p_star, gap, iters, status, s);
        return value_fixed_impl<float>(prob, opts, P, x, t, t_stride, p_init, phi, p_star, gap, iters, status, s);
    }
    if (opts->precision == HOPF_FP64)
        return value_impl<double>(prob, opts, P, x, t, t_stride, p_init, phi, p_star, gap, iters, status, s);
    return value_impl<float>(prob, opts, P, x, t, t_stride, p_init, phi, p_star, gap, iters, status, s);
}

int hopf_value_stacked(const hopf_stacked *prob, const hopf_opts *opts, int P, const void *x, const void *t,
                       int t_stride, const void *p_init, void *phi, void *p_star, void *gap, int *iters, int *status,
                       void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    if (!prob || !opts) return fail(HOPF_EINVAL, "null problem or options");
    const int nb = prob->base.n, k = prob->copies;
    if (k < 1 || k > 64) return fail(HOPF_EINVAL, "copies must be in [1, 64]");
    if (nb < 1 || nb > 8) return fail(HOPF_EINVAL, "the base state dimension must be in [1, 8]");
    if (!prob->W_blocks) return fail(HOPF_EINVAL, "W_blocks is required");
    hopf_problem first = prob->base;
    first.W = prob->W_blocks;              // validate the base system with the first block
    int rc = check_problem(&first, opts, true);
    if (rc) return rc;
    for (int j = 1; j < k; ++j) {
        const double *Wj = prob->W_blocks + (long long)j * nb * nb;
        if (!all_finite(Wj, (long long)nb * nb)) return fail(HOPF_ENONFINITE, "W block %d has a non-finite entry", j);
        if (!is_spd(Wj, nb)) return fail(HOPF_ENOTSPD, "W block %d is not symmetric positive definite", j);
    }
    if (opts->host_io) return fail(HOPF_EINVAL, "hopf_value_stacked takes device arrays only (host_io = 0)");
    if (opts->accel) return fail(HOPF_EINVAL, "hopf_value_stacked runs the iteration of Eq. 15 (accel = 0)");
    if (P < 0) return fail(HOPF_EINVAL, "P must be >= 0");
    if (P == 0) return HOPF_SUCCESS;
    if (t_stride != 0 && t_stride != 1) return fail(HOPF_EINVAL, "t_stride must be 0 or 1");
    if (!x || !t || !phi || !p_star || !gap || !iters || !status) return fail(HOPF_EINVAL, "null array");
    cudaStream_t s = (cudaStream_t)stream;
    if (opts->precision == HOPF_FP64)
        return stacked_impl<double>(prob, opts, P, x, t, t_stride, p_init, phi, p_star, gap, iters, status, s);
    return stacked_impl<float>(prob, opts, P, x, t, t_stride, p_init, phi, p_star, gap, iters, status, s);
}

int hopf_time_to_reach(const hopf_problem *prob, const hopf_opts *opts, int P, const void *x, const void *T_lo,
                       const void *T_hi, const void *p_init, void *T_star, void *p_star, void *gap, int *status,
                       int *steps, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    int rc = check_problem(prob, opts, true);
    if (rc) return rc;
    if (P < 0) return fail(HOPF_EINVAL, "P must be >= 0");
    if (steps) *steps = 0;
    if (P == 0) return HOPF_SUCCESS;
    if (!(opts->t_max > 0.0) || !std::isfinite(opts->t_max)) return fail(HOPF_EINVAL, "need finite t_max > 0");
    // below a few float64 ulps the bracket test hi - lo <= tol_T hi can never hold
    if (!(opts->tol_T >= 4.0 * DBL_EPSILON)) return fail(HOPF_EINVAL, "need tol_T >= 4 DBL_EPSILON");
    if (opts->max_steps < 0) return fail(HOPF_EINVAL, "need max_steps >= 0");
    if ((T_lo == nullptr) != (T_hi == nullptr)) return fail(HOPF_EINVAL, "give both T_lo and T_hi or neither");
    if (!x || !T_star || !p_star || !gap || !status) return fail(HOPF_EINVAL, "null array");
    cudaStream_t s = (cudaStream_t)stream;
    if (opts->rule == HOPF_LEFT_FIXED) {
        if (opts->precision == HOPF_FP64)
            return ttr_fixed_impl<double>(prob, opts, P, x, T_lo, T_hi, p_init, T_star, p_star, gap, status, steps, s);
        return ttr_fixed_impl<float>(prob, opts, P, x, T_lo, T_hi, p_init, T_star, p_star, gap, status, steps, s);
    }
    if (opts->precision == HOPF_FP64)
        return ttr_impl<double>(prob, opts, P, x, T_lo, T_hi, p_init, T_star, p_star, gap, status, steps, s);
    return ttr_impl<float>(prob, opts, P, x, T_lo, T_hi, p_init, T_star, p_star, gap, status, steps, s);
}

int hopf_trajectory(const hopf_problem *prob, const hopf_opts *opts, int P, const void *x, const void *T,
                    const void *p_star, int S, void *x_traj, void *u_traj, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    int rc = check_problem(prob, opts, false);
    if (rc) return rc;
    if (P < 0 || S < 1) return fail(HOPF_EINVAL, "need P >= 0 and S >= 1");
    if (P == 0) return HOPF_SUCCESS;
    if (!x || !T || !p_star || !x_traj || !u_traj) return fail(HOPF_EINVAL, "null array");
    cudaStream_t s = (cudaStream_t)stream;
    if (opts->precision == HOPF_FP64)
        return traj_impl<double>(prob, opts, P, x, T, p_star, S, x_traj, u_traj, s);
    return traj_impl<float>(prob, opts, P, x, T, p_star, S, x_traj, u_traj, s);
}

int hopf_node_table(const hopf_problem *prob, const hopf_opts *opts, double T, double *K, double *w, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    int rc = check_problem(prob, opts, true);
    if (rc) return rc;
    if (!(T >= 0.0) || !std::isfinite(T)) return fail(HOPF_EINVAL, "T must be finite and >= 0");
    if (opts->rule == HOPF_LEFT_FIXED) return fail(HOPF_EINVAL, "node table: give one of the T / N rules");
    if (!K || !w) return fail(HOPF_EINVAL, "null array");
    return node_table_impl(prob, opts, T, K, w, (cudaStream_t)stream);
}

long long hopf_mlp_param_count(int n_in, int hidden, int n_out) { return mlp_param_count(n_in, hidden, n_out); }

int hopf_mlp_sync(const hopf_mlp *net, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    int rc = check_mlp(net);
    if (rc) return rc;
    CU(mlp_sync_bf16(mlp_param_count(net->n_in, net->hidden, net->n_out), net->w, (__nv_bfloat16 *)net->w_bf16,
                     (cudaStream_t)stream));
    return HOPF_SUCCESS;
}

int hopf_mlp_forward(const hopf_mlp *net, int B, const float *x, float *y, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    int rc = check_mlp(net);
    if (rc) return rc;
    if (B < 0 || (B > 0 && (!x || !y))) return fail(HOPF_EINVAL, "bad batch or null array");
    if (B == 0) return HOPF_SUCCESS;
    void *base = nullptr;
    const size_t fl = (size_t)mlp_scratch_floats(net->n_in, net->hidden, net->n_out, B, false);
    rc = ensure_workspace(sizeof(float) * fl + 256, &base, (cudaStream_t)stream);
    if (rc) return rc;
    int *err = (int *)((char *)base + ((sizeof(float) * fl + 127) & ~(size_t)127));
    return net_predict(net, B, x, y, (float *)base, err, (cudaStream_t)stream);
}

int hopf_mlp_loss_grad(const hopf_mlp *net, int B, const float *x, const float *y, float *loss, float *grad,
                       void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    int rc = check_mlp(net);
    if (rc) return rc;
    if (B < 1 || !x || !y || !loss || !grad) return fail(HOPF_EINVAL, "bad batch or null array");
    void *base = nullptr;
    rc = ensure_workspace(sizeof(float) * (size_t)mlp_scratch_floats(net->n_in, net->hidden, net->n_out, B, true),
                          &base, (cudaStream_t)stream);
    if (rc) return rc;
    CU(mlp_loss_grad(net->n_in, net->hidden, net->n_out, (const __nv_bfloat16 *)net->w_bf16, net->w, net->x_shift,
                     net->x_scale, net->y_shift, net->y_scale, B, x, y, loss, grad, (float *)base,
                     (cudaStream_t)stream));
    return HOPF_SUCCESS;
}

int hopf_mlp_adam(const hopf_mlp *net, const float *grad, int step, double lr, double beta1, double beta2,
                  double eps, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    int rc = check_mlp(net);
    if (rc) return rc;
    if (!net->adam_m || !net->adam_v || !grad || step < 1) return fail(HOPF_EINVAL, "Adam needs moments, grad, step>=1");
    CU(mlp_adam(mlp_param_count(net->n_in, net->hidden, net->n_out), net->w, (__nv_bfloat16 *)net->w_bf16, grad,
                net->adam_m, net->adam_v, (float)lr, (float)beta1, (float)beta2, (float)eps, step,
                (cudaStream_t)stream));
    return HOPF_SUCCESS;
}

int hopf_value_warm(const hopf_problem *prob, const hopf_opts *opts, const hopf_mlp *net, int P, const void *x,
                    const void *t, int t_stride, int max_iter_warm, void *phi, void *p_star, void *gap, int *iters,
                    int *status, int *n_fallback, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    int rc = check_problem(prob, opts, true);
    if (rc) return rc;
    rc = check_mlp(net);
    if (rc) return rc;
    if (opts->adaptive) return fail(HOPF_EINVAL, "warm start: adaptive steps are not supported");
    if (opts->rule == HOPF_LEFT_FIXED) return fail(HOPF_EINVAL, "warm start: the fixed-step rule is not supported");
    if (opts->precision != HOPF_FP32) return fail(HOPF_EINVAL, "warm start: FP32 only");
    if (net->n_in != prob->n || net->n_out != prob->n) return fail(HOPF_EINVAL, "network must map R^n to R^n");
    if (P < 0 || (t_stride != 0 && t_stride != 1) || max_iter_warm < 0) return fail(HOPF_EINVAL, "bad P/t_stride");
    if (P == 0) return HOPF_SUCCESS;
    if (!x || !t || !phi || !p_star || !gap || !iters || !status) return fail(HOPF_EINVAL, "null array");
    return value_warm_impl(prob, opts, net, P, x, t, t_stride, max_iter_warm, phi, p_star, gap, iters, status,
                           n_fallback, (cudaStream_t)stream);
}

int hopf_tc_selftest(int N, int K, const float *A, const float *B, float *D, int *err, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    if (N < 16 || N > 256 || N % 16 || K < 8 || K > 128 || K % 8 || !A || !B || !D || !err)
        return fail(HOPF_EINVAL, "self-test sizes: 16 <= N <= 256 (multiple of 16), 8 <= K <= 128 (multiple of 8)");
    CU(launch_tc_selftest(N, K, A, B, D, err, (cudaStream_t)stream));
    return HOPF_SUCCESS;
}

const char *hopf_status_string(int code) {
    switch (code) {
        case HOPF_OK: return "ok";
        case HOPF_MAXITER: return "max_iter reached";
        case HOPF_NONFINITE: return "non-finite iterate";
        case HOPF_UNREACHABLE: return "target unreachable within t_max";
        case HOPF_AMBIGUOUS_SIGN: return "sign of phi not certified";
        case HOPF_EINVAL: return "invalid argument";
        case HOPF_ENOTSPD: return "W not symmetric positive definite";
        case HOPF_ECUDA: return "CUDA error";
        case HOPF_ENOMEM: return "device allocation failed";
        case HOPF_ENONFINITE: return "non-finite problem data";
        case HOPF_ESCRATCH: return "does not fit the static scratch of hopf_value_noalloc";
        default: return "unknown";
    }
}

const char *hopf_last_error(void) { return g_err.c_str(); }

int hopf_last_profile(double *ms_tables, double *ms_solve) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_prof.valid) return fail(HOPF_EINVAL, "no profiled hopf_value call");
    CU(cudaEventSynchronize(g_prof.ev[2]));
    float a = 0.f, b = 0.f;
    CU(cudaEventElapsedTime(&a, g_prof.ev[0], g_prof.ev[1]));
    CU(cudaEventElapsedTime(&b, g_prof.ev[1], g_prof.ev[2]));
    if (ms_tables) *ms_tables = a;
    if (ms_solve) *ms_solve = b;
    return HOPF_SUCCESS;
}

int hopf_release_workspace(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    CU(cudaGetDevice(&dev));
    bool synced = false;
    for (auto it = g_ws.begin(); it != g_ws.end();) {
        if (it->first.first == dev) {
            if (!synced) {
                CU(cudaDeviceSynchronize());
                synced = true;
            }
            if (it->second.ptr) CU(cudaFree(it->second.ptr));
            it = g_ws.erase(it);
        } else {
            ++it;
        }
    }
    return HOPF_SUCCESS;
}

}  // extern "C"
