// hopf_value_noalloc: the batched value solve for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at solve time: a
// control loop with a hard real-time budget, where an allocation may block
// on a device-wide synchronisation, or a host process that is forbidden to
// grow its memory footprint after start-up (for instance one sharing the GPU
// under a fixed memory quota).  This entry
// point serves them.  It runs the general primal-dual kernel (the one that
// keeps each point's dual variable in global scratch) with every byte of
// scratch taken from one file-scope device array of fixed size
// (HOPF_NOALLOC_SCRATCH_BYTES), which every GPU that loads the library holds
// until the process exits.  The caller still owns and passes all inputs and
// outputs.
//
// Properties:
//  * no cudaMalloc, cudaFree or other allocating routine, on the device or
//    the host (validation uses fixed-size stack storage);
//  * the first call on a device looks up the device address of the array
//    (cudaGetSymbolAddress, with that device current) and caches it; make
//    that first call before any stream capture;
//  * every call uses the same array, so calls that overlap on the GPU (on
//    different streams, or from different host threads without ordering)
//    race on it; calls ordered on one stream are safe;
//  * the array keeps the previous call's contents; nothing in it needs to
//    start at zero because each call writes every scratch byte it later reads
//    (node tables, dual variables) before reading it;
//  * sizes that do not fit the array are rejected with HOPF_ESCRATCH.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>

#include "common.cuh"

namespace hopf {
cudaError_t launch_build_instances(int grid, int threads, cudaStream_t s, const double *A, const double *B,
                                   const double *qd, const double *W, const double *Tv, const int *active,
                                   int n_inst, int n, int m, int N, int rule, double tau, double sigma_scale,
                                   double *out64, float *out32, double *scratch);
cudaError_t launch_horizons(int count, cudaStream_t s, const void *t, bool t_is_float, double *Tv);
template <typename R>
cudaError_t launch_pdhg_generic(const R *inst, const SolveParams &prm, const R *x, const R *p_init, R *phi,
                                R *pstar, R *gap, int *iters, int *status, R *Pv, R *Dv, R *y,
                                const int *active, cudaStream_t s);
}  // namespace hopf

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[HOPF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
// one cached address per device; host threads making their first call on the
// same device at once may both look it up, and both store the same value
std::atomic<void *> g_scratch_ptr[kMaxDevices];

// Device address of the static array for the current device (looked up once).
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HOPF_ECUDA;
    void *p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HOPF_ECUDA;
        g_scratch_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return HOPF_SUCCESS;
}

struct Carve {
    char *base;
    size_t off = 0;
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

bool finite_all(const double *a, long long c) {
    for (long long i = 0; i < c; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

bool spd_small(const double *W, int n) {
    double L[HOPF_NOALLOC_MAX_N * HOPF_NOALLOC_MAX_N];
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

int validate(const hopf_problem *pr, const hopf_opts *o) {
    if (!pr || !o) return HOPF_EINVAL;
    if (pr->n < 1 || pr->m < 1 || pr->n > HOPF_NOALLOC_MAX_N || pr->m > 16) return HOPF_EINVAL;
    if (!pr->A || !pr->B || !pr->W) return HOPF_EINVAL;
    if (pr->ctrl_kind != HOPF_BALL && pr->ctrl_kind != HOPF_BOX) return HOPF_EINVAL;
    if (pr->ctrl_kind == HOPF_BALL && !(pr->radius > 0.0 && std::isfinite(pr->radius))) return HOPF_EINVAL;
    if (pr->ctrl_kind == HOPF_BOX) {
        if (!pr->half_widths) return HOPF_EINVAL;
        for (int c = 0; c < pr->m; ++c)
            if (!(pr->half_widths[c] > 0.0) || !std::isfinite(pr->half_widths[c])) return HOPF_EINVAL;
    }
    const long long n = pr->n, m = pr->m;
    if (!finite_all(pr->A, n * n) || !finite_all(pr->B, n * m) || !finite_all(pr->W, n * n))
        return HOPF_ENONFINITE;
    if (!spd_small(pr->W, pr->n)) return HOPF_ENOTSPD;
    if (o->precision != HOPF_FP64 && o->precision != HOPF_FP32) return HOPF_EINVAL;
    if (o->host_io != 0) return HOPF_EINVAL;   // device arrays only: no staging buffers
    if (o->rule != HOPF_LEFT_RIEMANN && o->rule != HOPF_TRAPEZOID && o->rule != HOPF_SIMPSON) return HOPF_EINVAL;
    if (o->N < 1 || (o->rule == HOPF_TRAPEZOID && o->N < 2) ||
        (o->rule == HOPF_SIMPSON && (o->N < 3 || o->N % 2 == 0))) return HOPF_EINVAL;
    if (o->max_iter < 0 || o->gap_every < 1) return HOPF_EINVAL;
    if (!(o->tau > 0.0) || !(o->sigma_scale > 0.0) || !(o->sigma_scale <= 1.0)) return HOPF_EINVAL;
    if (!(o->tol_gap >= 0.0)) return HOPF_EINVAL;
    if (o->accel != 0 && o->accel != 1) return HOPF_EINVAL;
    if (o->variables != HOPF_VARS_INITIAL) return HOPF_EINVAL;   // the paper's variable only
    if (o->adaptive) return HOPF_EINVAL;
    return HOPF_SUCCESS;
}

template <typename R>
int run(const hopf_problem *pr, const hopf_opts *o, int P, const void *x, const void *t, int t_stride,
        const void *p_init, void *phi, void *p_star, void *gap, int *iters, int *status, cudaStream_t s) {
    using namespace hopf;
    const int n = pr->n, m = pr->m, N = o->N;
    const bool fp32 = o->precision == HOPF_FP32;
    const int n_inst = t_stride ? P : 1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HOPF_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HOPF_ECUDA;
    const int tgrid = n_inst < 4 * sms ? n_inst : 4 * sms;
    const InstanceLayout L = InstanceLayout::make(n, m, N);

    double *A, *B, *q, *W, *Tv, *i64, *tsc;
    float *i32;
    R *y;
    auto plan = [&](Carve &c) {
        A = c.take<double>((size_t)n * n);
        B = c.take<double>((size_t)n * m);
        q = c.take<double>((size_t)m);
        W = c.take<double>((size_t)n * n);
        Tv = c.take<double>((size_t)n_inst);
        i64 = c.take<double>((size_t)n_inst * L.stride);
        i32 = fp32 ? c.take<float>((size_t)n_inst * L.stride) : nullptr;
        tsc = c.take<double>((size_t)tgrid * table_scratch_doubles(n, m));
        y = c.take<R>((size_t)P * N * m);
    };
    Carve measure{nullptr};
    plan(measure);
    if (measure.off > (size_t)HOPF_NOALLOC_SCRATCH_BYTES) return HOPF_ESCRATCH;
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    Carve c{(char *)base};
    plan(c);

    double qh[16];
    for (int k = 0; k < m; ++k) qh[k] = pr->ctrl_kind == HOPF_BALL ? pr->radius : pr->half_widths[k];
    if (cudaMemcpyAsync(A, pr->A, sizeof(double) * n * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B, pr->B, sizeof(double) * n * m, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(q, qh, sizeof(double) * m, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(W, pr->W, sizeof(double) * n * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return HOPF_ECUDA;
    if (launch_horizons(n_inst, s, t, fp32, Tv) != cudaSuccess) return HOPF_ECUDA;
    if (launch_build_instances(tgrid, n <= 16 ? 32 : (n <= 32 ? 64 : 256), s, A, B, q, W, Tv, nullptr, n_inst, n, m, N, o->rule,
                               o->tau, o->sigma_scale, i64, i32, tsc) != cudaSuccess)
        return HOPF_ECUDA;
    SolveParams prm{};
    prm.n = n;
    prm.m = m;
    prm.N = N;
    prm.P = P;
    prm.ctrl_kind = pr->ctrl_kind;
    prm.max_iter = o->max_iter;
    prm.gap_every = o->gap_every;
    prm.warm = p_init != nullptr;
    prm.sign_mode = 0;
    prm.inst_stride = t_stride ? 1 : 0;
    prm.accel = o->accel;
    prm.tau = o->tau;
    prm.tol_gap = o->tol_gap;
    prm.sign_floor = fp32 ? 1e-6 : 1e-13;
    const R *inst = fp32 ? (const R *)(const void *)i32 : (const R *)(const void *)i64;
    if (launch_pdhg_generic<R>(inst, prm, (const R *)x, (const R *)p_init, (R *)phi, (R *)p_star, (R *)gap, iters,
                               status, nullptr, nullptr, y, nullptr, s) != cudaSuccess)
        return HOPF_ECUDA;
    return HOPF_SUCCESS;
}

}  // namespace

extern "C" int hopf_value_noalloc(const hopf_problem *prob, const hopf_opts *opts, int P, const void *x,
                                  const void *t, int t_stride, const void *p_init, void *phi, void *p_star,
                                  void *gap, int *iters, int *status, void *stream) {
    int rc = validate(prob, opts);
    if (rc) return rc;
    if (P < 0 || (t_stride != 0 && t_stride != 1)) return HOPF_EINVAL;
    if (P == 0) return HOPF_SUCCESS;
    if (!x || !t || !phi || !p_star || !gap || !iters || !status) return HOPF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (opts->precision == HOPF_FP64)
        return run<double>(prob, opts, P, x, t, t_stride, p_init, phi, p_star, gap, iters, status, s);
    return run<float>(prob, opts, P, x, t, t_stride, p_init, phi, p_star, gap, iters, status, s);
}
