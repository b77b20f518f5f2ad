// Time-to-reach bisection bookkeeping (§IV) and trajectory generation from
// the optimal dual p* (§IV Eq. 27, §V Eq. 33).
#include "common.cuh"
#include "cta_linalg.cuh"

namespace hopf {

enum { PH_HI = 0, PH_LO = 1, PH_BIS = 2, PH_DONE = 3 };

// Per point: inside the target already (J_x(x) <= 0, Eq. 34 with V = W^-1
// taken from the T = 0 instance) -> T* = 0; otherwise set up the bracket.
template <typename R>
__global__ void ttr_init_kernel(const double *__restrict__ inst0, int n, int m, int N, int P,
                                const R *__restrict__ x, const R *__restrict__ T_lo,
                                const R *__restrict__ T_hi, double t_max, double *lo, double *hi,
                                int *phase, int *warm, int *st, double *Tfinal) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    const InstanceLayout L = InstanceLayout::make(n, m, N);
    const double *V = inst0 + L.V;
    double J = -1.0;
    for (int a = 0; a < n; ++a) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s = fma(V[a * n + b], (double)x[(long long)k * n + b], s);
        J = fma((double)x[(long long)k * n + a], s, J);
    }
    st[k] = HOPF_OK;
    if (J <= 0.0) {
        phase[k] = PH_DONE;
        lo[k] = 0.0;
        hi[k] = 0.0;
        Tfinal[k] = 0.0;
        warm[k] = 0;
        return;
    }
    bool wb = T_lo && T_hi;
    double l = wb ? (double)T_lo[k] : 0.0, h = wb ? (double)T_hi[k] : t_max;
    if (!(l >= 0.0) || !(h > l) || !(h <= t_max)) { wb = false; l = 0.0; h = t_max; }
    lo[k] = l;
    hi[k] = h;
    Tfinal[k] = h;     // replaced when the point finishes; kept if the step cap stops it first
    warm[k] = wb ? 1 : 0;
    phase[k] = PH_HI;
}

// Step cap reached: every point still open gets the top of its bracket as
// T* (the final solve there gives p*) and the status HOPF_MAXITER.
__global__ void ttr_cap_kernel(int P, const double *hi, int *phase, int *st, double *Tfinal) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P || phase[k] == PH_DONE) return;
    phase[k] = PH_DONE;
    Tfinal[k] = hi[k];
    st[k] = HOPF_MAXITER;
}

__global__ void ttr_candidates_kernel(int P, const double *lo, const double *hi, const int *phase,
                                      double *cand, int *active) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    int ph = phase[k];
    active[k] = ph != PH_DONE;
    cand[k] = ph == PH_HI ? hi[k] : (ph == PH_LO ? lo[k] : 0.5 * (lo[k] + hi[k]));
}

// Bracket update from the certified interval phi(T_cand) in [-P, -D]:
// P < 0 certifies phi > 0 (target not reached by T_cand); otherwise the
// point counts as reached (D > 0 certifies phi < 0; a gap that straddles zero
// is the ambiguous case and is flagged).
template <typename R>
__global__ void ttr_update_kernel(int P, double t_max, double tol_T, const double *cand,
                                  const int *active, const R *Pv, const R *Dv, const int *sst,
                                  double *lo, double *hi, int *phase, int *warm, int *st,
                                  double *Tfinal, int *remaining) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P || !active[k]) return;
    const double Pk = (double)Pv[k], Dk = (double)Dv[k];
    const bool reached = !(Pk < 0.0);
    if (sst[k] == HOPF_MAXITER && !(Pk < 0.0) && !(Dk > 0.0)) st[k] = HOPF_MAXITER;
    else if (sst[k] == HOPF_OK && !(Pk < 0.0) && !(Dk > 0.0) && st[k] == HOPF_OK) st[k] = HOPF_AMBIGUOUS_SIGN;
    const double c = cand[k];
    int ph = phase[k];
    if (ph == PH_HI) {
        if (reached) {
            ph = (warm[k] && lo[k] > 0.0) ? PH_LO : PH_BIS;
        } else if (warm[k]) {
            warm[k] = 0;
            lo[k] = 0.0;
            hi[k] = t_max;
            ph = PH_HI;
        } else {
            st[k] = HOPF_UNREACHABLE;
            Tfinal[k] = t_max;
            phase[k] = PH_DONE;
            return;
        }
    } else if (ph == PH_LO) {
        if (reached) {             // T* <= lo: fall back to [0, lo]
            warm[k] = 0;
            hi[k] = lo[k];
            lo[k] = 0.0;
        }
        ph = PH_BIS;
    } else {
        if (reached) hi[k] = c;
        else lo[k] = c;
    }
    if (ph == PH_BIS && hi[k] - lo[k] <= tol_T * hi[k]) {
        phase[k] = PH_DONE;
        Tfinal[k] = hi[k];
        return;
    }
    phase[k] = ph;
    atomicAdd(remaining, 1);
}

// Hybrid Newton/bisection of §IV (Eq. 26): every candidate is solved until
// the sign of phi is certified (or to the gap tolerance); the certified signs
// keep the bracket [lo, hi]; the next candidate is t + phi / H_x(p*, x0) with
// phi the middle of the certified interval and H_x(p, x0) =
// -x0^T A^T p + |-Q^T B^T p|_* (d phi / dT = -H_x), or the bracket midpoint
// when that step leaves the bracket.  A point stops when the step is below tol_T t, the bracket below
// tol_T hi, or the certified interval [-P, -D] contains zero.
__global__ void ttr_newton_start_kernel(int P, const double *hi, const int *phase, double *cand, int *active) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    active[k] = phase[k] != PH_DONE;
    cand[k] = hi[k];
}

template <typename R>
__global__ void ttr_newton_update_kernel(int P, int n, int m, int ctrl_kind, const double *__restrict__ A,
                                         const double *__restrict__ B, const double *__restrict__ qd,
                                         const R *__restrict__ x, double t_max, double tol_T, const R *Pv,
                                         const R *Dv, const R *pstar, double *cand, int *active, double *lo,
                                         double *hi, int *phase, int *st, double *Tfinal, int *remaining) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P || !active[k]) return;
    const double Pk = (double)Pv[k], Dk = (double)Dv[k], t = cand[k];
    const bool above = Pk < 0.0, below = Dk > 0.0;
    if (phase[k] == PH_HI && above && t < t_max) {   // a warm bracket too short: restart from t_max
        lo[k] = t;
        hi[k] = t_max;
        cand[k] = t_max;
        atomicAdd(remaining, 1);
        return;
    }
    if (phase[k] == PH_HI && above) {            // phi(t_max) > 0
        st[k] = HOPF_UNREACHABLE;
        Tfinal[k] = t_max;
        phase[k] = PH_DONE;
        active[k] = 0;
        return;
    }
    if (above) lo[k] = t;
    if (below) hi[k] = t;
    const R *pk = pstar + (long long)k * n;
    const R *xk = x + (long long)k * n;
    double H = 0.0;                              // -x0^T A^T p = -(A x0) . p
    for (int i = 0; i < n; ++i) {
        double ax = 0.0;
        for (int j = 0; j < n; ++j) ax = fma(A[i * n + j], (double)xk[j], ax);
        H -= ax * (double)pk[i];
    }
    double nrm = 0.0;                            // |-Q^T B^T p|_*
    for (int c = 0; c < m; ++c) {
        double g = 0.0;
        for (int i = 0; i < n; ++i) g = fma(B[i * m + c] * qd[c], (double)pk[i], g);
        nrm += ctrl_kind == HOPF_BALL ? g * g : fabs(g);
    }
    H += ctrl_kind == HOPF_BALL ? sqrt(nrm) : nrm;
    double tn = t - 0.5 * (Pk + Dk) / H;         // phi estimate: middle of [-P, -D]
    if (!isfinite(tn) || tn <= lo[k] || tn >= hi[k]) tn = 0.5 * (lo[k] + hi[k]);
    const bool done = !(above || below) || fabs(tn - t) <= tol_T * tn || hi[k] - lo[k] <= tol_T * hi[k];
    if (done) {
        phase[k] = PH_DONE;
        Tfinal[k] = t;
        active[k] = 0;
        return;
    }
    phase[k] = PH_BIS;
    cand[k] = tn;
    atomicAdd(remaining, 1);
}

template <typename R>
__global__ void ttr_finish_kernel(int P, const int *st, const int *fst, const double *Tfinal,
                                  R *T_star, int *status) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    int s = st[k];
    if (s == HOPF_OK && fst[k] != HOPF_OK) s = fst[k];
    status[k] = s;
    T_star[k] = (R)Tfinal[k];
}

// Trajectory from p*: one thread block per point.  With h = T/S, s_j = j h:
//   lambda_j = e^{-s_j A^T} p* = (e^{-hA})^T lambda_{j-1},
//   u_j = Q argmax_{c in U} <c, -Q^T B^T lambda_j>                  (Eq. 27)
//   x_j = e^{hA} x_{j-1} + h B u_j                                   (Eq. 33,
// the partial sums z_j = x0 + sum_{k<=j} h e^{-s_k A} B u_k mapped back by
// x_j = e^{s_j A} z_j, Eq. 9).
template <typename R>
__global__ void trajectory_kernel(const double *__restrict__ A, const double *__restrict__ B,
                                  const double *__restrict__ qd, int n, int m, int ctrl_kind, int P,
                                  const R *__restrict__ x, const R *__restrict__ T,
                                  const R *__restrict__ pstar, int S, R *__restrict__ xt,
                                  R *__restrict__ ut, double *scratch, const double *Eh_sh,
                                  const double *G_sh) {
    double *sc = scratch + (long long)blockIdx.x * (5LL * n * n + 4LL * n + 4LL * n * m + 48);
    double *X = sc, *T1 = X + n * n, *Eh = T1 + n * n, *G = Eh + n * n, *BQ = G + n * n;
    // one horizon for every point: e^{hA} and e^{-hA} computed once, shared
    if (Eh_sh) {
        Eh = const_cast<double *>(Eh_sh);
        G = const_cast<double *>(G_sh);
    }
    double *xs = BQ + n * m, *lam = xs + n, *tmp = lam + n, *tmp2 = tmp + n, *gv = tmp2 + n;
    double *red = gv + 2 * n * m;   // >= 8 doubles
    for (int k = blockIdx.x; k < P; k += gridDim.x) {
        const double Tk = (double)T[k];
        const double h = Tk / (double)S;
        if (!Eh_sh) {
            cta::expm(Eh, A, h, n, X, T1, red);     // e^{hA}
            cta::expm(G, A, -h, n, X, T1, red);     // e^{-hA}
        }
        for (int e = threadIdx.x; e < n * m; e += blockDim.x) BQ[e] = B[e] * qd[e % m];
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            xs[j] = (double)x[(long long)k * n + j];
            lam[j] = (double)pstar[(long long)k * n + j];
        }
        __syncthreads();
        for (int j = 0; j <= S; ++j) {
            if (j > 0) {
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    double s = 0.0;
                    for (int l = 0; l < n; ++l) s = fma(G[l * n + i], lam[l], s);
                    tmp[i] = s;
                }
                __syncthreads();
                for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = tmp[i];
                __syncthreads();
            }
            // g = -Q^T B^T lambda (Q folded into BQ), control u = Q argmax_U <c, g>
            for (int c = threadIdx.x; c < m; c += blockDim.x) {
                double s = 0.0;
                for (int r = 0; r < n; ++r) s = fma(BQ[r * m + c], lam[r], s);
                gv[c] = -s;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double nrm = 0.0;
                for (int c = 0; c < m; ++c) nrm = fma(gv[c], gv[c], nrm);
                nrm = sqrt(nrm);
                for (int c = 0; c < m; ++c) {
                    double cs;
                    if (ctrl_kind == HOPF_BALL) cs = nrm > 0.0 ? gv[c] / nrm : 0.0;
                    else cs = gv[c] >= 0.0 ? 1.0 : -1.0;
                    gv[m + c] = cs;                      // unit-set maximiser c*
                }
            }
            __syncthreads();
            if (j > 0) {
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    double s = 0.0;
                    for (int l = 0; l < n; ++l) s = fma(Eh[i * n + l], xs[l], s);
                    for (int c = 0; c < m; ++c) s = fma(h * BQ[i * m + c], gv[m + c], s);
                    tmp2[i] = s;
                }
                __syncthreads();
                for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = tmp2[i];
                __syncthreads();
            }
            R *xo = xt + ((long long)k * (S + 1) + j) * n;
            R *uo = ut + ((long long)k * (S + 1) + j) * m;
            for (int i = threadIdx.x; i < n; i += blockDim.x) xo[i] = (R)xs[i];
            for (int c = threadIdx.x; c < m; c += blockDim.x) uo[c] = (R)(qd[c] * gv[m + c]);
            __syncthreads();
        }
    }
}

template <typename R>
cudaError_t launch_ttr_init(int P, cudaStream_t s, const double *inst0, int n, int m, int N, const R *x,
                            const R *T_lo, const R *T_hi, double t_max, double *lo, double *hi, int *phase,
                            int *warm, int *st, double *Tfinal) {
    ttr_init_kernel<R><<<(P + 127) / 128, 128, 0, s>>>(inst0, n, m, N, P, x, T_lo, T_hi, t_max, lo, hi, phase,
                                                       warm, st, Tfinal);
    return cudaGetLastError();
}

cudaError_t launch_ttr_candidates(int P, cudaStream_t s, const double *lo, const double *hi, const int *phase,
                                  double *cand, int *active) {
    ttr_candidates_kernel<<<(P + 127) / 128, 128, 0, s>>>(P, lo, hi, phase, cand, active);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_ttr_update(int P, cudaStream_t s, double t_max, double tol_T, const double *cand,
                              const int *active, const R *Pv, const R *Dv, const int *sst, double *lo,
                              double *hi, int *phase, int *warm, int *st, double *Tfinal, int *remaining) {
    ttr_update_kernel<R><<<(P + 127) / 128, 128, 0, s>>>(P, t_max, tol_T, cand, active, Pv, Dv, sst, lo, hi,
                                                         phase, warm, st, Tfinal, remaining);
    return cudaGetLastError();
}

cudaError_t launch_ttr_newton_start(int P, cudaStream_t s, const double *hi, const int *phase, double *cand,
                                    int *active) {
    ttr_newton_start_kernel<<<(P + 127) / 128, 128, 0, s>>>(P, hi, phase, cand, active);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_ttr_newton_update(int P, cudaStream_t s, int n, int m, int ctrl_kind, const double *A,
                                     const double *B, const double *qd, const R *x, double t_max, double tol_T,
                                     const R *Pv, const R *Dv, const R *pstar, double *cand, int *active, double *lo,
                                     double *hi, int *phase, int *st, double *Tfinal, int *remaining) {
    ttr_newton_update_kernel<R><<<(P + 127) / 128, 128, 0, s>>>(P, n, m, ctrl_kind, A, B, qd, x, t_max, tol_T, Pv,
                                                                Dv, pstar, cand, active, lo, hi, phase, st, Tfinal,
                                                                remaining);
    return cudaGetLastError();
}

cudaError_t launch_ttr_cap(int P, cudaStream_t s, const double *hi, int *phase, int *st, double *Tfinal) {
    ttr_cap_kernel<<<(P + 127) / 128, 128, 0, s>>>(P, hi, phase, st, Tfinal);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_ttr_finish(int P, cudaStream_t s, const int *st, const int *fst, const double *Tfinal,
                              R *T_star, int *status) {
    ttr_finish_kernel<R><<<(P + 127) / 128, 128, 0, s>>>(P, st, fst, Tfinal, T_star, status);
    return cudaGetLastError();
}

// smallest and largest horizon of the batch (one block)
template <typename R>
__global__ void traj_minmax_kernel(int P, const R *__restrict__ T, double *out) {
    __shared__ double lo[256], hi[256];
    double a = 1e300, b = -1e300;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        const double t = (double)T[k];
        a = fmin(a, t);
        b = fmax(b, t);
    }
    lo[threadIdx.x] = a;
    hi[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            lo[threadIdx.x] = fmin(lo[threadIdx.x], lo[threadIdx.x + w]);
            hi[threadIdx.x] = fmax(hi[threadIdx.x], hi[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = lo[0];
        out[1] = hi[0];
    }
}

// e^{hA} and e^{-hA} for the shared horizon T (h = T / S), one block
__global__ void traj_shared_expm_kernel(const double *__restrict__ A, int n, int S, const double *TT,
                                        double *Eh, double *G, double *scratch) {
    double *X = scratch, *T1 = X + n * n, *red = T1 + n * n;
    const double h = TT[0] / (double)S;
    cta::expm(Eh, A, h, n, X, T1, red);
    cta::expm(G, A, -h, n, X, T1, red);
}

template <typename R>
cudaError_t launch_traj_minmax(int P, const R *T, double *out, cudaStream_t s) {
    traj_minmax_kernel<R><<<1, 256, 0, s>>>(P, T, out);
    return cudaGetLastError();
}

cudaError_t launch_traj_shared_expm(int threads, const double *A, int n, int S, const double *TT, double *Eh,
                                    double *G, double *scratch, cudaStream_t s) {
    traj_shared_expm_kernel<<<1, threads, 0, s>>>(A, n, S, TT, Eh, G, scratch);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_trajectory(int grid, int threads, cudaStream_t s, const double *A, const double *B,
                              const double *qd, int n, int m, int ctrl_kind, int P, const R *x, const R *T,
                              const R *pstar, int S, R *xt, R *ut, double *scratch, const double *Eh_sh,
                              const double *G_sh) {
    trajectory_kernel<R><<<grid, threads, 0, s>>>(A, B, qd, n, m, ctrl_kind, P, x, T, pstar, S, xt, ut, scratch,
                                                  Eh_sh, G_sh);
    return cudaGetLastError();
}

#define HOPF_TTR_INST(R)                                                                                  \
    template cudaError_t launch_ttr_init<R>(int, cudaStream_t, const double *, int, int, int, const R *,  \
                                            const R *, const R *, double, double *, double *, int *,      \
                                            int *, int *, double *);                                      \
    template cudaError_t launch_ttr_update<R>(int, cudaStream_t, double, double, const double *,          \
                                              const int *, const R *, const R *, const int *, double *,   \
                                              double *, int *, int *, int *, double *, int *);            \
    template cudaError_t launch_ttr_newton_update<R>(int, cudaStream_t, int, int, int, const double *,     \
                                                     const double *, const double *, const R *, double, double, \
                                                     const R *, const R *, const R *, double *, int *, double *, \
                                                     double *, int *, int *, double *, int *);                  \
    template cudaError_t launch_ttr_finish<R>(int, cudaStream_t, const int *, const int *,                \
                                              const double *, R *, int *);                                \
    template cudaError_t launch_trajectory<R>(int, int, cudaStream_t, const double *, const double *,     \
                                              const double *, int, int, int, int, const R *, const R *,   \
                                              const R *, int, R *, R *, double *, const double *,         \
                                              const double *);                                            \
    template cudaError_t launch_traj_minmax<R>(int, const R *, double *, cudaStream_t);
HOPF_TTR_INST(float)
HOPF_TTR_INST(double)

}  // namespace hopf
