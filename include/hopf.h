/*
 * hopf.h - C ABI of the GB300 generalized-Hopf primal-dual solver.
 *
 * The library evaluates, for very many independent query points at once,
 * the generalized Hopf formula for the linear system  xdot = A x + B u
 * (Kirchner, Hewer, Darbon, Osher, "A Primal-Dual Method for Optimal Control
 * and Trajectory Generation in High-Dimensional Systems"):
 *
 *   phi(x, T) = -min_p { J_z*(p) + sum_i w_i |K_i p|_* - <x, p> }      (Eq. 18)
 *   K_i = (-e^{-(T - t_i) A} B Q)^T                                      (Eq. 20)
 *
 * with a ball or box control set (support function = dual norm, §III.A,
 * Eq. 16) and the ellipsoidal target  { x : x^T W^-1 x <= 1 }  whose terminal
 * cost is J_x(x) = x^T W^-1 x - 1 (§VI.A, Eq. 34 - Eq. 35).  The minimisation
 * is the Chambolle-Pock iteration of Eq. 15 with the separable prox of
 * Eq. 23 and the quadratic prox of Eq. 37.  On top of it sit the minimum
 * time to reach the target (§IV) and the optimal control and trajectory
 * generated from the optimal dual p* (Eq. 27, Eq. 33).
 *
 * Conventions shared by every entry point
 *  - Problem matrices (A, B, W, half_widths) are HOST float64 arrays, row
 *    major, read during the call only; the caller keeps ownership.
 *  - Per-point arrays (x, t, outputs) are caller-owned DEVICE arrays unless
 *    opts->host_io is non-zero, in which case they are HOST arrays and the
 *    library copies them to and from the device inside the call (the call
 *    then returns after the results are back on the host).
 *  - Element type of per-point float arrays: double when opts->precision is
 *    HOPF_FP64, float otherwise.  Integer outputs are int32.
 *  - Calls are ordered on `stream` (a cudaStream_t, NULL = legacy default
 *    stream).  hopf_value and hopf_trajectory do not synchronise the host
 *    unless host_io is set; hopf_time_to_reach reads one int32 per
 *    bisection step back to the host to know when every point has finished.
 *  - The library keeps a grow-only device workspace per device and stream
 *    (released by hopf_release_workspace): calls on one stream reuse it in
 *    stream order, calls on different streams use different workspaces and
 *    may overlap on the GPU (e.g. several systems at once).  Concurrent calls
 *    from several host threads are serialised by an internal lock (the GPU
 *    work they enqueue still runs asynchronously).
 *  - Return value: HOPF_SUCCESS (0) or a negative HOPF_E* code; the message
 *    of the last failure is available from hopf_last_error().  Per-point
 *    outcomes are reported separately in status[] (HOPF_OK, ...).
 */
#ifndef HOPF_GB300_H
#define HOPF_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

/* control set kinds (§III.A) */
#define HOPF_BALL 0 /* {u : |u|_2 <= radius}; dual norm = 2-norm            */
#define HOPF_BOX 1  /* {u : |u_j| <= half_widths[j]}; dual norm = 1-norm     */

/* quadrature rules (§III.A, Eq. 17 and the trapezoid rule it mentions) */
#define HOPF_LEFT_RIEMANN 0 /* t_i = i T/N, i = 0..N-1, weights T/N          */
#define HOPF_TRAPEZOID 1    /* t_i = i T/(N-1), end weights halved           */
#define HOPF_SIMPSON 2      /* composite Simpson: N odd, t_i = i T/(N-1),
                               weights T/(3(N-1)) (1, 4, 2, 4, ..., 2, 4, 1)   */
#define HOPF_LEFT_FIXED 3   /* left Riemann sum with the fixed step
                               dt = t_max/N (another quadrature of the kind
                               §III.A allows): nodes t_i = i dt with t_i < T,
                               weights dt, the last one T - t_last; Eq. 17
                               with k nodes at T = k dt.  Needs terminal-time
                               variables (the table on [0, t_max] then serves
                               every horizon), a finite t_max >= every horizon
                               (a horizon outside [0, t_max] gets phi = NaN and
                               HOPF_NONFINITE), n <= 512, adaptive = 0; not
                               for hopf_value_warm, hopf_value_stacked,
                               hopf_value_noalloc or hopf_node_table.  float32
                               runs the tiled kernel (17 <= n <= 256) or the
                               general one, never the tensor-core kernel.     */

/* arithmetic of the iteration */
#define HOPF_FP64 0 /* float64 everywhere                                    */
#define HOPF_FP32 1 /* float64 tables, float32 iteration and certificates    */

/* per-point status */
#define HOPF_OK 0             /* certified: relative duality gap <= tol_gap      */
#define HOPF_MAXITER 1        /* max_iter reached; outputs are the last iterate  */
#define HOPF_NONFINITE 2      /* NaN/Inf met in the iteration                    */
#define HOPF_UNREACHABLE 3    /* time-to-reach: phi(x, t_max) > 0                */
#define HOPF_AMBIGUOUS_SIGN 4 /* time-to-reach: |phi| below the certificate    */

/* return codes */
#define HOPF_SUCCESS 0
#define HOPF_EINVAL (-1)       /* bad size, pointer or option                   */
#define HOPF_ENOTSPD (-2)      /* W is not symmetric positive definite          */
#define HOPF_ECUDA (-3)        /* a CUDA runtime call failed                    */
#define HOPF_ENOMEM (-4)       /* device allocation failed                      */
#define HOPF_ENONFINITE (-5)   /* non-finite A, B, W or bounds                  */
#define HOPF_ESCRATCH (-6)     /* hopf_value_noalloc: the call does not fit the
                                  library's static scratch array               */

typedef struct {
    int n;                      /* state dimension, >= 1                         */
    int m;                      /* control dimension, >= 1                       */
    const double *A;            /* host, n*n row-major: xdot = A x + B u (Eq. 8) */
    const double *B;            /* host, n*m row-major                            */
    int ctrl_kind;              /* HOPF_BALL or HOPF_BOX                          */
    double radius;              /* ball radius (HOPF_BALL), > 0                   */
    const double *half_widths;  /* host, m, > 0 (HOPF_BOX; ignored for a ball)    */
    const double *W;            /* host, n*n SPD: target {x : x^T W^-1 x <= 1}    */
} hopf_problem;

typedef struct {
    int rule;           /* HOPF_LEFT_RIEMANN, _TRAPEZOID, _SIMPSON or _LEFT_FIXED */
    int N;              /* quadrature nodes (>= 1; >= 2 trapezoid; odd >= 3 Simpson;
                           fixed step: nodes on [0, t_max]) */
    int max_iter;       /* iteration cap per solve                                */
    int gap_every;      /* duality-gap check period g (>= 1)                      */
    int precision;      /* HOPF_FP64 or HOPF_FP32                                 */
    int host_io;        /* 0: per-point arrays are device pointers; 1: host       */
    double tau;         /* primal step (> 0)                                      */
    double sigma_scale; /* dual step sigma = sigma_scale / (tau |K|^2), (0, 1]    */
    double tol_gap;     /* stop when (P - D) / max(1, |P|, |D|) <= tol_gap        */
    double t_max;       /* time-to-reach: bisection bracket [0, t_max]            */
    double tol_T;       /* time-to-reach: stop when hi - lo <= tol_T * hi         */
    int profile;        /* non-zero: record CUDA events around the table build
                           and the solve kernel of hopf_value (see
                           hopf_last_profile)                                     */
    int accel;          /* 0: the iteration of Eq. 15 with theta = 1 (§VI).
                           1: the accelerated variant for a strongly convex G
                           that §III names (Chambolle and Pock 2011, Alg. 2):
                           G of Eq. 36 is gamma-strongly convex with
                           gamma = lambda_min(M)/2; after each step
                           theta = 1/sqrt(1 + 2 gamma tau), tau *= theta,
                           sigma /= theta, pbar = p + theta (p - p_old).  The
                           starting tau is opts->tau.                             */
    int park_iters;     /* small-state float32 solves run in up to three phases:
                           4 lanes per point, 32 lanes per point, one thread
                           block per point (less work per iteration first,
                           lower latency per iteration later).  A point moves
                           on after park_iters iterations in a phase (5x that
                           in the second), or as soon as its phase has no new
                           point left to start.  0 = library default (4096);
                           < 0 = first phase only.                                */
    int newton;         /* hopf_time_to_reach: 0 = bisection with certified signs;
                           1 = the hybrid of §IV: Newton steps
                           t + phi / H_x(p*, x) (Eq. 26) inside the certified
                           bracket, midpoint when a step leaves it; every
                           candidate is solved to tol_gap.                        */
    int kernel;         /* hopf_value solve kernel: HOPF_KERNEL_AUTO (0) picks by
                           size; HOPF_KERNEL_GENERIC (1) forces one warp per
                           point (the reference layout of the iteration; used
                           to compare the specialised kernels with it);
                           HOPF_KERNEL_TENSOR (2) asks for the tensor-core
                           kernel wherever it applies (float32, one horizon,
                           terminal-time variables, diagonal W, accel 0,
                           16 <= n <= 256), else AUTO's choice among the others;
                           HOPF_KERNEL_TILE (3) the CUDA-core tiled kernel for
                           large states.                                          */
    int variables;      /* variable the iteration of Eq. 15 runs in.
                           HOPF_VARS_INITIAL (0): the paper's p of Eq. 18.
                           HOPF_VARS_TERMINAL (1): q with p = e^{T A^T} q (the
                           costate carried to the terminal time).  The
                           minimisation is the same (Eq. 18 with
                           K'_i = (-e^{t_i A} B Q)^T = K_i e^{T A^T}, M' = W and
                           z0' = e^{TA} z0), so phi, the certified gap and p* (mapped
                           back) are the same quantities; the iterates differ
                           and usually need far fewer steps, because the
                           quadratic term q^T W q is as well conditioned as W
                           while e^{-TA} W e^{-TA^T} is not.  Inputs (x, p_init)
                           and p_star stay in the paper's variable.               */
    int max_steps;      /* hopf_time_to_reach: cap on the candidate horizons solved
                           per point (0 = 256).  A point still open at the cap
                           returns T_star = the top of its bracket and the status
                           HOPF_MAXITER.                                          */
    int adaptive;       /* 1: step sizes balanced on the two residuals §III.B uses
                           for its stopping rule (the adaptive PDHG of Goldstein
                           et al. cited there): after each step, if
                           |r_p| > 1.5 |r_d| then tau /= (1 - a), sigma *= (1 - a),
                           if 1.5 |r_p| < |r_d| the reverse, then a *= 0.95
                           (a starts at 0.5; tau sigma stays 1/|K|^2).  Runs on
                           the general warp-per-point kernel; not with accel,
                           the warm start or the stacked solve.                  */
} hopf_opts;

#define HOPF_KERNEL_AUTO 0
#define HOPF_KERNEL_GENERIC 1
#define HOPF_KERNEL_TENSOR 2
#define HOPF_KERNEL_TILE 3

#define HOPF_VARS_INITIAL 0
#define HOPF_VARS_TERMINAL 1

/* Fills *opts with the defaults: left Riemann, N = 100 (§VI), max_iter 100000,
 * gap_every 8, FP32, device io, tau 1, sigma_scale 1 (§VI: sigma = 1/(tau |K|^2)),
 * tol_gap 1e-5, t_max 10, tol_T 1e-5, no profiling, accel 0, variables
 * HOPF_VARS_INITIAL.
 * A point counts as converged when its computed relative gap plus an
 * allowance for the rounding of P and D (4 u (|P parts| + |D| + 1) / scale,
 * u the unit roundoff of the iteration's precision) is <= tol_gap. */
void hopf_default_opts(hopf_opts *opts);

/*
 * hopf_value - phi(x_k, t_k) of Eq. 18 for P query points (§III.A, §VI).
 *   x       [P*n]  query states (at time zero, so z0 = x, Eq. 9)
 *   t       [1] if t_stride == 0 (one horizon for every point: one shared
 *           node table), else [P] per-point horizons (t_stride == 1; one table
 *           per point).  t >= 0; t = 0 gives phi = J_x(x).  With
 *           HOPF_LEFT_FIXED one table on [0, opts->t_max] serves every
 *           horizon; a t outside [0, t_max] gives phi = NaN, p_star = NaN and
 *           HOPF_NONFINITE for that point.
 *   p_init  NULL (cold start of §VI: p0 = x, y0 = K x) or [P*n] warm start
 *           (p0 = p_init, y0_i = w_i argmax_{c in U} <c, K_i p0>).
 *   phi     [P]    -P(pbar): certified to lie within gap of the exact value
 *   p_star  [P*n]  the primal point of the certificate (approximates p*, Eq. 24)
 *   gap     [P]    relative duality gap of the certificate
 *   iters   [P]    iterations used
 *   status  [P]    HOPF_OK / HOPF_MAXITER / HOPF_NONFINITE
 * P = 0 is allowed and does nothing.
 */
int hopf_value(const hopf_problem *prob, const hopf_opts *opts, int P,
               const void *x, const void *t, int t_stride, const void *p_init,
               void *phi, void *p_star, void *gap, int *iters, int *status,
               void *stream);

/*
 * Stacked copies (§VI.B unscented control, §VI.C dimensional scaling): k
 * copies of a base system (n_b states, m controls) driven by ONE shared
 * control.  The stacked state is x = (chi_1, ..., chi_k) (n = k n_b),
 * A~ = blockdiag(A, ..., A), B~ = (B; ...; B), and the target is
 * {x : x^T W~^-1 x <= 1} with W~ = blockdiag(W_1, ..., W_k).
 */
typedef struct {
    hopf_problem base;          /* n_b = base.n <= 8, m <= 16, A, B and the control
                                   set of one copy; base.W is not used            */
    int copies;                 /* k, 1 <= k <= 64                                */
    const double *W_blocks;     /* host, k * n_b * n_b: the SPD blocks W_j        */
} hopf_stacked;

/*
 * hopf_value_stacked - hopf_value for a stacked-copy system, with the
 * structure used instead of the dense n x n stacked table: the node matrix of
 * the stacked system is K~_i = (K_i, ..., K_i) (K_i of the base system,
 * Eq. 20), so K~_i p = K_i (p_1 + ... + p_k) and K~^T y = (K^T y, ..., K^T y),
 * |K~|^2 = k |K|^2, and M~, V~, S~ (Eq. 35, 37) are block diagonal.  Work per
 * iteration and point: 4 N m n_b + O(k n_b^2).  Arguments, layouts and status
 * as hopf_value with n = k n_b; per-point arrays must be device arrays
 * (host_io = 0); accel must be 0.
 */
int hopf_value_stacked(const hopf_stacked *prob, const hopf_opts *opts, int P, const void *x,
                       const void *t, int t_stride, const void *p_init, void *phi, void *p_star,
                       void *gap, int *iters, int *status, void *stream);

/*
 * hopf_time_to_reach - minimum time T* with phi(x, T*) <= 0 (§IV), by
 * bisection on [lo_k, hi_k] (default [0, opts->t_max]).  The sign of phi at a
 * candidate horizon is read from the certified interval phi in [-P, -D]; the
 * iteration at that horizon stops as soon as the interval excludes zero.
 *   x        [P*n]
 *   (opts->tol_T >= 4 DBL_EPSILON; opts->t_max finite and > 0)
 *   T_lo,T_hi NULL, or [P] per-point bracket (warm start: a bracket known to
 *            contain T*; a wrong bracket is detected by the two end-point signs
 *            and replaced by [0, t_max])
 *   (HOPF_LEFT_FIXED: one float64 table on [0, t_max] for every point and
 *   candidate, no per-point tables; each inner solve starts from the point's
 *   previous solution, the first from p_init or cold)
 *   p_init   NULL or [P*n]: warm start of every inner solve
 *   T_star   [P]  hi at termination (0 inside the target; t_max if unreachable)
 *   p_star   [P*n] certificate primal point at T_star (solved to tol_gap)
 *   gap      [P]  relative gap of that final solve
 *   status   [P]  HOPF_OK / HOPF_UNREACHABLE / HOPF_MAXITER / HOPF_AMBIGUOUS_SIGN
 *   steps    NULL or host int*: number of bisection steps taken
 */
int hopf_time_to_reach(const hopf_problem *prob, const hopf_opts *opts, int P,
                       const void *x, const void *T_lo, const void *T_hi,
                       const void *p_init, void *T_star, void *p_star, void *gap,
                       int *status, int *steps, void *stream);

/*
 * hopf_trajectory - optimal control and state on S uniform steps of [0, T_k]
 * generated from p*_k (§IV Eq. 27, §V Eq. 33).  With h = T/S and s_j = j h:
 *   u_j = Q argmax_{c in U} <c, -Q^T B^T e^{-s_j A^T} p*>,
 *   x_j = e^{h A} x_{j-1} + h B u_j,  x_0 = x,
 * which is the variation-of-constants sum of Eq. 33 in the variable x.
 *   x       [P*n], T [P] (>= 0), p_star [P*n]
 *   x_traj  [P*(S+1)*n]  point-major, then sample, then state
 *   u_traj  [P*(S+1)*m]  (u_0 is the control at s = 0)
 */
int hopf_trajectory(const hopf_problem *prob, const hopf_opts *opts, int P,
                    const void *x, const void *T, const void *p_star, int S,
                    void *x_traj, void *u_traj, void *stream);

/*
 * hopf_node_table - the float64 node table that the solves build for one
 * horizon T (§III.A): node matrices of Eq. 20 generated on the device by
 * repeated multiplication with e^{-hA} (e^{hA} in terminal-time variables)
 * and the quadrature weights of Eq. 17 (or of opts->rule).
 *   K  [N*m*n]  node-major, then control, then state:
 *               K_i = (-e^{-(T - t_i) A} B Q)^T for HOPF_VARS_INITIAL,
 *               K'_i = (-e^{t_i A} B Q)^T for HOPF_VARS_TERMINAL
 *   w  [N]      weights
 * Device arrays, or host arrays when opts->host_io (then the call waits for
 * the copy).  T must be finite and >= 0.
 */
int hopf_node_table(const hopf_problem *prob, const hopf_opts *opts, double T, double *K, double *w,
                    void *stream);

/* Human-readable name of a per-point status or a return code. */
const char *hopf_status_string(int code);

/* Message of the most recent failed call on this host thread ("" if none). */
const char *hopf_last_error(void);

/* Frees the library's device workspaces (every stream) on the current device;
 * waits for the device first. */
int hopf_release_workspace(void);

/* Device time of the phases of the most recent hopf_value call made with
 * opts->profile set: node-table build and the primal-dual solve kernel, in
 * milliseconds, measured with CUDA events on the call's stream.  Waits for
 * the call to finish.  Returns HOPF_EINVAL if no profiled call was made. */
int hopf_last_profile(double *ms_tables, double *ms_solve);

/* ------------------------------------------------------------------------
 * Learned warm start.  The paper has no learned part; these entry points
 * serve the warm-started batched solve: a small network predicts p* from x,
 * the primal-dual iteration starts from the prediction, and any point whose
 * warm solve is not certified is solved again from the cold start of §VI.
 *
 * Network: n_in -> hidden -> hidden -> n_out, exact GELU after each hidden
 * layer, inputs standardised by (x - x_shift)/x_scale, outputs mapped back by
 * out * y_scale + y_shift.  Weights are used as bfloat16, all products
 * accumulate in float32; a float32 master copy is kept for training.
 * Parameter layout (both copies): W1[hidden][n_in], b1[hidden],
 * W2[hidden][hidden], b2[hidden], W3[n_out][hidden], b3[n_out], row-major.
 * All pointers are caller-owned device arrays.
 * ---------------------------------------------------------------------- */
typedef struct {
    int n_in, hidden, n_out;
    float *w;                 /* float32 master parameters, hopf_mlp_param_count() */
    void *w_bf16;             /* bfloat16 copy used by the products, same count    */
    float *adam_m, *adam_v;   /* optimiser moments (training only; may be NULL)     */
    const float *x_shift, *x_scale;   /* [n_in]  */
    const float *y_shift, *y_scale;   /* [n_out] */
    int use_tc;               /* prediction (hopf_mlp_forward, hopf_value_warm) on
                                 the tensor cores: tcgen05 MMA with bfloat16
                                 activations and weights, float32 accumulation
                                 (hidden, n_out <= 256); 0: float32 CUDA-core
                                 products with bfloat16 weights.  Training
                                 (hopf_mlp_loss_grad) always uses the latter.    */
} hopf_mlp;

/* Number of parameters of the network (weights and biases). */
long long hopf_mlp_param_count(int n_in, int hidden, int n_out);

/* Refreshes the bfloat16 copy from the float32 master parameters. */
int hopf_mlp_sync(const hopf_mlp *net, void *stream);

/* y[B][n_out] = prediction for x[B][n_in] (physical units). */
int hopf_mlp_forward(const hopf_mlp *net, int B, const float *x, float *y, void *stream);

/* Mean squared error of the standardised output against the standardised
 * target y[B][n_out], written to *loss (device float), and its gradient with
 * respect to every parameter (grad: param_count floats, device). */
int hopf_mlp_loss_grad(const hopf_mlp *net, int B, const float *x, const float *y, float *loss,
                       float *grad, void *stream);

/* One Adam step (bias-corrected, step >= 1) on the master parameters with
 * gradient grad; refreshes the bfloat16 copy. */
int hopf_mlp_adam(const hopf_mlp *net, const float *grad, int step, double lr, double beta1,
                  double beta2, double eps, void *stream);

/*
 * hopf_value_warm - hopf_value (float32 only) with the network's prediction
 * as the warm start p_init.  Each warm solve runs at most max_iter_warm
 * iterations; a point that is not certified (status != HOPF_OK) is solved
 * again from the cold start with opts->max_iter, and its outputs are those of
 * the cold solve.  Outputs as in hopf_value (host arrays when opts->host_io;
 * the network's parameters are always device arrays).  n_fallback: NULL or an
 * int (device, or host when opts->host_io) that receives the number of points
 * solved again.  With opts->profile, hopf_last_profile reports the table build
 * plus network prediction as ms_tables and both solves as ms_solve.
 */
int hopf_value_warm(const hopf_problem *prob, const hopf_opts *opts, const hopf_mlp *net, int P,
                    const void *x, const void *t, int t_stride, int max_iter_warm,
                    void *phi, void *p_star, void *gap, int *iters, int *status,
                    int *n_fallback, void *stream);

/*
 * hopf_tc_selftest - diagnostic of the library's tcgen05 tensor-core
 * primitives (shared-memory operand descriptors, instruction descriptor,
 * tensor-memory accumulator and its read-back), which the warm-start
 * network's tensor-core prediction uses; no counterpart in the paper.  One
 * thread block computes D[128][N] = A[128][K] B[N][K]^T with tcgen05.mma of
 * kind::tf32 (float32 accumulation in tensor memory) and writes D.  Device
 * arrays, row-major; 16 <= N <= 256 (multiple of 16), 8 <= K <= 128 (multiple
 * of 8).  *err (device int) is set to 1 if the completion wait timed out.
 */
int hopf_tc_selftest(int N, int K, const float *A, const float *B, float *D, int *err, void *stream);

/*
 * hopf_value_noalloc - hopf_value for callers that cannot allocate memory.
 *
 * The paper has no counterpart; this is a deployment variant.  Some callers
 * must not allocate at solve time: a hard real-time control loop (a device
 * allocation can synchronise the whole device and has no time bound), or a
 * process whose memory footprint is fixed after start-up (for instance one
 * sharing the GPU under a fixed memory quota).
 * This entry point takes all of its scratch (a copy of A, B, Q and W, the node
 * tables, and each point's dual variable) from one static device array of
 * HOPF_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits, and calls no cudaMalloc, cudaFree or other allocating
 * routine.  It always runs the general warp-per-point kernel.
 *
 * Arguments and results are those of hopf_value, with these limits:
 *   - opts->host_io must be 0 (x, t, p_init and outputs are device arrays);
 *   - n <= HOPF_NOALLOC_MAX_N, m <= 16;
 *   - opts->variables must be HOPF_VARS_INITIAL;
 *   - the scratch the call needs must fit the array, about
 *     8 (n_tables (N m n + N + 7 n^2 + n) + 9 n^2) + P N m sizeof(element)
 *     bytes with n_tables = 1 (t_stride 0) or P (t_stride 1); otherwise the
 *     call returns HOPF_ESCRATCH and does nothing.
 *   Validation failures return the codes of hopf_value; hopf_last_error() is
 *   not updated by this entry point.
 *
 * The first call on a device looks up the array's device address with that
 * device current and keeps it; make that first call before any stream
 * capture.  Every call shares the one array and it keeps the last call's
 * contents (no part of it needs to start at zero: a call writes every scratch
 * byte before reading it).  Calls that overlap on the GPU - on different
 * streams, or from host threads without ordering between them - race on the
 * array and give wrong results; calls ordered on one stream are safe.
 */
#define HOPF_NOALLOC_SCRATCH_BYTES (32 * 1024 * 1024)
#define HOPF_NOALLOC_MAX_N 64
int hopf_value_noalloc(const hopf_problem *prob, const hopf_opts *opts, int P,
                       const void *x, const void *t, int t_stride, const void *p_init,
                       void *phi, void *p_star, void *gap, int *iters, int *status,
                       void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HOPF_GB300_H */
