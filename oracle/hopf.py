"""FP64 CPU oracle for the generalized Hopf formula solved by primal-dual splitting.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
It shares no code with the CUDA library (it does not import the package and
the package does not import it); both sides only share the seeded input
generators in ``inputs``.

Everything is plain float64 numpy, written to be read side by side with the
paper (Kirchner, Hewer, Darbon, Osher, "A Primal-Dual Method for Optimal
Control and Trajectory Generation in High-Dimensional Systems"):

  * quadrature nodes and weights ............ §III.A, Eq. 17 (+ trapezoid rule,
                                              + the fixed-step left sum FixedStep)
  * node matrices K_i ....................... §III.A, Eq. 16 and Eq. 20
  * quadratic terminal cost and its conjugate §VI.A, Eq. 34 - Eq. 37
  * primal-dual iteration ................... §III, Eq. 15 with Eq. 22, Eq. 23, Eq. 37
  * accelerated iteration for a strongly convex G (named in §III, from
    Chambolle and Pock 2011, Algorithm 2) ..... pdhg(..., accel=True)
  * the same minimisation in terminal-time variables p = e^{T A^T} q
    (an exact substitution in Eq. 18; a preconditioning of Eq. 15) ......
                                              setup(..., variables="terminal")
  * duality gap (stopping rule) ............. §III.B (primal/dual residuals) and
                                              the Fenchel dual of Eq. 18
  * time-to-reach ........................... §IV (zero of phi(x, T) in T, bisection)
  * optimal control ......................... §IV, Eq. 27
  * trajectory .............................. §V, Eq. 29 and Eq. 33

Batched code only stacks independent query points along the leading axis;
the arithmetic per point is exactly the formula it cites.

Pins (tests/test_oracle_*.py) tie every function to something other than
itself: the closed-form single-integrator value and time-to-reach, the
closed-form double-integrator node table, an independent projected-gradient
solver of the discrete-control problem, exhaustive active-set enumeration on
tiny problems, the gradient identity p* = grad phi (Eq. 24), the HJ identity
d phi / dT = -H_x (§IV), the terminal-point identity (Eq. 29) and the
bang-bang switching-curve time of the double integrator.  The fixed-step
rule is pinned by an independent walk of its partition, its reduction to
Eq. 17 at multiples of the step, the single-integrator time to reach at every
horizon and FISTA on the primal-control form with the partition's nodes.
"""
import numpy as np
from scipy.linalg import expm

BALL, BOX = 0, 1
LEFT_RIEMANN, TRAPEZOID, SIMPSON = 0, 1, 2

OK, MAXITER, NONFINITE, UNREACHABLE, AMBIGUOUS_SIGN = 0, 1, 2, 3, 4


# ----------------------------------------------------------------- quadrature
class FixedStep:
    """Left Riemann sum with a step that does not depend on T: dt = t_max / N.

    §III.A takes N equal steps of T / N and allows other quadratures.  Here
    the step is fixed: the nodes are t_i = i dt for every i >= 0 with
    t_i < T, each weighted dt, except the last, weighted T - t_last.  This is
    the left Riemann sum of the partition {0, dt, 2 dt, ..., t_last, T}; at
    T = k dt it is Eq. 17 with k nodes.  In terminal-time variables the node
    matrices (-e^{t_i A} B Q)^T do not depend on T, so one table on
    [0, t_max] serves every horizon (the nodes of horizon T are a prefix of
    it).  N is the node count of that table: at most N nodes, T <= t_max."""

    def __init__(self, t_max, N):
        self.t_max = float(t_max)
        self.N = int(N)
        self.dt = self.t_max / self.N

    def count(self, T):
        """Number of nodes of horizon T > 0: the i >= 0 with i dt < T."""
        if not (0.0 < T <= self.t_max):
            raise ValueError("the fixed-step rule needs 0 < T <= t_max")
        return min(max(int(np.ceil(T / self.dt)), 1), self.N)

    def __eq__(self, other):
        return isinstance(other, FixedStep) and (other.t_max, other.N) == (self.t_max, self.N)


def nodes(T, N, rule):
    """Quadrature in Hopf time on [0, T].

    Left Riemann sum (§III.A, Eq. 17): t_i = i T/N, i = 0..N-1, weights T/N.
    Trapezoid rule (named in §III.A as an alternative): N samples including
    both ends, t_i = i T/(N-1), weights T/(N-1) with the two end weights halved.
    Composite Simpson rule (also named there): N odd samples including both
    ends, t_i = i h with h = T/(N-1), weights h/3 (1, 4, 2, 4, ..., 2, 4, 1).
    FixedStep(t_max, N): t_i = i dt (dt = t_max/N) while t_i < T, weights dt,
    the last one T - t_last (len(t) <= N nodes).
    Returns (t, w)."""
    if isinstance(rule, FixedStep):
        k = rule.count(T)
        t = np.arange(k, dtype=np.float64) * rule.dt
        w = np.full(k, rule.dt)
        w[-1] = T - (k - 1) * rule.dt
    elif rule == LEFT_RIEMANN:
        t = np.arange(N, dtype=np.float64) * (T / N)
        w = np.full(N, T / N)
    elif rule == TRAPEZOID:
        h = T / (N - 1)
        t = np.arange(N, dtype=np.float64) * h
        w = np.full(N, h)
        w[0] *= 0.5
        w[-1] *= 0.5
    elif rule == SIMPSON:
        if N < 3 or N % 2 == 0:
            raise ValueError("Simpson's rule needs an odd number of nodes >= 3")
        h = T / (N - 1)
        t = np.arange(N, dtype=np.float64) * h
        w = np.where(np.arange(N) % 2 == 1, 4.0, 2.0) * (h / 3.0)
        w[0] = w[-1] = h / 3.0
    else:
        raise ValueError("unknown quadrature rule")
    return t, w


# ------------------------------------------------------------ control set U
def control_scaling(sysd):
    """Q of §III.A (Eq. 16): the control set is Q applied to a unit set.
    Ball {|u|_2 <= rho}: Q = rho I, unit 2-ball.  Box {|u_j| <= b_j}: Q = diag(b),
    unit infinity-ball."""
    m = sysd["B"].shape[1]
    if sysd["ctrl_kind"] == BALL:
        return sysd["radius"] * np.eye(m)
    return np.diag(np.asarray(sysd["half_widths"], dtype=np.float64))


def dual_norm(kind, v):
    """Support function of the unit control set, i.e. the dual norm of §III.A:
    2-norm for the unit ball, 1-norm for the unit box.  v has shape (..., m)."""
    if kind == BALL:
        return np.sqrt(np.sum(v * v, axis=-1))
    return np.sum(np.abs(v), axis=-1)


def project_scaled(kind, v, r):
    """Euclidean projection of v onto r * U (unit set U), the prox of the
    indicator F_i* = I_{w_i U} of Eq. 22 used in Eq. 23.  v (..., m), r (...,)."""
    if kind == BALL:
        nv = np.sqrt(np.sum(v * v, axis=-1))
        scale = np.where(nv > r, r / np.where(nv > 0, nv, 1.0), 1.0)
        return v * scale[..., None]
    return np.clip(v, -r[..., None], r[..., None])


def argmax_unit(kind, v):
    """argmax over the unit set U of <c, v> (the gradient of the support
    function, used for the optimal control of Eq. 27).  Ball: v/|v| (0 at v = 0).
    Box: sign(v) with sign(0) = +1 as defined in §VI.A."""
    if kind == BALL:
        nv = np.sqrt(np.sum(v * v, axis=-1, keepdims=True))
        return np.where(nv > 0, v / np.where(nv > 0, nv, 1.0), 0.0)
    return np.where(v >= 0, 1.0, -1.0)


# ------------------------------------------------------------ problem data
def node_matrices(sysd, T, N, rule):
    """K_i = (-e^{-(T - t_i) A} B Q)^T for every node (Eq. 20), stacked as an
    array of shape (N, m, n).  Each matrix exponential is evaluated directly
    with scipy's expm (one call per node)."""
    A, B = sysd["A"], sysd["B"]
    Q = control_scaling(sysd)
    t, _ = nodes(T, N, rule)
    K = np.empty((t.size, B.shape[1], A.shape[0]))
    for i in range(t.size):
        K[i] = -(expm(-(T - t[i]) * A) @ B @ Q).T
    return K


def node_matrices_terminal(sysd, T, N, rule):
    """Node matrices of Eq. 18 after the substitution p = e^{T A^T} q:
    K_i e^{T A^T} = (-e^{-(T - t_i) A} B Q)^T e^{T A^T} = (-e^{t_i A} B Q)^T,
    shape (N, m, n), one direct expm per node (forward times t_i of Eq. 17)."""
    A, B = sysd["A"], sysd["B"]
    Q = control_scaling(sysd)
    t, _ = nodes(T, N, rule)
    K = np.empty((t.size, B.shape[1], A.shape[0]))
    for i in range(t.size):
        K[i] = -(expm(t[i] * A) @ B @ Q).T
    return K


def terminal_matrices(sysd, T):
    """Quadratic target cost of §VI.A.  J_x(x) = x^T W^-1 x - 1 (Eq. 34), so
    J_z(z) = z^T V z - 1 with V = e^{T A^T} W^-1 e^{T A}, and its conjugate is
    J_z*(p) = p^T V^-1 p / 4 + 1 (Eq. 35), where V^-1 = e^{-TA} W e^{-TA^T}.
    Returns (M, V) with M = V^-1."""
    A, W = sysd["A"], sysd["W"]
    E = expm(-T * A)
    M = E @ W @ E.T
    M = 0.5 * (M + M.T)
    V = np.linalg.inv(M)
    return M, 0.5 * (V + V.T)


def setup(sysd, T, N, rule, tau, sigma_scale=1.0, variables="initial"):
    """All data of one primal-dual problem at horizon T.

    K (N, m, n) from Eq. 20, weights w (N,), M and V (Eq. 35), the prox matrix
    S = (I + tau M / 2)^-1 of Eq. 37, L2 = |K|_2^2 (largest eigenvalue of
    K^T K) and the dual step sigma = 1 / (tau |K|^2) of §VI (times sigma_scale).

    variables="terminal" sets the same problem up in the variable q of
    p = E^T q, E = e^{TA} (the costate carried to the terminal time).  Every
    term of Eq. 18 keeps its form: K_i p = K'_i q with K'_i = (-e^{t_i A} B Q)^T,
    p^T M p = q^T W q (M' = W, V' = W^-1), <z0, p> = <E z0, q>.  The objective
    values P and D and the gap are unchanged; the primal-dual iteration of
    Eq. 15 run in q is a different (preconditioned) iteration with the same
    solution p* = E^T q*.  E is returned (identity for variables="initial"),
    and value() maps x and p in and out."""
    n = sysd["A"].shape[0]
    _, w = nodes(T, N, rule)
    if variables == "initial":
        K = node_matrices(sysd, T, N, rule)
        M, V = terminal_matrices(sysd, T)
        E = np.eye(n)
    elif variables == "terminal":
        K = node_matrices_terminal(sysd, T, N, rule)
        W = sysd["W"]
        M = 0.5 * (W + W.T)
        V = np.linalg.inv(M)
        V = 0.5 * (V + V.T)
        E = expm(T * sysd["A"])
    else:
        raise ValueError("variables must be 'initial' or 'terminal'")
    Kf = K.reshape(-1, n)
    L2 = float(np.linalg.eigvalsh(Kf.T @ Kf)[-1])
    S = np.linalg.inv(np.eye(n) + 0.5 * tau * M)
    return dict(K=K, w=w, M=M, V=V, S=S, L2=L2, tau=float(tau),
                sigma=float(sigma_scale) / (float(tau) * L2),
                kind=sysd["ctrl_kind"], T=float(T), E=E, variables=variables)


def _batched(prob_list):
    """Stack per-point problems (same n, m) along a leading point axis.  Node
    counts that differ (the fixed-step rule) are padded with zero rows of K
    and zero weights: such a node adds 0 to every sum, its dual variable is
    held at 0 by the projection onto 0 U, and |K| is unchanged."""
    Nmax = max(p["K"].shape[0] for p in prob_list)

    def pad(p, k):
        a = p[k]
        if k not in ("K", "w") or a.shape[0] == Nmax:
            return a
        return np.concatenate([a, np.zeros((Nmax - a.shape[0],) + a.shape[1:])])
    keys = ("K", "w", "M", "V", "S")
    out = {k: np.stack([pad(p, k) for p in prob_list]) for k in keys}
    out["sigma"] = np.array([p["sigma"] for p in prob_list])
    out["tau"] = prob_list[0]["tau"]
    out["kind"] = prob_list[0]["kind"]
    return out


def _as_batch(prob, P):
    """View a shared problem as a batch of P identical problems (broadcast only)."""
    if np.ndim(prob["sigma"]) == 1:
        return prob
    out = dict(prob)
    for k in ("K", "w", "M", "V", "S"):
        out[k] = prob[k][None]
    out["sigma"] = np.full(P, prob["sigma"])
    return out


# ----------------------------------------------------------------- objectives
def _Kp(K, p):
    """K_i p for every node: (B?, N, m, n) x (P, n) -> (P, N, m)."""
    return np.einsum("...imn,...n->...im", K, p)


def _KTy(K, y):
    """sum_i K_i^T y_i: (B?, N, m, n) x (P, N, m) -> (P, n)."""
    return np.einsum("...imn,...im->...n", K, y)


def primal_objective(prob, x0, p):
    """Objective of Eq. 18 with J_z* of Eq. 35:
    P(p) = p^T M p / 4 + 1 - <x0, p> + sum_i w_i |K_i p|_*."""
    quad = 0.25 * np.einsum("...i,...ij,...j->...", p, prob["M"], p)
    H = np.sum(prob["w"] * dual_norm(prob["kind"], _Kp(prob["K"], p)), axis=-1)
    return quad + 1.0 - np.sum(x0 * p, axis=-1) + H


def dual_objective(prob, x0, y):
    """Fenchel dual of min_p G(p) + F(Kp) (G of Eq. 36, F of Eq. 21):
    D(y) = -G*(-K^T y) - F*(y) = 1 - (x0 - K^T y)^T V (x0 - K^T y)
    for y_i in w_i U (F* of Eq. 22); -inf outside, never reached here because
    every iterate y is a projection."""
    r = x0 - _KTy(prob["K"], y)
    return 1.0 - np.einsum("...i,...ij,...j->...", r, prob["V"], r)


def relative_gap(Pv, Dv):
    """(P - D) / max(1, |P|, |D|): the certified relative duality gap."""
    return (Pv - Dv) / np.maximum(1.0, np.maximum(np.abs(Pv), np.abs(Dv)))


# ---------------------------------------------------------------------- PDHG
ADAPT_ALPHA0, ADAPT_ETA, ADAPT_DELTA = 0.5, 0.95, 1.5


def pdhg(prob, x0, tol=1e-8, max_iter=200000, p0=None, y0=None, stop=None, accel=False, adaptive=False):
    """Chambolle-Pock iteration of Eq. 15 for every point in x0 (P, n).

      y <- prox_{sigma F*}(y + sigma K pbar)   (Eq. 23: projection onto w_i U per node)
      p <- prox_{tau G}(p - tau K^T y)          (Eq. 37: S (p - tau K^T y + tau x0))
      pbar <- p + theta (p - p_old), theta = 1  (§VI)

    Initial point of §VI: p0 = pbar0 = x0, y0 = K p0 (unless given).
    A point stops at the first iteration whose relative gap is <= tol, or whose
    ``stop(P, D)`` predicate holds; its iterate is then frozen.

    accel=True is the variant for a strongly convex G that §III mentions
    (Chambolle and Pock 2011, Algorithm 2): G of Eq. 36 has Hessian M/2, so it
    is gamma-strongly convex with gamma = lambda_min(M)/2; after each step
    theta = 1/sqrt(1 + 2 gamma tau), tau <- theta tau, sigma <- sigma/theta and
    pbar = p_new + theta (p_new - p).  The prox of G is then (I + tau M/2)^-1
    at the current tau, evaluated by a fresh linear solve.

    adaptive=True balances the two residuals that §III.B uses as its
    stopping rule (after Goldstein et al., the adaptive PDHG cited there),
      r_p = (p^k - p^{k-1})/tau - K^T (y^k - y^{k-1}),
      r_d = (y^k - y^{k-1})/sigma - K (p^k - p^{k-1}):
    after a step, if |r_p| > Delta |r_d| then tau <- tau/(1 - a),
    sigma <- sigma (1 - a), a <- eta a; if |r_p| < |r_d|/Delta the reverse;
    tau sigma stays 1/|K|^2 (a0 = 0.5, eta = 0.95, Delta = 1.5; no
    backtracking).  theta stays 1; the prox of G is taken at the current tau.
    Returns dict(phi=-P, p, y, P, D, gap, iters, status)."""
    x0 = np.atleast_2d(np.asarray(x0, dtype=np.float64))
    P_, n = x0.shape
    pb = _as_batch(prob, P_)
    K, w, S, sigma, tau = pb["K"], pb["w"], pb["S"], pb["sigma"], pb["tau"]
    kind = pb["kind"]
    shared = K.shape[0] == 1 and P_ > 1
    p = x0.copy() if p0 is None else np.array(p0, dtype=np.float64)
    y = _Kp(K, p) if y0 is None else np.array(y0, dtype=np.float64)
    pbar = p.copy()
    iters = np.zeros(P_, dtype=np.int64)
    status = np.full(P_, MAXITER, dtype=np.int64)
    Pv = np.full(P_, np.inf)
    Dv = np.full(P_, -np.inf)
    active = np.arange(P_)
    tau_k = np.full(P_, float(tau))
    sig_k = np.array(sigma, dtype=np.float64)
    alpha_k = np.full(P_, ADAPT_ALPHA0)
    eye = np.eye(n)
    if accel:
        Mb = pb["M"] if pb["M"].shape[0] == P_ else np.broadcast_to(pb["M"], (P_,) + pb["M"].shape[1:])
        gamma = 0.5 * np.linalg.eigvalsh(Mb)[:, 0]
        eye = np.eye(n)

    def sub(a, idx):
        return a if shared else a[idx]

    for k in range(1, max_iter + 1):
        if active.size == 0:
            break
        Ka, wa, Sa = sub(K, active), sub(w, active), sub(S, active)
        sa = sig_k[active]
        ta = tau_k[active]
        # dual step: projection of y_i + sigma K_i pbar onto w_i U (Eq. 23)
        v = y[active] + sa[:, None, None] * _Kp(Ka, pbar[active])
        ynew = project_scaled(kind, v, np.broadcast_to(wa, v.shape[:-1]))
        # primal step: prox of G (Eq. 37)
        rhs = p[active] - ta[:, None] * _KTy(Ka, ynew) + ta[:, None] * x0[active]
        if accel or adaptive:
            A_ = eye + 0.5 * ta[:, None, None] * np.broadcast_to(sub(pb["M"], active), (active.size, n, n))
        if accel:
            pnew = np.linalg.solve(A_, rhs[..., None])[..., 0]
            th = 1.0 / np.sqrt(1.0 + 2.0 * gamma[active] * ta)
            tau_k[active] = th * ta
            sig_k[active] = sa / th
            pbar[active] = pnew + th[:, None] * (pnew - p[active])
        elif adaptive:
            pnew = np.linalg.solve(A_, rhs[..., None])[..., 0]
            pbar[active] = 2.0 * pnew - p[active]
            # residuals of §III.B at the step just taken, then the balance
            dp = pnew - p[active]
            dy = ynew - y[active]
            r_p = dp / ta[:, None] - _KTy(Ka, dy)
            r_d = dy / sa[:, None, None] - _Kp(Ka, dp)
            npr = np.linalg.norm(r_p, axis=-1)
            ndr = np.linalg.norm(r_d.reshape(active.size, -1), axis=-1)
            al = alpha_k[active]
            up = npr > ADAPT_DELTA * ndr
            dn = ADAPT_DELTA * npr < ndr
            fac = np.where(up, 1.0 / (1.0 - al), np.where(dn, 1.0 - al, 1.0))
            tau_k[active] = ta * fac
            sig_k[active] = sa / fac
            alpha_k[active] = np.where(up | dn, ADAPT_ETA * al, al)
        else:
            pnew = np.einsum("...ij,...j->...i", Sa, rhs)
            pbar[active] = 2.0 * pnew - p[active]
        p[active] = pnew
        y[active] = ynew
        iters[active] = k
        # duality gap
        pa = {"K": Ka, "w": wa, "M": sub(pb["M"], active), "V": sub(pb["V"], active),
              "kind": kind}
        Pa = primal_objective(pa, x0[active], pnew)
        Da = dual_objective(pa, x0[active], ynew)
        Pv[active], Dv[active] = Pa, Da
        bad = ~(np.isfinite(Pa) & np.isfinite(Da))
        done = relative_gap(Pa, Da) <= tol
        if stop is not None:
            done |= stop(Pa, Da)
        status[active[bad]] = NONFINITE
        status[active[done & ~bad]] = OK
        active = active[~(done | bad)]
    return dict(phi=-Pv, p=p, y=y, P=Pv, D=Dv, gap=relative_gap(Pv, Dv), iters=iters,
                status=status)


def terminal_cost(sysd, x):
    """J_x(x) = x^T W^-1 x - 1 (Eq. 34), row-wise."""
    Wi = np.linalg.inv(sysd["W"])
    return np.einsum("...i,ij,...j->...", x, Wi, x) - 1.0


def solve_in_variables(probs, x, p0=None, **kw):
    """pdhg() for per-point problems probs (a list, one per row of x, or one
    shared problem) in the problems' variables: rows of x and of the warm
    start p0 are mapped to q (x' = E x, q0 = E^-T p0), and the solution back
    to p = E^T q.  The returned dict carries p (original variables) and q."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    shared = isinstance(probs, dict)
    Es = np.broadcast_to(probs["E"], (x.shape[0],) + probs["E"].shape) if shared else \
        np.stack([pr["E"] for pr in probs])
    xq = np.einsum("kij,kj->ki", Es, x)
    q0 = None if p0 is None else np.linalg.solve(np.transpose(Es, (0, 2, 1)),
                                                 np.atleast_2d(np.asarray(p0, dtype=np.float64))[..., None])[..., 0]
    r = pdhg(probs if shared else _batched(probs), xq, p0=q0, **kw)
    r["q"] = r["p"]
    r["p"] = np.einsum("kji,kj->ki", Es, r["q"])
    return r


def value(sysd, x, T, N, rule, tau, tol=1e-8, max_iter=200000, p0=None, sigma_scale=1.0, accel=False,
          variables="initial", adaptive=False):
    """phi_N(x, T): the generalized Hopf formula with the N-node quadrature
    (Eq. 18) for every row of x at one horizon T.  At T = 0 the value is the
    terminal cost itself (Eq. 4 initial condition) and p* = grad J_x.
    variables="terminal" runs the iteration in the variable q (see setup);
    phi, P, D and the gap are the same quantities, p is returned in the
    original variable."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    if T == 0.0:
        Wi = np.linalg.inv(sysd["W"])
        P_ = x.shape[0]
        return dict(phi=terminal_cost(sysd, x), p=2.0 * x @ Wi.T, gap=np.zeros(P_),
                    iters=np.zeros(P_, dtype=np.int64), status=np.zeros(P_, dtype=np.int64),
                    P=-terminal_cost(sysd, x), D=-terminal_cost(sysd, x))
    prob = setup(sysd, T, N, rule, tau, sigma_scale, variables)
    if variables == "initial":
        return pdhg(prob, x, tol=tol, max_iter=max_iter, p0=p0, accel=accel, adaptive=adaptive)
    return solve_in_variables(prob, x, p0=p0, tol=tol, max_iter=max_iter, accel=accel, adaptive=adaptive)


# ---------------------------------------------------------------- time-to-reach
def hamiltonian_x(sysd, p, x0):
    """H_x(p, x0) = -x0^T A^T p + |-Q^T B^T p|_* (§IV); d phi/dT = -H_x(p*, x0)."""
    A, B = sysd["A"], sysd["B"]
    Q = control_scaling(sysd)
    return -np.einsum("...i,...i->...", x0 @ A.T, p) + dual_norm(sysd["ctrl_kind"], p @ B @ Q)


def time_to_reach(sysd, x, t_max, N, rule, tau, tol_T=1e-6, tol_gap=1e-8,
                  sign_floor=1e-13, max_iter=400000, sigma_scale=1.0, variables="initial"):
    """Minimum time T* to reach the target (§IV): the smallest T with
    phi_N(x, T) <= 0, found by bisection on [0, t_max].

    The sign of phi at each midpoint is read from the certified interval
    phi in [-P, -D]: the primal-dual iteration runs until 0 lies outside it or
    the relative gap falls below sign_floor (then phi is taken as zero, i.e.
    reached, and the status records AMBIGUOUS_SIGN).  The bracket [lo, hi]
    shrinks until hi - lo <= tol_T * hi; T* = hi, and p* is the solution at hi
    solved to tol_gap.  Points already inside the target return T* = 0;
    points with phi(t_max) > 0 return UNREACHABLE.  Every point is independent.
    Every inner solve runs in the given variables (see setup).
    Returns dict(T, p, status, steps)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    P_, n = x.shape
    T_out = np.zeros(P_)
    p_out = np.zeros((P_, n))
    st = np.zeros(P_, dtype=np.int64)
    Wi = np.linalg.inv(sysd["W"])

    def sign_solve(idx, Tvals):
        """phi <= 0 ? for the points idx at their own horizons Tvals."""
        probs = [setup(sysd, float(Tv), N, rule, tau, sigma_scale, variables) for Tv in Tvals]
        r = solve_in_variables(probs, x[idx], tol=sign_floor, max_iter=max_iter,
                               stop=lambda Pa, Da: (Pa < 0.0) | (Da > 0.0))
        # phi = -P(p*) lies in [-P, -D]
        reached = r["D"] > 0.0
        amb = ~(reached | (r["P"] < 0.0))
        return reached | amb, amb, r

    inside = terminal_cost(sysd, x) <= 0.0
    T_out[inside] = 0.0
    p_out[inside] = 2.0 * x[inside] @ Wi.T
    todo = np.where(~inside)[0]
    if todo.size:
        reach_max, amb, _ = sign_solve(todo, np.full(todo.size, t_max))
        st[todo[amb]] = AMBIGUOUS_SIGN
        unreach = todo[~reach_max]
        st[unreach] = UNREACHABLE
        T_out[unreach] = np.inf
        todo = todo[reach_max]
    lo = np.zeros(P_)
    hi = np.full(P_, float(t_max))
    steps = 0
    while todo.size:
        steps += 1
        mid = 0.5 * (lo[todo] + hi[todo])
        reached, amb, _ = sign_solve(todo, mid)
        st[todo[amb]] = AMBIGUOUS_SIGN
        hi[todo[reached]] = mid[reached]
        lo[todo[~reached]] = mid[~reached]
        todo = todo[hi[todo] - lo[todo] > tol_T * hi[todo]]
    fin = np.where(~inside & (st != UNREACHABLE))[0]
    if fin.size:
        probs = [setup(sysd, float(hi[i]), N, rule, tau, sigma_scale, variables) for i in fin]
        r = solve_in_variables(probs, x[fin], tol=tol_gap, max_iter=max_iter)
        T_out[fin] = hi[fin]
        p_out[fin] = r["p"]
    return dict(T=T_out, p=p_out, status=st, steps=steps)


def time_to_reach_newton(sysd, x, t_max, N, rule, tau, tol_T=1e-6, tol_gap=1e-10, max_steps=100,
                         max_iter=400000, sigma_scale=1.0, variables="initial"):
    """Minimum time to reach by the hybrid of §IV: Newton steps on phi(x, T)
    using the HJ equation for the derivative, t_{k+1} = t_k + phi / H_x(p*, x0)
    (Eq. 26 with H_x of §IV), safeguarded by the bracket [lo, hi] that the
    certified signs of phi maintain; a step that leaves the bracket is replaced
    by its midpoint.  Every candidate is solved to tol_gap.  Stops when a step
    is below tol_T * t, the bracket is below tol_T * hi, or the certified
    interval [-P, -D] contains 0 (|phi| below the gap).  Starts at t_max.
    Returns dict(T, p, status, steps)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    P_, n = x.shape
    Wi = np.linalg.inv(sysd["W"])
    T_out = np.zeros(P_)
    p_out = np.zeros((P_, n))
    st = np.zeros(P_, dtype=np.int64)

    def solve(idx, Tvals):
        probs = [setup(sysd, float(Tv), N, rule, tau, sigma_scale, variables) for Tv in Tvals]
        return solve_in_variables(probs, x[idx], tol=tol_gap, max_iter=max_iter)

    inside = terminal_cost(sysd, x) <= 0.0
    p_out[inside] = 2.0 * x[inside] @ Wi.T
    todo = np.where(~inside)[0]
    lo = np.zeros(P_)
    hi = np.full(P_, float(t_max))
    t = np.full(P_, float(t_max))
    steps = 0
    first = True
    while todo.size and steps < max_steps:
        steps += 1
        r = solve(todo, t[todo])
        Pv, Dv = r["P"], r["D"]
        above = Pv < 0.0                  # phi >= -P > 0: not reached by t
        below = Dv > 0.0                  # phi <= -D < 0: reached
        if first:
            unreach = todo[above]
            st[unreach] = UNREACHABLE
            T_out[unreach] = np.inf
            first = False
        p_out[todo] = r["p"]
        T_out[todo] = t[todo]
        lo[todo[above]] = t[todo[above]]
        hi[todo[below]] = t[todo[below]]
        # Newton step with the HJ derivative d phi / dT = -H_x(p*, x0)
        H = hamiltonian_x(sysd, r["p"], x[todo])
        phi = -Pv
        with np.errstate(divide="ignore", invalid="ignore"):
            tn = t[todo] + phi / H
        bad = ~np.isfinite(tn) | (tn <= lo[todo]) | (tn >= hi[todo])
        tn = np.where(bad, 0.5 * (lo[todo] + hi[todo]), tn)
        done = (~(above | below)) | (np.abs(tn - t[todo]) <= tol_T * tn) | \
            (hi[todo] - lo[todo] <= tol_T * hi[todo])
        if steps == 1:
            done |= above                 # unreachable
        t[todo] = np.where(done, t[todo], tn)
        todo = todo[~done]
    return dict(T=T_out, p=p_out, status=st, steps=steps)


# ------------------------------------------------------------------ trajectory
def optimal_control(sysd, p, s):
    """u*(s) = Q argmax_{c in U} <c, -Q^T B^T e^{-s A^T} p>  (Eq. 27), the control
    applied at physical time s in [0, T] (Hopf time t = T - s).  p (n,), s scalar."""
    A, B = sysd["A"], sysd["B"]
    Q = control_scaling(sysd)
    g = -(Q.T @ B.T @ expm(-s * A.T) @ p)
    return Q @ argmax_unit(sysd["ctrl_kind"], g)


def trajectory_from_dual(sysd, x0, prob, y):
    """Trajectory at the left-Riemann nodes from the discrete dual solution:
    y_i = w_i u_i with u_i in U (the prox of Eq. 23 keeps y_i in w_i U), so the
    node controls are u_i = Q y_i / w_i.  Sorted by physical time s_i = T - t_i
    (ascending), z after node i adds w_i e^{-s_i A} B u_i.  This is the
    trajectory of Eq. 33 with the subgradient of H_z chosen by the dual, which
    is exact even at nodes where K_i p* = 0 and the argmax of Eq. 27 is not
    unique.  Returns (s (N+1,), x (N+1, n)) with s_0 = 0, x_0 = x0."""
    A, B = sysd["A"], sysd["B"]
    Q = control_scaling(sysd)
    T = prob["T"]
    N = prob["w"].shape[0]
    t, w = nodes(T, N, LEFT_RIEMANN)
    order = np.argsort(T - t)
    z = np.asarray(x0, dtype=np.float64).copy()
    ss = [0.0]
    xs = [z.copy()]
    for i in order:
        s = T - t[i]
        z = z + w[i] * (expm(-s * A) @ B @ (Q @ (y[i] / w[i])))
        ss.append(s)
        xs.append(expm(s * A) @ z)
    return np.array(ss), np.array(xs)


def trajectory(sysd, x0, T, p, S):
    """Optimal trajectory from p* (§V, Eq. 33) on S uniform steps of [0, T].

    Physical sample times s_j = j T/S, j = 0..S.  The control on (s_{j-1}, s_j]
    is u_j = u*(s_j) of Eq. 27; in the variable z = e^{-sA} x (Eq. 9) the state
    is the sum z_j = x0 + sum_{k=1..j} (T/S) e^{-s_k A} B u_k (Eq. 10 integrated
    with the right-endpoint rule, which is the left Riemann rule of Eq. 17 read
    in Hopf time), and x_j = e^{s_j A} z_j.  When S equals the number of
    left-Riemann nodes, z_S is the minimiser of Eq. 29, (1/2) V^-1 p*.
    Returns (x_traj (S+1, n), u_traj (S+1, m))."""
    A, B = sysd["A"], sysd["B"]
    x0 = np.asarray(x0, dtype=np.float64)
    n, m = B.shape
    h = T / S
    xs = np.empty((S + 1, n))
    us = np.empty((S + 1, m))
    z = x0.copy()
    xs[0] = x0
    us[0] = optimal_control(sysd, p, 0.0)
    for j in range(1, S + 1):
        s = j * h
        u = optimal_control(sysd, p, s)
        z = z + h * (expm(-s * A) @ B @ u)
        xs[j] = expm(s * A) @ z
        us[j] = u
    return xs, us
