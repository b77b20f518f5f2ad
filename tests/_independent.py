"""Independent FP64 references used to pin the oracle.

None of this calls the oracle.  It solves the *primal control* form of the
discretised problem,

    phi_N(x0, T) = min over u_i in U of  J_x( e^{TA} x0 + sum_i w_i e^{t_i A} B u_i ),

which equals the Hopf value of Eq. 18 by Fenchel-Rockafellar duality (the
PDHG oracle solves the dual form).  Two methods: accelerated projected
gradient (FISTA, Beck and Teboulle 2009) for any size, and exhaustive
active-set enumeration for scalar box controls on very few nodes.
"""
import itertools

import numpy as np
from scipy.linalg import expm


def quad_nodes(T, N, trapezoid):
    if trapezoid:
        h = T / (N - 1)
        t = h * np.arange(N)
        w = np.full(N, h)
        w[[0, -1]] *= 0.5
    else:
        t = (T / N) * np.arange(N)
        w = np.full(N, T / N)
    return t, w


def fixed_step_nodes(T, dt):
    """Left ends of the partition 0, dt, 2 dt, ... of [0, T], the last piece
    running to T: nodes t_k = k dt while k dt < T, widths dt and T - t_last."""
    t = []
    k = 0
    while k * dt < T:
        t.append(k * dt)
        k += 1
    w = [dt] * len(t)
    w[-1] = T - t[-1]
    return np.array(t), np.array(w)


def control_form(A, B, T, N, trapezoid, tw=None):
    """c = e^{TA} x0 map and G = [w_i e^{t_i A} B]_i (n x N m); tw = (t, w)
    gives the nodes explicitly."""
    t, w = quad_nodes(T, N, trapezoid) if tw is None else tw
    G = np.concatenate([w[i] * expm(t[i] * A) @ B for i in range(len(t))], axis=1)
    return expm(T * A), G


def _project(u, kind, m, bounds):
    U = u.reshape(-1, m)
    if kind == "ball":
        nr = np.linalg.norm(U, axis=1, keepdims=True)
        U = U * np.minimum(1.0, bounds / np.maximum(nr, 1e-300))
    else:
        U = np.clip(U, -bounds, bounds)
    return U.ravel()


def fista_value(A, B, W, x0, T, N, kind, bound=1.0, trapezoid=False, iters=200000, tol=1e-15, tw=None):
    """min over u_i in U of (e^{TA}x0 + G u)^T W^-1 (...) - 1 by FISTA with
    projection onto the product of control sets (ball radius `bound`, or box
    half-widths `bound` given as scalar or (m,) array)."""
    m = B.shape[1]
    E, G = control_form(A, B, T, N, trapezoid, tw)
    Wi = np.linalg.inv(W)
    c = E @ x0
    H = G.T @ Wi @ G
    L = 2.0 * np.linalg.eigvalsh(H)[-1]
    bounds = np.broadcast_to(np.asarray(bound, dtype=np.float64), (m,))
    if kind == "ball":
        bounds = float(bound)
    u = np.zeros(G.shape[1])
    v = u.copy()
    tk = 1.0
    f_old = np.inf
    for _ in range(iters):
        r = c + G @ v
        g = 2.0 * G.T @ (Wi @ r)
        un = _project(v - g / L, kind, m, bounds)
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * tk * tk))
        v = un + ((tk - 1.0) / tn) * (un - u)
        u, tk = un, tn
        rr = c + G @ u
        f = rr @ Wi @ rr - 1.0
        if abs(f_old - f) < tol * max(1.0, abs(f)):
            break
        f_old = f
    rr = c + G @ u
    return rr @ Wi @ rr - 1.0, u


def brute_force_value(A, B, W, x0, T, N, trapezoid=False):
    """Exact minimum for a scalar control |u_i| <= 1 on N (<= 8) nodes: every
    node is at -1, at +1, or free; the free block is an unconstrained
    least-squares problem; keep the best pattern whose free part is feasible."""
    assert B.shape[1] == 1 and N <= 8
    E, G = control_form(A, B, T, N, trapezoid)
    Wi = np.linalg.inv(W)
    R = np.linalg.cholesky(Wi).T          # Wi = R^T R
    c = E @ x0
    best = np.inf
    for pat in itertools.product((-1, 0, 1), repeat=N):
        pat = np.array(pat)
        fixed = pat != 0
        r0 = c + G[:, fixed] @ pat[fixed].astype(float)
        if (~fixed).any():
            Gf = G[:, ~fixed]
            uf, *_ = np.linalg.lstsq(R @ Gf, -(R @ r0), rcond=None)
            if np.any(np.abs(uf) > 1.0 + 1e-12):
                continue
            r = r0 + Gf @ uf
        else:
            r = r0
        best = min(best, r @ Wi @ r - 1.0)
    return best


def di_min_time_to_origin(x):
    """Bang-bang minimum time to the origin for xdot1 = x2, xdot2 = u, |u| <= 1
    (classical switching-curve result)."""
    x1, x2 = x
    s = x1 + 0.5 * x2 * abs(x2)
    if s > 0:
        return x2 + 2.0 * np.sqrt(x1 + 0.5 * x2 * x2)
    if s < 0:
        return -x2 + 2.0 * np.sqrt(-x1 + 0.5 * x2 * x2)
    return abs(x2)
