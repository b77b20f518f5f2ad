"""Python binding of the C ABI (argument marshalling only).

Per-point arrays may be CUDA torch tensors (device pointers, asynchronous on
the current torch stream) or numpy arrays (host buffers: the library copies
them in and out inside the call).  Problem matrices are numpy float64 arrays.
"""
import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib

BALL, BOX = 0, 1
LEFT_RIEMANN, TRAPEZOID, SIMPSON, LEFT_FIXED = 0, 1, 2, 3
FP64, FP32 = 0, 1
VARS_INITIAL, VARS_TERMINAL = 0, 1
STATUS = {0: "ok", 1: "max_iter", 2: "nonfinite", 3: "unreachable", 4: "ambiguous_sign"}


class HopfError(RuntimeError):
    pass


def _check(lib, rc):
    if rc != 0:
        raise HopfError(f"{lib.hopf_status_string(rc).decode()} ({rc}): {lib.hopf_last_error().decode()}")


class System:
    """xdot = A x + B u, control set (ball of `radius` or box of `half_widths`),
    target {x : x^T W^-1 x <= 1}.  Accepts the dicts of inputs.workloads."""

    def __init__(self, A, B, W, ctrl_kind=BALL, radius=1.0, half_widths=None):
        self.A = np.ascontiguousarray(A, dtype=np.float64)
        self.B = np.ascontiguousarray(B, dtype=np.float64)
        self.W = np.ascontiguousarray(W, dtype=np.float64)
        self.n, self.m = self.B.shape
        self.ctrl_kind = int(ctrl_kind)
        self.radius = float(radius)
        hw = np.ones(self.m) if half_widths is None else half_widths
        self.half_widths = np.ascontiguousarray(hw, dtype=np.float64)

    @classmethod
    def from_dict(cls, d):
        return cls(d["A"], d["B"], d["W"], d["ctrl_kind"], d.get("radius", 1.0), d.get("half_widths"))

    def c_struct(self):
        dp = lambda a: a.ctypes.data_as(_lib.P_double)  # noqa: E731
        return _lib.HopfProblem(self.n, self.m, dp(self.A), dp(self.B), self.ctrl_kind, self.radius,
                                dp(self.half_widths), dp(self.W))


@dataclass
class Options:
    rule: int = LEFT_RIEMANN
    N: int = 100
    max_iter: int = 100000
    gap_every: int = 8
    precision: int = FP32
    tau: float = 1.0
    sigma_scale: float = 1.0
    tol_gap: float = 1e-5
    t_max: float = 10.0
    tol_T: float = 1e-5
    profile: bool = False
    accel: bool = False
    park_iters: int = 0
    newton: bool = False
    kernel: int = 0          # 0 auto, 1 force one warp per point
    variables: int = VARS_INITIAL   # VARS_TERMINAL: iterate in q, p = e^{T A^T} q
    max_steps: int = 0       # time-to-reach: cap on candidate horizons per point (0 = 256)
    adaptive: bool = False   # residual-balanced step sizes (general kernel)

    def c_struct(self, host_io):
        return _lib.HopfOpts(self.rule, self.N, self.max_iter, self.gap_every, self.precision, int(host_io),
                             self.tau, self.sigma_scale, self.tol_gap, self.t_max, self.tol_T,
                             int(self.profile), int(self.accel), int(self.park_iters),
                             int(self.newton), int(self.kernel), int(self.variables), int(self.max_steps),
                             int(self.adaptive))


def _is_torch(a):
    return type(a).__module__.startswith("torch")


class _Marshal:
    """Puts every per-point array on one side (device tensors or host numpy)."""

    def __init__(self, precision, like):
        self.device = _is_torch(like)
        self.np_dtype = np.float64 if precision == FP64 else np.float32
        if self.device:
            import torch
            self.torch = torch
            self.t_dtype = torch.float64 if precision == FP64 else torch.float32
            self.dev = like.device

    def inp(self, a):
        if a is None:
            return None
        if self.device:
            t = a if _is_torch(a) else self.torch.as_tensor(np.asarray(a))
            return t.to(device=self.dev, dtype=self.t_dtype).contiguous()
        return np.ascontiguousarray(np.asarray(a), dtype=self.np_dtype)

    def out(self, shape, integer=False):
        if self.device:
            dt = self.torch.int32 if integer else self.t_dtype
            return self.torch.empty(shape, dtype=dt, device=self.dev)
        return np.empty(shape, dtype=np.int32 if integer else self.np_dtype)

    @staticmethod
    def ptr(a):
        if a is None:
            return None
        if _is_torch(a):
            return ctypes.c_void_p(a.data_ptr())
        return a.ctypes.data_as(ctypes.c_void_p)

    def stream(self, stream):
        if not self.device:
            return None
        s = stream if stream is not None else self.torch.cuda.current_stream(self.dev)
        return ctypes.c_void_p(s.cuda_stream)


def value(system, x, t, opts=None, p_init=None, stream=None):
    """phi(x, t) of the generalized Hopf formula (Eq. 18) for every row of x.
    t is a scalar (one horizon for all points) or an array with one per point.
    Returns dict(phi, p, gap, iters, status)."""
    lib = _lib.load()
    opts = opts or Options()
    mar = _Marshal(opts.precision, x)
    xx = mar.inp(x)
    P = int(xx.shape[0])
    scalar_t = np.ndim(t) == 0 and not (_is_torch(t) and t.ndim > 0)
    tt = mar.inp(np.array([float(t)]) if scalar_t else t)
    pi = mar.inp(p_init)
    out = dict(phi=mar.out((P,)), p=mar.out((P, system.n)), gap=mar.out((P,)),
               iters=mar.out((P,), True), status=mar.out((P,), True))
    prob = system.c_struct()
    o = opts.c_struct(not mar.device)
    rc = lib.hopf_value(ctypes.byref(prob), ctypes.byref(o), P, mar.ptr(xx), mar.ptr(tt), 0 if scalar_t else 1,
                        mar.ptr(pi), mar.ptr(out["phi"]), mar.ptr(out["p"]), mar.ptr(out["gap"]),
                        mar.ptr(out["iters"]), mar.ptr(out["status"]), mar.stream(stream))
    _check(lib, rc)
    return out


def value_stacked(base, W_blocks, x, t, opts=None, p_init=None, stream=None):
    """phi for k copies of the base System sharing one control (§VI.B-C):
    stacked state x = (chi_1, ..., chi_k) per row, target blockdiag(W_blocks)
    (W_blocks: (k, n_b, n_b)); base.W is not used.  Device (torch) arrays
    only.  Returns dict(phi, p, gap, iters, status)."""
    lib = _lib.load()
    opts = opts or Options()
    if not _is_torch(x):
        raise TypeError("value_stacked takes device (torch) arrays")
    Wb = np.ascontiguousarray(W_blocks, dtype=np.float64)
    k = int(Wb.shape[0])
    mar = _Marshal(opts.precision, x)
    xx = mar.inp(x)
    P = int(xx.shape[0])
    scalar_t = np.ndim(t) == 0 and not (_is_torch(t) and t.ndim > 0)
    tt = mar.inp(np.array([float(t)]) if scalar_t else t)
    pi = mar.inp(p_init)
    out = dict(phi=mar.out((P,)), p=mar.out((P, k * base.n)), gap=mar.out((P,)),
               iters=mar.out((P,), True), status=mar.out((P,), True))
    sp = _lib.HopfStacked(base.c_struct(), k, Wb.ctypes.data_as(_lib.P_double))
    o = opts.c_struct(False)
    rc = lib.hopf_value_stacked(ctypes.byref(sp), ctypes.byref(o), P, mar.ptr(xx), mar.ptr(tt),
                                0 if scalar_t else 1, mar.ptr(pi), mar.ptr(out["phi"]), mar.ptr(out["p"]),
                                mar.ptr(out["gap"]), mar.ptr(out["iters"]), mar.ptr(out["status"]),
                                mar.stream(stream))
    _check(lib, rc)
    return out


def time_to_reach(system, x, opts=None, T_lo=None, T_hi=None, p_init=None, stream=None):
    """Minimum time to reach the target (§IV) by certified bisection on
    [0, opts.t_max] (or on [T_lo, T_hi] when given).  Returns dict(T, p, gap,
    status, steps)."""
    lib = _lib.load()
    opts = opts or Options()
    mar = _Marshal(opts.precision, x)
    xx = mar.inp(x)
    P = int(xx.shape[0])
    lo, hi, pi = mar.inp(T_lo), mar.inp(T_hi), mar.inp(p_init)
    out = dict(T=mar.out((P,)), p=mar.out((P, system.n)), gap=mar.out((P,)), status=mar.out((P,), True))
    steps = ctypes.c_int(0)
    prob = system.c_struct()
    o = opts.c_struct(not mar.device)
    rc = lib.hopf_time_to_reach(ctypes.byref(prob), ctypes.byref(o), P, mar.ptr(xx), mar.ptr(lo), mar.ptr(hi),
                                mar.ptr(pi), mar.ptr(out["T"]), mar.ptr(out["p"]), mar.ptr(out["gap"]),
                                mar.ptr(out["status"]), ctypes.byref(steps), mar.stream(stream))
    _check(lib, rc)
    out["steps"] = steps.value
    return out


def node_table(system, T, opts=None, device=None):
    """The float64 node table the solves build for horizon T (§III.A, Eq. 20):
    K (N, m, n) and weights w (N,), in opts.variables.  Host numpy arrays, or
    float64 torch tensors on `device` when given."""
    lib = _lib.load()
    opts = opts or Options()
    N, m, n = opts.N, system.m, system.n
    if device is not None:
        import torch
        K = torch.empty((N, m, n), dtype=torch.float64, device=device)
        w = torch.empty((N,), dtype=torch.float64, device=device)
        s = ctypes.c_void_p(torch.cuda.current_stream(K.device).cuda_stream)
    else:
        K, w, s = np.empty((N, m, n)), np.empty(N), None
    prob = system.c_struct()
    o = opts.c_struct(device is None)
    ptr = _Marshal.ptr
    _check(lib, lib.hopf_node_table(ctypes.byref(prob), ctypes.byref(o), float(T), ptr(K), ptr(w), s))
    return K, w


def last_profile():
    """(ms_tables, ms_solve) of the last hopf_value call made with profile=True."""
    lib = _lib.load()
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib, lib.hopf_last_profile(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def trajectory(system, x, T, p_star, S, opts=None, stream=None):
    """Optimal control and state on S uniform steps of [0, T] from p* (Eq. 27,
    Eq. 33).  Returns dict(x (P, S+1, n), u (P, S+1, m))."""
    lib = _lib.load()
    opts = opts or Options()
    mar = _Marshal(opts.precision, x)
    xx, TT, pp = mar.inp(x), mar.inp(T), mar.inp(p_star)
    P = int(xx.shape[0])
    out = dict(x=mar.out((P, S + 1, system.n)), u=mar.out((P, S + 1, system.m)))
    prob = system.c_struct()
    o = opts.c_struct(not mar.device)
    rc = lib.hopf_trajectory(ctypes.byref(prob), ctypes.byref(o), P, mar.ptr(xx), mar.ptr(TT), mar.ptr(pp), S,
                             mar.ptr(out["x"]), mar.ptr(out["u"]), mar.stream(stream))
    _check(lib, rc)
    return out
