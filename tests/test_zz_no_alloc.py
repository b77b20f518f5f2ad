"""hopf_value_noalloc: the value solve for callers that cannot allocate.

Real-time control loops and processes with a fixed memory footprint cannot
call cudaMalloc at solve time; this entry
point takes its scratch from a static device array instead.  The test calls it
through the C ABI twice in a row (the array keeps the first call's contents)
and checks each result against hopf_value within the value tolerance of the
other parity tests (1e-5 relative).  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from inputs import workloads as wl

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(H, sysd, opts, x, t_host):
    """One call through the C ABI; t_host is a scalar (one horizon, t_stride 0)
    or an array with one horizon per point (t_stride 1)."""
    import torch
    lib = H._lib.load()
    P, n = x.shape
    per_point = np.ndim(t_host) > 0
    t = torch.tensor(np.atleast_1d(t_host), dtype=x.dtype, device="cuda")
    out = dict(phi=torch.empty(P, dtype=x.dtype, device="cuda"),
               p=torch.empty(P, n, dtype=x.dtype, device="cuda"),
               gap=torch.empty(P, dtype=x.dtype, device="cuda"),
               iters=torch.empty(P, dtype=torch.int32, device="cuda"),
               status=torch.empty(P, dtype=torch.int32, device="cuda"))
    prob = sysd.c_struct()
    o = opts.c_struct(False)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.hopf_value_noalloc(ctypes.byref(prob), ctypes.byref(o), P, _ptr(x), _ptr(t), 1 if per_point else 0,
                                None, _ptr(out["phi"]), _ptr(out["p"]), _ptr(out["gap"]), _ptr(out["iters"]),
                                _ptr(out["status"]), stream)
    return rc, out, t


CASES = [("fp32", "ball", False), ("fp32", "ball", True), ("fp64", "ball", False), ("fp64", "ball", True),
         ("fp32", "box", False), ("fp64", "box", True)]


@pytest.mark.parametrize("prec,ctrl,per_point", CASES)
def test_noalloc_matches_value_twice(prec, ctrl, per_point):
    # float32 and float64, one shared horizon and one per point (the largest
    # use of the table scratch), ball control (random n = 10 system) and box
    # control (two-mass chain, n = 4, m = 1); two calls in a row, each
    # compared with hopf_value at the tolerance of the other parity tests
    import torch
    import paper_1712_08226_gb300 as H
    from paper_1712_08226_gb300 import build
    build.build()
    fp64 = prec == "fp64"
    dt = torch.float64 if fp64 else torch.float32
    if ctrl == "ball":
        w = wl.workload_random10(1000)
        sysd_d, xs, T, N, tau = w["system"], w["x"], w["t"], w["N"], w["tau"]
    else:
        sysd_d = wl.spring_chain(masses=2, actuators=1, radius_target=0.5)
        xs, T, N, tau = wl.normal_points(31, 1000, 4, 1.0), 1.7, 64, 0.5
    sysd = H.System.from_dict(sysd_d)
    tol = 1e-9 if fp64 else 1e-5
    opts = H.Options(N=N, tau=tau, tol_gap=tol, precision=H.FP64 if fp64 else H.FP32, max_iter=400000)
    n_pts = 200 if (fp64 or per_point) else 600
    for k, lo in enumerate((0, 1000 - n_pts)):        # two calls in a row, overlapping points
        x = torch.tensor(xs[lo:lo + n_pts], dtype=dt, device="cuda")
        t_host = np.full(n_pts, T) if per_point else T
        rc, got, t_dev = _noalloc(H, sysd, opts, x, t_host)
        assert rc == 0, (k, rc)
        ref = H.value(sysd, x, t_dev if per_point else T, opts)
        torch.cuda.synchronize()
        assert np.all(got["status"].cpu().numpy() == 0)
        a = got["phi"].cpu().numpy().astype(np.float64)
        b = ref["phi"].cpu().numpy().astype(np.float64)
        err = np.abs(a - b) / np.maximum(1.0, np.abs(b))
        assert err.max() <= (2 * tol if fp64 else tol), (k, err.max())


def test_noalloc_rejects_what_does_not_fit():
    import torch
    import paper_1712_08226_gb300 as H
    w = wl.workload_random10(20000)                 # 20000 x 256 x 2 floats > 32 MiB
    sysd = H.System.from_dict(w["system"])
    x = torch.tensor(w["x"], dtype=torch.float32, device="cuda")
    rc, _, _ = _noalloc(H, sysd, H.Options(N=w["N"], tau=w["tau"]), x, w["t"])
    assert rc == -6
    # the allocation-free path runs the paper's variable only
    rc, _, _ = _noalloc(H, sysd, H.Options(N=w["N"], tau=w["tau"], variables=1), x[:10].contiguous(), w["t"])
    assert rc == -1
