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


def _noalloc(H, sysd, opts, x, t_scalar):
    import torch
    lib = H._lib.load()
    P, n = x.shape
    t = torch.tensor([t_scalar], dtype=x.dtype, device="cuda")
    out = dict(phi=torch.empty(P, dtype=x.dtype, device="cuda"),
               p=torch.empty(P, n, dtype=x.dtype, device="cuda"),
               gap=torch.empty(P, dtype=x.dtype, device="cuda"),
               iters=torch.empty(P, dtype=torch.int32, device="cuda"),
               status=torch.empty(P, dtype=torch.int32, device="cuda"))
    prob = sysd.c_struct()
    o = opts.c_struct(False)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.hopf_value_noalloc(ctypes.byref(prob), ctypes.byref(o), P, _ptr(x), _ptr(t), 0, None,
                                _ptr(out["phi"]), _ptr(out["p"]), _ptr(out["gap"]), _ptr(out["iters"]),
                                _ptr(out["status"]), stream)
    return rc, out


def test_noalloc_matches_value_twice():
    import torch
    import paper_1712_08226_gb300 as H
    from paper_1712_08226_gb300 import build
    build.build()
    w = wl.workload_random10(1000)
    sysd = H.System.from_dict(w["system"])
    opts = H.Options(N=w["N"], tau=w["tau"], tol_gap=1e-5)
    for k, sl in enumerate((slice(0, 600), slice(400, 1000))):     # two calls in a row
        x = torch.tensor(w["x"][sl], dtype=torch.float32, device="cuda")
        rc, got = _noalloc(H, sysd, opts, x, w["t"])
        assert rc == 0, (k, rc)
        ref = H.value(sysd, x, w["t"], opts)
        torch.cuda.synchronize()
        assert np.all(got["status"].cpu().numpy() == 0)
        a = got["phi"].cpu().numpy().astype(np.float64)
        b = ref["phi"].cpu().numpy().astype(np.float64)
        err = np.abs(a - b) / np.maximum(1.0, np.abs(b))
        assert err.max() <= 1e-5, (k, err.max())


def test_noalloc_rejects_what_does_not_fit():
    import torch
    import paper_1712_08226_gb300 as H
    w = wl.workload_random10(20000)                 # 20000 x 256 x 2 floats > 32 MiB
    sysd = H.System.from_dict(w["system"])
    x = torch.tensor(w["x"], dtype=torch.float32, device="cuda")
    rc, _ = _noalloc(H, sysd, H.Options(N=w["N"], tau=w["tau"]), x, w["t"])
    assert rc == -6
