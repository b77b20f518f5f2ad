"""Residual-balanced adaptive step sizes (the §III.B residuals, Goldstein et
al.'s adaptive PDHG) on the general kernel against the FP64 oracle: values
to the usual tolerances, and in float64 the same step-size schedule (the
iteration count of the oracle's adaptive run, checked every iteration)."""
import json
import os

import numpy as np
import pytest

from inputs import workloads as wl

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1712_08226_gb300 as H
    from paper_1712_08226_gb300 import build
    build.build()
    H._lib.load()
    return H


def cuda(a, dtype=None):
    import torch
    return torch.as_tensor(np.asarray(a), dtype=dtype or torch.float32, device="cuda")


def np_(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel_err(a, b):
    return np.abs(a - b) / np.maximum(1.0, np.abs(b))


@pytest.mark.parametrize("variables", [0, 1])
def test_adaptive_fp32_random10_against_oracle(H, variables):
    g = gold("random10_values.json")
    P = 96
    w = wl.workload_random10(P)
    sysd = H.System.from_dict(w["system"])
    r = H.value(sysd, cuda(w["x"]), w["t"], H.Options(N=w["N"], tau=w["tau"], adaptive=True, variables=variables))
    assert np.all(r["status"].cpu().numpy() == 0)
    assert rel_err(np_(r["phi"]), np.array(g["phi"][:P])).max() <= 1e-5


def test_adaptive_fp64_follows_the_oracle_schedule(H):
    # float64, gap checked every iteration: the GPU's adaptive run stops at
    # the oracle's iteration (same tau/sigma decisions) and on its value
    import torch
    from oracle import hopf as oh
    w = wl.workload_random10(12)
    ref = oh.value(w["system"], w["x"], w["t"], w["N"], oh.LEFT_RIEMANN, tau=w["tau"], tol=1e-9, adaptive=True)
    r = H.value(H.System.from_dict(w["system"]), cuda(w["x"], torch.float64), w["t"],
                H.Options(N=w["N"], tau=w["tau"], tol_gap=1e-9, precision=H.FP64, gap_every=1, max_iter=400000,
                          adaptive=True))
    assert np.all(r["status"].cpu().numpy() == 0)
    assert rel_err(np_(r["phi"]), ref["phi"]).max() <= 2e-9
    it_g, it_o = r["iters"].cpu().numpy(), ref["iters"]
    assert np.all(np.abs(it_g - it_o) <= 3), (it_g, it_o)


def test_adaptive_fp64_double_integrator_box(H):
    import torch
    g = gold("di_values_T1.5.json")
    w = wl.workload_di(g["meta"]["P"])
    r = H.value(H.System.from_dict(w["system"]), cuda(w["x"], torch.float64), g["meta"]["T"],
                H.Options(N=w["N"], rule=H.TRAPEZOID, tau=w["tau"], tol_gap=1e-11, precision=H.FP64,
                          max_iter=2000000, adaptive=True))
    assert np.all(r["status"].cpu().numpy() == 0)
    assert rel_err(np_(r["phi"]), np.array(g["phi"])).max() <= 1e-9


def test_adaptive_time_to_reach_chain10(H):
    g = gold("chain10_time_to_reach.json")
    m = g["meta"]
    sysd = H.System.from_dict(wl.spring_chain(masses=10, actuators=2, radius_target=1.0))
    opts = H.Options(N=m["N"], tau=m["tau"], t_max=m["t_max"], tol_T=1e-5, tol_gap=1e-5, max_iter=400000,
                     adaptive=True)
    r = H.time_to_reach(sysd, cuda(g["x"]), opts)
    assert np.all(np.isin(r["status"].cpu().numpy(), (0, 4))), r["status"]
    Tg = np.array(g["T"])
    assert np.all(np.abs(np_(r["T"]) - Tg) <= 1e-4 * Tg), (np_(r["T"]), Tg)


def test_adaptive_rejects_accel_and_warm(H):
    w = wl.workload_random10(4)
    sysd = H.System.from_dict(w["system"])
    with pytest.raises(H.HopfError):
        H.value(sysd, cuda(w["x"]), 2.0, H.Options(N=64, adaptive=True, accel=True))
