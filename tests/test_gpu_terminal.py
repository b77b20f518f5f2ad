"""Parity of the terminal-time-variable solves (p = e^{T A^T} q) with the FP64
oracle, full-size parity of the large-state configurations, and the node
table against one matrix exponential per node (§III.A, Eq. 20).

The value phi, the certified gap and p* (mapped back) are the same
quantities in either variable, so the stored oracle values serve both.
Tolerances as in test_gpu_parity: value 1e-5 max(1, |phi|) in float32,
time-to-reach 1e-4 T.
"""
import json
import os

import numpy as np
import pytest

from inputs import workloads as wl

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TERM = 1


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


# ------------------------------------------------------- small states
def test_random10_terminal_small_kernel_fewer_iterations(H):
    g = gold("random10_values.json")
    P = g["meta"]["P"]
    w = wl.workload_random10(P)
    sysd = H.System.from_dict(w["system"])
    rt = H.value(sysd, cuda(w["x"]), w["t"], H.Options(N=w["N"], tau=0.5, variables=TERM))
    st = rt["status"].cpu().numpy()
    assert np.all(st == 0), np.unique(st, return_counts=True)
    assert rel_err(np_(rt["phi"]), np.array(g["phi"])).max() <= 1e-5
    pe = np.linalg.norm(np_(rt["p"]) - np.array(g["p"]), axis=1) / np.maximum(1, np.linalg.norm(g["p"], axis=1))
    assert pe.max() < 5e-2
    ri = H.value(sysd, cuda(w["x"]), w["t"], H.Options(N=w["N"], tau=w["tau"]))
    assert rt["iters"].float().mean() < 0.5 * ri["iters"].float().mean()


def test_random10_terminal_full_size_sampled_against_oracle(H):
    # the benchmark launch (65,536 points, one call) in terminal-time variables
    from oracle import hopf as oh
    w = wl.workload_random10(65536)
    sysd = H.System.from_dict(w["system"])
    r = H.value(sysd, cuda(w["x"]), w["t"], H.Options(N=w["N"], tau=0.5, variables=TERM))
    st = r["status"].cpu().numpy()
    assert np.all(st == 0), np.unique(st, return_counts=True)
    idx = np.random.default_rng(15).choice(65536, 24, replace=False)
    ref = oh.value(w["system"], w["x"][idx], w["t"], w["N"], oh.LEFT_RIEMANN, tau=w["tau"], tol=1e-10,
                   max_iter=400000)
    assert rel_err(np_(r["phi"])[idx], ref["phi"]).max() <= 1e-5


@pytest.mark.parametrize("accel", [False, True])
def test_random10_terminal_parking_through_all_phases(H, accel):
    g = gold("random10_values.json")
    w = wl.workload_random10(320)
    sysd = H.System.from_dict(w["system"])
    opts = H.Options(N=w["N"], tau=2.0 if accel else 0.5, accel=accel, park_iters=8, variables=TERM)
    r = H.value(sysd, cuda(w["x"]), w["t"], opts)
    assert np.all(r["status"].cpu().numpy() == 0)
    assert rel_err(np_(r["phi"]), np.array(g["phi"])).max() <= 1e-5


def test_random10_terminal_generic_per_point_and_warm(H):
    g = gold("random10_values.json")
    P = 64
    w = wl.workload_random10(P)
    sysd = H.System.from_dict(w["system"])
    opts = H.Options(N=w["N"], tau=0.5, variables=TERM)
    r = H.value(sysd, cuda(w["x"]), cuda(np.full(P, w["t"])), opts)
    assert np.all(r["status"].cpu().numpy() == 0)
    assert rel_err(np_(r["phi"]), np.array(g["phi"][:P])).max() <= 1e-5
    # a warm start in the paper's variable is mapped in: from the oracle's p*
    # the solve is short and lands on the same value
    rw = H.value(sysd, cuda(w["x"]), w["t"], opts, p_init=cuda(np.array(g["p"][:P])))
    assert np.all(rw["status"].cpu().numpy() == 0)
    assert rw["iters"].float().mean() < 0.5 * r["iters"].float().mean()
    assert rel_err(np_(rw["phi"]), np.array(g["phi"][:P])).max() <= 1e-5


def test_di_terminal_fp64_trapezoid_box(H):
    import torch
    g = gold("di_values_T1.5.json")
    w = wl.workload_di(g["meta"]["P"])
    sysd = H.System.from_dict(w["system"])
    opts = H.Options(N=w["N"], rule=H.TRAPEZOID, tau=w["tau"], tol_gap=1e-11, precision=H.FP64,
                     max_iter=1000000, variables=TERM)
    r = H.value(sysd, cuda(w["x"], torch.float64), g["meta"]["T"], opts)
    assert np.all(r["status"].cpu().numpy() == 0)
    assert rel_err(np_(r["phi"]), np.array(g["phi"])).max() <= 1e-9
    # p* mapped back to the paper's variable
    assert np.allclose(np_(r["p"]), np.array(g["p"]), rtol=1e-3, atol=1e-3)


# ------------------------------------------------------- large states
def test_tile_kernel_terminal_against_oracle(H):
    from oracle import hopf as oh
    sysd = wl.random_system(324, 40, 5)
    x = wl.normal_points(424, 70, 40, 2.0)
    r = H.value(H.System.from_dict(sysd), cuda(x), 1.0, H.Options(N=48, tau=0.5, max_iter=200000, variables=TERM))
    assert np.all(r["status"].cpu().numpy() == 0)
    idx = [0, 33, 69]
    ref = oh.value(sysd, x[idx], 1.0, 48, oh.LEFT_RIEMANN, tau=0.5, tol=1e-9, max_iter=400000, variables="terminal")
    assert rel_err(np_(r["phi"])[idx], ref["phi"]).max() <= 1e-5


@pytest.mark.parametrize("variables,tau", [(TERM, 0.1), (0, 0.5)])
def test_chain200_full_size_against_oracle(H, variables, tau):
    # the 100-mass chain at full size (n = 200, m = 10 box, N = 512, T = 10)
    # on the tiled kernel: 32 points solved, every fourth compared
    g = gold("chain200_values_T10.json")
    m = g["meta"]
    w = wl.workload_chain(m["P"])
    sysd = H.System.from_dict(w["system"])
    r = H.value(sysd, cuda(w["x"]), m["T"], H.Options(N=m["N"], tau=tau, max_iter=400000, variables=variables))
    st = r["status"].cpu().numpy()
    assert np.all(st == 0), np.unique(st, return_counts=True)
    idx = np.array(g["idx"])
    err = rel_err(np_(r["phi"])[idx], np.array(g["phi"]))
    assert err.max() <= 1e-5, err


@pytest.mark.parametrize("variables,tau", [(TERM, 0.15), (0, 0.15)])
def test_random128_full_size_against_oracle(H, variables, tau):
    # the largest of the 64 random systems' sizes: n = 128, m = 16, N = 256
    g = gold("random128_values.json")
    sysd = wl.random_system(328, 128, 16)
    x = wl.normal_points(428, 8, 128, 2.0)
    r = H.value(H.System.from_dict(sysd), cuda(x), 2.0,
                H.Options(N=256, tau=tau, max_iter=400000, variables=variables))
    st = r["status"].cpu().numpy()
    assert np.all(st == 0), np.unique(st, return_counts=True)
    err = rel_err(np_(r["phi"]), np.array(g["phi"]))
    assert err.max() <= 1e-5, err


@pytest.mark.parametrize("T", [10.0, 40.0])
@pytest.mark.parametrize("variables", [0, TERM])
def test_node_table_against_expm_per_node(H, T, variables):
    # §III.A: the device builds K_i by repeated multiplication with e^{-hA}
    # (e^{hA} for terminal-time variables) over N = 512 nodes; compared with
    # one scipy expm per node at the chain's full size
    from oracle import hopf as oh
    sysd = wl.spring_chain()
    o = H.Options(N=512, precision=H.FP64, variables=variables)
    K, w = H.node_table(H.System.from_dict(sysd), T, o)
    if variables == 0:
        ref = oh.node_matrices(sysd, T, 512, oh.LEFT_RIEMANN)
    else:
        ref = oh.node_matrices_terminal(sysd, T, 512, oh.LEFT_RIEMANN)
    _, wref = oh.nodes(T, 512, oh.LEFT_RIEMANN)
    assert np.allclose(w, wref, rtol=1e-15)
    scale = np.abs(ref).max()
    assert np.abs(K - ref).max() <= 1e-10 * scale, np.abs(K - ref).max() / scale


# ------------------------------------------------------ time to reach
def test_di_time_to_reach_terminal_fp64(H):
    import torch
    g = gold("di_time_to_reach.json")
    m = g["meta"]
    w = wl.workload_di(m["P"])
    sysd = H.System.from_dict(w["system"])
    opts = H.Options(N=m["N"], rule=H.TRAPEZOID, tau=m["tau"], tol_gap=1e-8, precision=H.FP64, t_max=m["t_max"],
                     tol_T=1e-6, max_iter=1000000, variables=TERM)
    r = H.time_to_reach(sysd, cuda(w["x"], torch.float64), opts)
    T, Tg = np_(r["T"]), np.array(g["T"])
    st = r["status"].cpu().numpy()
    assert np.all((st == 0) | (st == 4)), np.unique(st, return_counts=True)
    assert np.all(np.abs(T - Tg) <= 1e-4 * np.maximum(Tg, 1e-3)), np.max(np.abs(T - Tg) / Tg)


@pytest.mark.parametrize("newton", [False, True])
def test_chain10_time_to_reach_terminal_fp32(H, newton):
    g = gold("chain10_time_to_reach.json")
    m = g["meta"]
    sysd = H.System.from_dict(wl.spring_chain(masses=10, actuators=2, radius_target=1.0))
    opts = H.Options(N=m["N"], tau=0.2, t_max=m["t_max"], tol_T=1e-5, tol_gap=1e-5, newton=newton,
                     max_iter=400000, variables=TERM)
    r = H.time_to_reach(sysd, cuda(g["x"]), opts)
    assert np.all(np.isin(r["status"].cpu().numpy(), (0, 4))), r["status"]
    Tg = np.array(g["T"])
    assert np.all(np.abs(np_(r["T"]) - Tg) <= 1e-4 * Tg), (np_(r["T"]), Tg)


def test_time_to_reach_step_cap_reports_maxiter(H):
    # with 3 candidate horizons per point the bisection cannot close the
    # bracket: open points return the top of their bracket (an upper bound on
    # T*) with HOPF_MAXITER; a point inside the target still returns 0
    import torch
    g = gold("di_time_to_reach.json")
    m = g["meta"]
    w = wl.workload_di(m["P"])
    x = np.vstack([w["x"][:6], [[0.01, 0.0]]])
    sysd = H.System.from_dict(w["system"])
    opts = H.Options(N=m["N"], rule=H.TRAPEZOID, tau=m["tau"], tol_gap=1e-8, precision=H.FP64, t_max=m["t_max"],
                     tol_T=1e-6, max_iter=1000000, max_steps=3)
    r = H.time_to_reach(sysd, cuda(x, torch.float64), opts)
    st = r["status"].cpu().numpy()
    T = np_(r["T"])
    Tg = np.array(g["T"][:6])
    assert r["steps"] == 3
    assert np.all(st[:6] == 1) and st[6] == 0 and T[6] == 0.0, st
    assert np.all(T[:6] >= Tg - 1e-9) and np.all(T[:6] <= m["t_max"])


def test_time_to_reach_rejects_tol_below_float64_resolution(H):
    sysd = H.System.from_dict(wl.double_integrator(0.1))
    with pytest.raises(H.HopfError):
        H.time_to_reach(sysd, cuda(np.ones((2, 2))), H.Options(tol_T=1e-17))
