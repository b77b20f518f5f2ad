"""Parity of the fixed-step rule (left Riemann sum with dt = t_max / N, the
last node weighted T - t_last; one table on [0, t_max] in terminal-time
variables serves every horizon) with the FP64 oracle's FixedStep rule.

Values: 1e-5 max(1, |phi|) in float32, 1e-9 in float64.  Time to reach:
|T - T_oracle| <= 1e-4 T in float32.
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


def oracle_values(sysd, x, T, rule, tau, tol):
    """Oracle value of every point at its own horizon (one call per distinct T)."""
    from oracle import hopf as oh
    phi = np.empty(len(T))
    p = np.empty_like(np.asarray(x, dtype=np.float64))
    for Tv in np.unique(T):
        idx = np.where(T == Tv)[0]
        r = oh.value(sysd, x[idx], float(Tv), rule.N, rule, tau=tau, tol=tol, max_iter=2000000,
                     variables="terminal")
        phi[idx] = r["phi"]
        p[idx] = r["p"]
    return phi, p


# ------------------------------------------------------------------ values
def test_fixed_step_fp64_double_integrator_per_point_horizons(H):
    # general kernel in float64: horizons between multiples of the step,
    # T = 0 (the terminal cost itself), T = t_max, and one out of range
    import torch
    from oracle import hopf as oh
    sysd = wl.double_integrator(0.1)
    rule = oh.FixedStep(2.0, 64)
    T = np.array([0.0, 0.013, 0.5, 0.77, 1.0, 1.31, 2.0, 2.5])
    x = np.random.default_rng(5).uniform(-1.2, 1.2, (T.size, 2))
    opts = H.Options(rule=H.LEFT_FIXED, N=64, t_max=2.0, tau=2.0, tol_gap=1e-11, precision=H.FP64,
                     max_iter=2000000, variables=TERM)
    r = H.value(H.System.from_dict(sysd), cuda(x, torch.float64), cuda(T, torch.float64), opts)
    st = r["status"].cpu().numpy()
    assert np.all(st[:-1] == 0), st
    assert st[-1] == 2 and np.isnan(np_(r["phi"])[-1])
    phi, p = oracle_values(sysd, x[:-1], T[:-1], rule, 2.0, 1e-13)
    assert rel_err(np_(r["phi"])[:-1], phi).max() <= 1e-9, (np_(r["phi"])[:-1], phi)
    assert np.allclose(np_(r["p"])[:-1], p, rtol=1e-3, atol=1e-3)


def test_fixed_step_fp32_general_kernel_small_state(H):
    from oracle import hopf as oh
    sysd = wl.random_system(11, 4, 2)
    rule = oh.FixedStep(2.0, 40)
    P = 16
    x = wl.normal_points(12, P, 4, 1.0)
    T = np.tile([0.3, 0.77, 1.313, 2.0], P // 4)
    opts = H.Options(rule=H.LEFT_FIXED, N=40, t_max=2.0, tau=0.2, max_iter=400000, variables=TERM)
    r = H.value(H.System.from_dict(sysd), cuda(x), cuda(T), opts)
    assert np.all(r["status"].cpu().numpy() == 0)
    phi, _ = oracle_values(sysd, x, T, rule, 0.2, 1e-11)
    assert rel_err(np_(r["phi"]), phi).max() <= 1e-5


def test_fixed_step_tile_kernel_ragged_horizons(H):
    # the tiled kernel with one table on [0, 8] (256 nodes): 96 points (three
    # tiles and a ragged tail) at spread horizons, T = 0 and one out of range;
    # a warm start from the oracle's p* lands on the same values in fewer steps
    from oracle import hopf as oh
    sysd = wl.spring_chain(masses=20, actuators=2, radius_target=1.0)
    rule = oh.FixedStep(8.0, 256)
    P = 96
    x = wl.normal_points(21, P, 40, 0.7)
    T = np.round(np.random.default_rng(22).uniform(0.2, 8.0, P), 3)
    T[5], T[40] = 0.0, 8.5
    opts = H.Options(rule=H.LEFT_FIXED, N=256, t_max=8.0, tau=0.2, max_iter=400000, variables=TERM)
    sys_ = H.System.from_dict(sysd)
    r = H.value(sys_, cuda(x), cuda(T), opts)
    st = r["status"].cpu().numpy()
    assert st[40] == 2 and np.isnan(np_(r["phi"])[40])
    ok = np.delete(np.arange(P), 40)
    assert np.all(st[ok] == 0), np.unique(st, return_counts=True)
    idx = np.array([0, 5, 17, 33, 64, 95])
    phi, p = oracle_values(sysd, x[idx], T[idx], rule, 0.2, 1e-9)
    assert rel_err(np_(r["phi"])[idx], phi).max() <= 1e-5, (np_(r["phi"])[idx], phi)
    rw = H.value(sys_, cuda(x[idx]), cuda(T[idx]), opts, p_init=cuda(p))
    assert np.all(rw["status"].cpu().numpy() == 0)
    assert rel_err(np_(rw["phi"]), phi).max() <= 1e-5
    assert rw["iters"].float().mean() < r["iters"][idx].float().mean()


def test_fixed_step_chain200_at_a_multiple_of_the_step_equals_eq17(H):
    # T = 10 = 512 dt: the fixed-step nodes are Eq. 17's N = 512 nodes, so the
    # stored full-size oracle values apply (one table on [0, 40], 2048 nodes)
    g = gold("chain200_values_T10.json")
    m = g["meta"]
    w = wl.workload_chain(m["P"])
    opts = H.Options(rule=H.LEFT_FIXED, N=2048, t_max=40.0, tau=0.1, max_iter=400000, variables=TERM)
    r = H.value(H.System.from_dict(w["system"]), cuda(w["x"]), m["T"], opts)
    st = r["status"].cpu().numpy()
    assert np.all(st == 0), np.unique(st, return_counts=True)
    idx = np.array(g["idx"])
    err = rel_err(np_(r["phi"])[idx], np.array(g["phi"]))
    assert err.max() <= 1e-5, err


def test_fixed_step_chain200_between_multiples_of_the_step(H):
    name = os.path.join(GOLD, "chain200_fixed_values.json")
    if not os.path.exists(name):
        pytest.skip("stored values not generated")
    g = gold("chain200_fixed_values.json")
    w = wl.workload_chain(8)
    idx = np.array(g["idx"])
    opts = H.Options(rule=H.LEFT_FIXED, N=2048, t_max=40.0, tau=0.1, max_iter=400000, variables=TERM)
    r = H.value(H.System.from_dict(w["system"]), cuda(w["x"][idx]), cuda(np.array(g["T"])), opts)
    assert np.all(r["status"].cpu().numpy() == 0)
    err = rel_err(np_(r["phi"]), np.array(g["phi"]))
    assert err.max() <= 1e-5, err


# ----------------------------------------------------------- time to reach
@pytest.mark.parametrize("newton", [False, True])
def test_fixed_step_time_to_reach_fp64_double_integrator(H, newton):
    import torch
    from oracle import hopf as oh
    sysd = wl.double_integrator(0.1)
    w = wl.workload_di(12)
    x = np.vstack([w["x"], [[0.02, 0.0]]])          # the last point starts inside the target
    ref = oh.time_to_reach(sysd, x, 8.0, 512, oh.FixedStep(8.0, 512), tau=2.0, tol_T=1e-9, tol_gap=1e-10,
                           variables="terminal")
    opts = H.Options(rule=H.LEFT_FIXED, N=512, t_max=8.0, tau=2.0, tol_gap=1e-10, tol_T=1e-8, precision=H.FP64,
                     max_iter=2000000, newton=newton, variables=TERM)
    r = H.time_to_reach(H.System.from_dict(sysd), cuda(x, torch.float64), opts)
    st = r["status"].cpu().numpy()
    assert np.all(np.isin(st, (0, 4))), st
    T = np_(r["T"])
    assert T[-1] == 0.0
    assert np.all(np.abs(T - ref["T"]) <= 1e-6 * np.maximum(ref["T"], 1e-3)), (T, ref["T"])


def test_fixed_step_time_to_reach_warm_bracket_and_start(H):
    # a bracket around T* and a warm p_init (the oracle's p* at T*) give the
    # same T*; a bracket below T* is detected and replaced by [0, t_max]
    import torch
    from oracle import hopf as oh
    sysd = wl.double_integrator(0.1)
    w = wl.workload_di(8)
    ref = oh.time_to_reach(sysd, w["x"], 8.0, 512, oh.FixedStep(8.0, 512), tau=2.0, tol_T=1e-9, tol_gap=1e-10,
                           variables="terminal")
    opts = H.Options(rule=H.LEFT_FIXED, N=512, t_max=8.0, tau=2.0, tol_gap=1e-10, tol_T=1e-8, precision=H.FP64,
                     max_iter=2000000, variables=TERM)
    S = H.System.from_dict(sysd)
    x = cuda(w["x"], torch.float64)
    lo = cuda(ref["T"] * 0.9, torch.float64)
    hi = cuda(np.minimum(ref["T"] * 1.1, 8.0), torch.float64)
    r = H.time_to_reach(S, x, opts, T_lo=lo, T_hi=hi, p_init=cuda(ref["p"], torch.float64))
    assert np.all(np.isin(r["status"].cpu().numpy(), (0, 4)))
    assert np.all(np.abs(np_(r["T"]) - ref["T"]) <= 1e-6 * ref["T"]), (np_(r["T"]), ref["T"])
    lo2 = cuda(ref["T"] * 0.5, torch.float64)
    hi2 = cuda(ref["T"] * 0.8, torch.float64)
    r2 = H.time_to_reach(S, x, opts, T_lo=lo2, T_hi=hi2)
    assert np.all(np.abs(np_(r2["T"]) - ref["T"]) <= 1e-6 * ref["T"]), (np_(r2["T"]), ref["T"])


@pytest.mark.parametrize("newton", [False, True])
def test_fixed_step_time_to_reach_fp32_chain_tile(H, newton):
    # tiled kernel in sign mode (n = 20): 24 points, three against the oracle
    g = gold("chain10_fixed_time_to_reach.json")
    m = g["meta"]
    sysd = wl.spring_chain(masses=10, actuators=2, radius_target=1.0)
    x = wl.normal_points(11, m["P"], 20, 0.7)
    opts = H.Options(rule=H.LEFT_FIXED, N=m["N"], t_max=m["t_max"], tau=m["tau"], tol_gap=1e-5, tol_T=1e-5,
                     newton=newton, max_iter=400000, variables=TERM)
    r = H.time_to_reach(H.System.from_dict(sysd), cuda(x), opts)
    st = r["status"].cpu().numpy()
    assert np.all(np.isin(st, (0, 4))), st
    Tg = np.array(g["T"])
    T = np_(r["T"])[g["idx"]]
    assert np.all(np.abs(T - Tg) <= 1e-4 * Tg), (T, Tg)


def test_fixed_step_rejects_paper_variables_and_adaptive(H):
    sysd = H.System.from_dict(wl.double_integrator(0.1))
    with pytest.raises(H.HopfError):
        H.value(sysd, cuda(np.ones((2, 2))), 1.0, H.Options(rule=H.LEFT_FIXED, t_max=2.0))
    with pytest.raises(H.HopfError):
        H.value(sysd, cuda(np.ones((2, 2))), 1.0,
                H.Options(rule=H.LEFT_FIXED, t_max=2.0, variables=TERM, adaptive=True))
