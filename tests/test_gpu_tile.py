"""Parity of the tiled large-state kernel (one shared table, float32) with the
FP64 oracle and with the warp-per-point kernel, through the C ABI.

Cases: random systems with n = 24..125 and m = 1..16 (ball), the spring chain
with box control and m = 10, several tiles with a ragged last tile, slots that
take new points from the queue (P larger than the slots), a warm start from
the oracle's p*, and T = 0.  Tolerance: |phi - phi_ref| <= 1e-5 max(1, |phi|)
at certified gap <= 1e-5 (float32).
"""
import numpy as np
import pytest

from inputs import workloads as wl

pytestmark = pytest.mark.gpu


def cuda(a, dtype=None):
    import torch
    return torch.as_tensor(np.asarray(a), dtype=dtype or torch.float32, device="cuda")


def np_(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel_err(a, b):
    return np.abs(a - b) / np.maximum(1.0, np.abs(b))


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1712_08226_gb300 as H
    from paper_1712_08226_gb300 import build
    build.build()
    return H


def oracle_phi(sysd, x, T, N, rule, tau, tol=1e-8):
    from oracle import hopf as oh
    return oh.value(sysd, x, T, N, rule, tau, tol=tol)["phi"]


@pytest.mark.parametrize("n,m,P", [(24, 3, 70), (40, 5, 33), (33, 1, 40), (48, 12, 36)])
def test_tile_random_system_against_oracle(H, n, m, P):
    sysd = wl.random_system(300 + n, n, m)
    x = wl.normal_points(400 + n, P, n, 2.0)
    N, T, tau = 64, 1.0, 0.2
    r = H.value(H.System.from_dict(sysd), cuda(x), T, H.Options(N=N, tau=tau, tol_gap=1e-5, max_iter=200000))
    st = r["status"].cpu().numpy()
    assert np.all(st == 0), np.unique(st, return_counts=True)
    assert np_(r["gap"]).max() <= 1e-5
    idx = np.arange(0, P, max(1, P // 8))
    ref = oracle_phi(sysd, x[idx], T, N, wl.LEFT_RIEMANN, tau)
    err = rel_err(np_(r["phi"])[idx], ref)
    assert err.max() <= 1e-5, err


def test_tile_chain_box_m10_against_oracle_and_generic(H):
    sysd = wl.spring_chain(masses=20, actuators=10, radius_target=0.5)   # n = 40, m = 10, box
    x = wl.normal_points(5, 45, 40, 1.0)
    N, T, tau = 64, 3.0, 0.5
    o = H.Options(N=N, tau=tau, tol_gap=1e-5, max_iter=400000)
    r = H.value(H.System.from_dict(sysd), cuda(x), T, o)
    assert np.all(r["status"].cpu().numpy() == 0)
    idx = np.arange(0, 45, 9)
    ref = oracle_phi(sysd, x[idx], T, N, wl.LEFT_RIEMANN, tau)
    assert rel_err(np_(r["phi"])[idx], ref).max() <= 1e-5
    o.kernel = 1
    g = H.value(H.System.from_dict(sysd), cuda(x), T, o)
    assert np.all(g["status"].cpu().numpy() == 0)
    assert rel_err(np_(r["phi"]), np_(g["phi"])).max() <= 2e-5


def test_tile_wide_tiles_and_queue_refill_sampled(H):
    # more points than 152 blocks x 64 slots: 64-slot tiles, slots refilled
    n, m, P = 20, 3, 12000
    sysd = wl.random_system(77, n, m)
    x = wl.normal_points(78, P, n, 2.0)
    N, T, tau = 32, 1.0, 0.3
    r = H.value(H.System.from_dict(sysd), cuda(x), T, H.Options(N=N, tau=tau, tol_gap=1e-5, max_iter=200000))
    st = r["status"].cpu().numpy()
    assert np.all(st == 0)
    idx = np.random.default_rng(0).choice(P, 10, replace=False)
    ref = oracle_phi(sysd, x[idx], T, N, wl.LEFT_RIEMANN, tau)
    assert rel_err(np_(r["phi"])[idx], ref).max() <= 1e-5


def test_tile_large_ragged_system_and_warm_start(H):
    # one system of the 64-system workload at its largest size (n = 125, m = 16)
    from oracle import hopf as oh
    n, m = 125, 16
    sysd = wl.random_system(107, n, m)
    x = wl.normal_points(207, 3, n, 2.0)
    N, T, tau = 256, 2.0, 0.15
    ref = oh.value(sysd, x, T, N, wl.LEFT_RIEMANN, tau, tol=1e-7)
    o = H.Options(N=N, tau=tau, tol_gap=1e-5, max_iter=200000)
    r = H.value(H.System.from_dict(sysd), cuda(x), T, o)
    assert np.all(r["status"].cpu().numpy() == 0)
    assert rel_err(np_(r["phi"]), ref["phi"]).max() <= 1e-5
    o.tol_gap = 5e-6                # margin for the float32 evaluation of P at the edge
    w = H.value(H.System.from_dict(sysd), cuda(x), T, o, p_init=cuda(ref["p"]))
    assert np.all(w["status"].cpu().numpy() == 0)
    assert rel_err(np_(w["phi"]), ref["phi"]).max() <= 1e-5
    assert w["iters"].cpu().numpy().max() < r["iters"].cpu().numpy().min()


def test_tile_zero_horizon(H):
    sysd = wl.random_system(9, 30, 4)
    x = wl.normal_points(10, 5, 30, 0.1)
    r = H.value(H.System.from_dict(sysd), cuda(x), 0.0, H.Options(N=16, tau=0.5))
    W = sysd["W"]
    J = np.einsum("ij,jk,ik->i", x, np.linalg.inv(W), x) - 1.0
    assert np.allclose(np_(r["phi"]), J, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("which", ["unscented", "d30", "d120"])
def test_stacked_copy_workloads_against_oracle(H, which):
    # §VI.B / §VI.C: copies of the double integrator sharing one control
    # (n = 10 runs on the small-state kernel, n = 30 and 120 on the tiled one)
    w = wl.workload_unscented(6) if which == "unscented" else wl.workload_dimension(int(which[1:]), 4)
    T = 2.5
    r = H.value(H.System.from_dict(w["system"]), cuda(w["x"]), T,
                H.Options(N=w["N"], tau=w["tau"], tol_gap=1e-5, max_iter=400000))
    assert np.all(r["status"].cpu().numpy() == 0)
    ref = oracle_phi(w["system"], w["x"], T, w["N"], w["rule"], w["tau"], tol=1e-8)
    assert rel_err(np_(r["phi"]), ref).max() <= 1e-5


@pytest.mark.parametrize("which,prec", [("unscented", 64), ("unscented", 32), ("d30", 32), ("d120", 32)])
def test_structured_stacked_solve_matches_dense(H, which, prec):
    # hopf_value_stacked (K~_i p = K_i sum_j p_j, block-diagonal prox) against
    # the dense stacked problem in the oracle
    import torch
    w = wl.workload_unscented(5) if which == "unscented" else wl.workload_dimension(int(which[1:]), 4)
    T = 2.5
    base = H.System.from_dict(w["system"]["base"])
    if prec == 64:
        o = H.Options(N=w["N"], tau=w["tau"], tol_gap=1e-10, precision=H.FP64, max_iter=1000000)
        x, tol = cuda(w["x"], torch.float64), 1e-9
    else:
        o = H.Options(N=w["N"], tau=w["tau"], tol_gap=1e-5, max_iter=400000)
        x, tol = cuda(w["x"]), 1e-5
    r = H.value_stacked(base, w["system"]["W_blocks"], x, T, o)
    assert np.all(r["status"].cpu().numpy() == 0)
    ref = oracle_phi(w["system"], w["x"], T, w["N"], w["rule"], w["tau"], tol=1e-11 if prec == 64 else 1e-8)
    assert rel_err(np_(r["phi"]), ref).max() <= tol
    # per-point horizons (one base table per copy and point)
    Tp = np.linspace(1.0, 3.0, len(w["x"]))
    r2 = H.value_stacked(base, w["system"]["W_blocks"], x, cuda(Tp, x.dtype), o)
    assert np.all(r2["status"].cpu().numpy() == 0)
    ref2 = np.array([oracle_phi(w["system"], w["x"][i:i + 1], Tp[i], w["N"], w["rule"], w["tau"],
                                tol=1e-11 if prec == 64 else 1e-8)[0] for i in range(len(Tp))])
    assert rel_err(np_(r2["phi"]), ref2).max() <= tol


@pytest.mark.parametrize("case", ["chain_box", "random_ball"])
def test_tile_accelerated_against_oracle(H, case):
    # the accelerated steps (strongly convex G, per-slot tau and sigma, prox
    # through the eigen-decomposition of M) reach the oracle's value
    if case == "chain_box":
        sysd = wl.spring_chain(masses=20, actuators=10, radius_target=0.5)
        x, T, N = wl.normal_points(5, 40, 40, 1.0), 3.0, 64
    else:
        sysd = wl.random_system(341, 36, 4)
        x, T, N = wl.normal_points(342, 40, 36, 2.0), 1.5, 64
    o = H.Options(N=N, tau=2.0, tol_gap=1e-5, max_iter=400000, accel=True)
    r = H.value(H.System.from_dict(sysd), cuda(x), T, o)
    assert np.all(r["status"].cpu().numpy() == 0)
    from oracle import hopf as oh
    idx = np.arange(0, 40, 8)
    ref = oh.value(sysd, x[idx], T, N, wl.LEFT_RIEMANN, 2.0, tol=1e-8, max_iter=400000, accel=True)
    assert np.all(ref["status"] == 0)
    assert rel_err(np_(r["phi"])[idx], ref["phi"]).max() <= 1e-5


def test_calls_on_two_streams_overlap_safely(H):
    # one workspace per stream: two systems solved concurrently on two streams
    # give the same results as the same calls one after the other
    import torch
    sysA, sysB = wl.random_system(501, 30, 4), wl.random_system(502, 44, 6)
    xA, xB = wl.normal_points(503, 300, 30, 2.0), wl.normal_points(504, 300, 44, 2.0)
    o = H.Options(N=64, tau=0.2, tol_gap=1e-5, max_iter=200000)
    SA, SB = H.System.from_dict(sysA), H.System.from_dict(sysB)
    ref = [H.value(SA, cuda(xA), 1.0, o), H.value(SB, cuda(xB), 1.0, o)]
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a_in, b_in = cuda(xA), cuda(xB)
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        ra = H.value(SA, a_in, 1.0, o, stream=s1)
    with torch.cuda.stream(s2):
        rb = H.value(SB, b_in, 1.0, o, stream=s2)
    torch.cuda.synchronize()
    # (the certificate sums use shared-memory float atomics, so the last bits
    # and the exact stopping iteration may differ between runs)
    for r, rr in ((ra, ref[0]), (rb, ref[1])):
        assert np.all(r["status"].cpu().numpy() == 0)
        assert rel_err(np_(r["phi"]), np_(rr["phi"])).max() <= 2e-5


def test_tile_warm_start_path_and_fallback_list(H):
    # value_warm on a large state runs the tiled kernel twice: the warm solve
    # from the network's prediction (capped), then a cold solve of the listed
    # points it left uncertified.  An untrained network and a tiny cap send
    # most points down the fallback; every value must still match a cold solve.
    import torch
    from paper_1712_08226_gb300.warmstart import WarmStartNet, value_warm
    sysd = wl.random_system(601, 40, 5)
    x = cuda(wl.normal_points(602, 300, 40, 2.0))
    S = H.System.from_dict(sysd)
    o = H.Options(N=64, tau=0.2, tol_gap=1e-5, max_iter=200000)
    cold = H.value(S, x, 1.0, o)
    net = WarmStartNet(40, 40, hidden=64, seed=3)
    net.set_normalisation(x, cold["p"])
    w = value_warm(S, x, 1.0, net, o, max_iter_warm=40)
    torch.cuda.synchronize()
    assert int(w["n_fallback"].item()) > 0
    assert np.all(w["status"].cpu().numpy() == 0)
    assert rel_err(np_(w["phi"]), np_(cold["phi"])).max() <= 2e-5
