"""The tensor-core (tcgen05) large-state kernel against the FP64 oracle and
against the CUDA-core tiled kernel: terminal-time variables, diagonal W, one
shared horizon, 3 x tf32 products with float32 accumulation in tensor memory.
Tolerance: value 1e-5 max(1, |phi|), as in the other parity tests."""
import json
import os

import numpy as np
import pytest

from inputs import workloads as wl

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TERM, TENSOR, TILE = 1, 2, 3


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


def cuda(a):
    import torch
    return torch.as_tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def np_(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel_err(a, b):
    return np.abs(a - b) / np.maximum(1.0, np.abs(b))


def test_chain200_tensor_kernel_against_oracle(H):
    # n = 200, m = 10 box (10 rows per node, 6 nodes per 64-row block), N = 512:
    # 520 points = 5 tiles, the last one ragged; slots refill from the queue
    g = gold("chain200_values_T10.json")
    m = g["meta"]
    w = wl.workload_chain(520)
    sysd = H.System.from_dict(w["system"])
    r = H.value(sysd, cuda(w["x"]), m["T"], H.Options(N=m["N"], tau=0.1, max_iter=200000, variables=TERM,
                                                     kernel=TENSOR))
    st = r["status"].cpu().numpy()
    assert np.all(st == 0), np.unique(st, return_counts=True)
    idx = np.array(g["idx"])
    err = rel_err(np_(r["phi"])[idx], np.array(g["phi"]))
    assert err.max() <= 1e-5, err
    assert np_(r["gap"]).max() <= 1e-5


def test_random128_tensor_kernel_against_oracle(H):
    g = gold("random128_values.json")
    sysd = wl.random_system(328, 128, 16)
    x = wl.normal_points(428, 8, 128, 2.0)
    r = H.value(H.System.from_dict(sysd), cuda(x), 2.0,
                H.Options(N=256, tau=0.15, max_iter=400000, variables=TERM, kernel=TENSOR))
    assert np.all(r["status"].cpu().numpy() == 0)
    assert rel_err(np_(r["phi"]), np.array(g["phi"])).max() <= 1e-5


@pytest.mark.parametrize("n,m,N,kind", [(40, 5, 48, 0), (24, 3, 37, 1), (64, 8, 100, 0), (96, 12, 64, 1)])
def test_tensor_kernel_matches_tiled_kernel_and_oracle(H, n, m, N, kind):
    # ball and box control, control paddings 4, 8 and 16, node counts that do
    # not fill the last block; 300 points (3 tiles, one ragged)
    from oracle import hopf as oh
    sysd = wl.random_system(500 + n, n, m)
    if kind == 1:
        sysd["ctrl_kind"] = 1
        sysd["half_widths"] = np.full(m, 0.7)
    x = wl.normal_points(600 + n, 300, n, 2.0)
    S = H.System.from_dict(sysd)
    base = dict(N=N, tau=0.3, max_iter=200000, variables=TERM)
    rt = H.value(S, cuda(x), 1.5, H.Options(kernel=TENSOR, **base))
    rs = H.value(S, cuda(x), 1.5, H.Options(kernel=TILE, **base))
    assert np.all(rt["status"].cpu().numpy() == 0)
    assert np.all(rs["status"].cpu().numpy() == 0)
    assert rel_err(np_(rt["phi"]), np_(rs["phi"])).max() <= 2e-5
    idx = [0, 151, 299]
    ref = oh.value(sysd, x[idx], 1.5, N, oh.LEFT_RIEMANN, tau=0.3, tol=1e-9, max_iter=400000, variables="terminal")
    assert rel_err(np_(rt["phi"])[idx], ref["phi"]).max() <= 1e-5


def test_tensor_kernel_warm_start_and_zero_horizon(H):
    # warm start from the oracle's p* (mapped to q inside the library): few
    # iterations, same values; T = 0 returns the terminal cost
    from oracle import hopf as oh
    sysd = wl.random_system(77, 48, 6)
    x = wl.normal_points(78, 160, 48, 2.0)
    S = H.System.from_dict(sysd)
    o = H.Options(N=64, tau=0.3, max_iter=200000, variables=TERM, kernel=TENSOR)
    ref = oh.value(sysd, x, 1.0, 64, oh.LEFT_RIEMANN, tau=0.3, tol=1e-10, max_iter=400000, variables="terminal")
    cold = H.value(S, cuda(x), 1.0, o)
    warm = H.value(S, cuda(x), 1.0, o, p_init=cuda(ref["p"]))
    assert np.all(warm["status"].cpu().numpy() == 0)
    assert rel_err(np_(warm["phi"]), ref["phi"]).max() <= 1e-5
    assert warm["iters"].float().mean() < 0.5 * cold["iters"].float().mean()
    z = H.value(S, cuda(x), 0.0, o)
    J = np.einsum("pi,ij,pj->p", x, np.linalg.inv(sysd["W"]), x) - 1.0
    assert np.allclose(np_(z["phi"]), J, rtol=1e-5)


def _first_steps(sysd, x, T, N, tau, steps):
    """float64 restatement of the kernel's iteration in terminal-time
    variables (Eq. 15 with the prox of Eq. 23 and a diagonal Eq. 37), cold
    start; returns -P at the pbar of step `steps` (what a point reports when
    it stops at max_iter = steps - 1) and the relative gap."""
    from oracle import hopf as oh
    prob = oh.setup(sysd, T, N, oh.LEFT_RIEMANN, tau, variables="terminal")
    K, w = prob["K"], prob["w"]
    Wd = np.diag(prob["M"])
    Sd = np.diag(prob["S"])
    xq = x @ prob["E"].T
    p = xq.copy()
    pb = p.copy()
    y = None
    for it in range(steps):
        z = np.einsum("imn,pn->pim", K, pb)
        yo = z if y is None else y
        v = yo + prob["sigma"] * z
        if sysd["ctrl_kind"] == 0:
            nv = np.linalg.norm(v, axis=2, keepdims=True)
            y = v * np.minimum(1.0, w[None, :, None] / np.maximum(nv, 1e-300))
            H = np.sum(w[None, :] * np.linalg.norm(z, axis=2), axis=1)
        else:
            y = np.clip(v, -w[None, :, None], w[None, :, None])
            H = np.sum(w[None, :] * np.abs(z).sum(axis=2), axis=1)
        u = np.einsum("imn,pim->pn", K, y)
        Pv = np.sum(pb * (0.25 * Wd * pb - xq), axis=1) + 1.0 + H
        Dv = 1.0 - np.sum((xq - u) ** 2 / Wd, axis=1)
        pn = Sd * (p + tau * (xq - u))
        pb = 2.0 * pn - p
        p = pn
    return -Pv, (Pv - Dv) / np.maximum(1.0, np.maximum(np.abs(Pv), np.abs(Dv)))


@pytest.mark.parametrize("which", ["ball_n24_m3", "chain_n200_m10"])
def test_tensor_kernel_first_iterations_match_float64_steps(H, which):
    # three iterations (max_iter = 2 stops every point after the third): the
    # reported -P and gap follow the float64 restatement of the same steps
    if which == "ball_n24_m3":
        sysd, T, N, tau = wl.random_system(91, 24, 3), 1.2, 37, 0.3
        x = wl.normal_points(92, 130, 24, 2.0)
    else:
        sysd, T, N, tau = wl.spring_chain(), 10.0, 512, 0.1
        x = wl.normal_points(3, 130, 200, 1.0)
    r = H.value(H.System.from_dict(sysd), cuda(x), T,
                H.Options(N=N, tau=tau, max_iter=2, variables=TERM, kernel=TENSOR))
    st = r["status"].cpu().numpy()
    assert np.all(st == 1), np.unique(st, return_counts=True)
    assert np.all(r["iters"].cpu().numpy() == 2)
    phi_ref, gap_ref = _first_steps(sysd, x, T, N, tau, 3)
    err = rel_err(np_(r["phi"]), phi_ref)
    # early on, phi = -P of the chain is a difference of terms about 100 times
    # larger (sum_i w_i |K_i pbar|_1 over 5,120 rows against the quadratic
    # part), so float32 rounding of the iterates shows at ~1e-4 there
    tol = 1e-5 if which == "ball_n24_m3" else 2e-3
    assert err.max() <= tol, (err.max(), np_(r["phi"])[:4], phi_ref[:4])
    assert np.allclose(np_(r["gap"]), gap_ref, rtol=1e-3, atol=1e-5), (np_(r["gap"])[:4], gap_ref[:4])
