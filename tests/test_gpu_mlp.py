"""Warm-start network kernels against the FP64 MLP oracle, and what the
trained network gains over the cold start."""
import numpy as np
import pytest

from inputs import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    import paper_1712_08226_gb300 as H
    from paper_1712_08226_gb300 import build
    build.build()
    H._lib.load()
    return H


def _net_and_oracle(seed=3, n_in=5, hidden=24, n_out=3):
    import torch
    from paper_1712_08226_gb300.warmstart import WarmStartNet
    net = WarmStartNet(n_in, n_out, hidden=hidden, seed=seed)
    rng = np.random.default_rng(seed + 1)
    # non-zero biases and normalisation so every term is exercised
    with torch.no_grad():
        cnt = net.count
        w = net.w.cpu().numpy()
        w += rng.normal(0, 0.05, cnt).astype(np.float32)
        net.w.copy_(torch.tensor(w))
        net.x_shift.copy_(torch.tensor(rng.normal(0, 0.2, n_in), dtype=torch.float32))
        net.x_scale.copy_(torch.tensor(rng.uniform(0.5, 2.0, n_in), dtype=torch.float32))
        net.y_shift.copy_(torch.tensor(rng.normal(0, 0.2, n_out), dtype=torch.float32))
        net.y_scale.copy_(torch.tensor(rng.uniform(0.5, 2.0, n_out), dtype=torch.float32))
    net.sync()
    # oracle layers with the bfloat16-rounded weights and float32 biases the kernels use
    wb = net.w_bf16.float().cpu().numpy().astype(np.float64)
    wf = net.w.cpu().numpy().astype(np.float64)
    sizes = [n_in, hidden, hidden, n_out]
    layers, off = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = wb[off:off + a * b].reshape(b, a)
        off += a * b
        bias = wf[off:off + b]
        off += b
        layers.append((W, bias))
    norm = [t.cpu().numpy().astype(np.float64) for t in (net.x_shift, net.x_scale, net.y_shift, net.y_scale)]
    return net, layers, norm


def test_forward_matches_oracle(H):
    import torch
    from oracle import mlp as om
    net, layers, (xs, xsc, ys, ysc) = _net_and_oracle()
    net.use_tc = False
    x = np.random.default_rng(7).normal(0, 1.5, (77, 5))        # ragged vs the 64-row tile
    y = net.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    ref = om.predict(layers, x, xs, xsc, ys, ysc)
    assert np.allclose(y, ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())


def _bf16(a):
    import torch
    return torch.tensor(a, dtype=torch.float64).to(torch.bfloat16).double().numpy()


@pytest.mark.parametrize("B,hidden", [(77, 24), (300, 256)])
def test_tensor_core_forward_matches_bf16_model(H, B, hidden):
    # The tcgen05 path multiplies bfloat16 activations by bfloat16 weights with
    # float32 accumulation: the oracle rounds every layer input to bfloat16 the
    # same way and must agree up to the summation order.
    import torch
    from oracle import mlp as om
    net, layers, (xs, xsc, ys, ysc) = _net_and_oracle(hidden=hidden)
    net.use_tc = True
    x = np.random.default_rng(17).normal(0, 1.5, (B, 5))        # B not a multiple of 128
    y = net.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy().astype(np.float64)
    h = _bf16((x - xs) / xsc)
    for li, (W, b) in enumerate(layers):
        a = h @ W.T + b
        h = _bf16(om.gelu(a)) if li + 1 < len(layers) else a
    ref = h * ysc + ys
    assert np.allclose(y, ref, rtol=2e-3, atol=2e-3 * np.abs(ref).max()), np.abs(y - ref).max()
    # and it stays close to the float32 path
    net.use_tc = False
    y32 = net.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert np.abs(y - y32).max() <= 0.05 * np.abs(y32).max()


def test_gradient_matches_oracle(H):
    import torch
    from oracle import mlp as om
    net, layers, (xs, xsc, ys, ysc) = _net_and_oracle()
    rng = np.random.default_rng(8)
    x = rng.normal(0, 1.5, (70, 5))
    t = rng.normal(0, 1.0, (70, 3))
    loss, g = net.loss_grad(torch.tensor(x, dtype=torch.float32, device="cuda"),
                            torch.tensor(t, dtype=torch.float32, device="cuda"))
    ref_loss, ref_g = om.loss_and_grads(layers, x, t, xs, xsc, ys, ysc)
    assert abs(float(loss[0]) - ref_loss) <= 1e-4 * ref_loss
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in ref_g])
    got = g.cpu().numpy().astype(np.float64)
    assert np.abs(got - flat).max() <= 1e-4 * np.abs(flat).max(), np.abs(got - flat).max()


def test_adam_step_matches_oracle(H):
    import torch
    from oracle import mlp as om
    net, _, _ = _net_and_oracle()
    rng = np.random.default_rng(9)
    g = rng.normal(0, 1e-2, net.count)
    w0 = net.w.cpu().numpy().astype(np.float64)
    net.grad.copy_(torch.tensor(g, dtype=torch.float32))
    for _ in range(3):
        net.adam(1e-3)
    params, m, v = [w0.copy()], [np.zeros_like(w0)], [np.zeros_like(w0)]
    gg = [net.grad.cpu().numpy().astype(np.float64)]
    for s in range(1, 4):
        om.adam_step(params, gg, m, v, s, 1e-3)
    assert np.allclose(net.w.cpu().numpy(), params[0], rtol=0, atol=1e-6)
    assert np.array_equal(net.w_bf16.float().cpu().numpy(), net.w.to(torch.bfloat16).float().cpu().numpy())


def test_trained_warm_start_beats_cold_start(H):
    # Train on solutions the GPU solver produces for one system, then solve
    # fresh points from the network's prediction: fewer iterations, same
    # certified values, every point certified (fallback to cold if needed).
    import torch
    from paper_1712_08226_gb300.warmstart import WarmStartNet, value_warm
    w = wl.workload_random10(1)
    sysd = H.System.from_dict(w["system"])
    opts = H.Options(N=256, tau=2.0, tol_gap=1e-5, accel=True)
    xtr = torch.tensor(wl.normal_points(40, 32768, 10, 2.0), dtype=torch.float32, device="cuda")
    lab = H.value(sysd, xtr, 2.0, H.Options(N=256, tau=2.0, tol_gap=2e-6, accel=True))
    assert np.all(lab["status"].cpu().numpy() == 0)
    net = WarmStartNet(10, 10, hidden=256, seed=0)
    net.set_normalisation(xtr, lab["p"])
    hist = net.fit(xtr, lab["p"], epochs=8, batch=2048, lr=2e-3)
    assert hist[-1] < 0.2 * hist[0]
    xte = torch.tensor(wl.normal_points(41, 4096, 10, 2.0), dtype=torch.float32, device="cuda")
    cold = H.value(sysd, xte, 2.0, opts)
    warm = value_warm(sysd, xte, 2.0, net, opts, max_iter_warm=2000)
    assert np.all(warm["status"].cpu().numpy() == 0)
    phi_c = cold["phi"].cpu().numpy().astype(np.float64)
    phi_w = warm["phi"].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(phi_w - phi_c) / np.maximum(1.0, np.abs(phi_c))) <= 2e-5
    it_c = cold["iters"].float().mean().item()
    it_w = warm["iters"].float().mean().item()
    assert it_w < 0.8 * it_c, (it_w, it_c)
    # the warm-started values against the FP64 oracle directly, on a sample
    from oracle import hopf as oh
    idx = np.random.default_rng(16).choice(4096, 16, replace=False)
    xs = wl.normal_points(41, 4096, 10, 2.0)[idx]
    ref = oh.value(w["system"], xs, 2.0, 256, oh.LEFT_RIEMANN, tau=0.15, tol=1e-10, max_iter=400000)
    assert np.max(np.abs(phi_w[idx] - ref["phi"]) / np.maximum(1.0, np.abs(ref["phi"]))) <= 1e-5
    # the same network warm-starting the solve in terminal-time variables: the
    # prediction of p* is mapped to q, the values are the oracle's
    opts_t = H.Options(N=256, tau=0.5, tol_gap=1e-5, variables=1)
    warm_t = value_warm(sysd, xte, 2.0, net, opts_t, max_iter_warm=2000)
    cold_t = H.value(sysd, xte, 2.0, opts_t)
    assert np.all(warm_t["status"].cpu().numpy() == 0)
    phi_t = warm_t["phi"].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(phi_t[idx] - ref["phi"]) / np.maximum(1.0, np.abs(ref["phi"]))) <= 1e-5
    # (this small network's prediction is too coarse to shorten the ~80-step
    # terminal-variable solves much; the benchmark's trained network does)
    assert warm_t["iters"].float().mean().item() < 1.25 * cold_t["iters"].float().mean().item()
