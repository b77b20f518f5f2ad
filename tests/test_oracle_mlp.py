"""Pins of the FP64 MLP oracle: GELU against tabulated normal-CDF values and
the hand-written backward pass against central finite differences of the
forward pass (a dropped term or transposed operand in the chain rule fails)."""
import numpy as np

from inputs import workloads as wl
from oracle import mlp as om


def test_gelu_values():
    # Phi(1) = 0.8413447460685429, Phi(-0.5) = 0.3085375387259869 (normal CDF tables)
    assert np.isclose(om.gelu(1.0), 0.8413447460685429, rtol=1e-14)
    assert np.isclose(om.gelu(-0.5), -0.5 * 0.3085375387259869, rtol=1e-14)
    a = np.linspace(-3, 3, 13)
    h = 1e-6
    assert np.allclose(om.gelu_grad(a), (om.gelu(a + h) - om.gelu(a - h)) / (2 * h), atol=1e-8)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    layers = wl.mlp_init(3, [4, 7, 6, 3])
    layers = [(W, rng.normal(0, 0.1, b.shape)) for W, b in layers]
    x = rng.normal(0, 1, (5, 4))
    y = rng.normal(0, 1, (5, 3))
    xs, xsc = rng.normal(0, 0.1, 4), rng.uniform(0.5, 2, 4)
    ys, ysc = rng.normal(0, 0.1, 3), rng.uniform(0.5, 2, 3)
    loss, grads = om.loss_and_grads(layers, x, y, xs, xsc, ys, ysc)
    h = 1e-6
    for li in range(len(layers)):
        for which in (0, 1):
            arr = layers[li][which]
            g = grads[li][which]
            it = np.nditer(arr, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = arr[idx]
                arr[idx] = old + h
                lp, _ = om.loss_and_grads(layers, x, y, xs, xsc, ys, ysc)
                arr[idx] = old - h
                lm, _ = om.loss_and_grads(layers, x, y, xs, xsc, ys, ysc)
                arr[idx] = old
                assert abs((lp - lm) / (2 * h) - g[idx]) < 1e-7, (li, which, idx)


def test_adam_first_step_is_signed_lr():
    # Bias correction makes the first Adam step -lr * g / (|g| + eps') ~ -lr sign(g).
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    om.adam_step(p, g, m, v, 1, 0.01)
    assert np.allclose(p[0], [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01 * 1e-3 / (1e-3 + 1e-8)], atol=1e-12)
