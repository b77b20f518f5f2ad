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


def test_adam_constant_gradient_steps_and_second_step_closed_form():
    # With a constant gradient the bias-corrected moments are exactly g and g^2
    # at every step, so each step is -lr g / (|g| + eps); a wrong bias-correction
    # exponent shows from the second step on.
    g0 = np.array([0.5, -4.0, 2e-3])
    p = [np.array([1.0, -2.0, 3.0])]
    m, v = [np.zeros(3)], [np.zeros(3)]
    want = p[0].copy()
    for step in range(1, 6):
        om.adam_step(p, [g0.copy()], m, v, step, 0.01)
        want = want - 0.01 * g0 / (np.abs(g0) + 1e-8)
        assert np.allclose(p[0], want, rtol=0, atol=1e-12), step
    # two different gradients: m_hat = (b1 g1 + g2)/(1 + b1), v_hat = (b2 g1^2 + g2^2)/(1 + b2)
    g1, g2 = np.array([1.0, -0.3]), np.array([-2.0, 0.7])
    p = [np.zeros(2)]
    m, v = [np.zeros(2)], [np.zeros(2)]
    om.adam_step(p, [g1], m, v, 1, 0.1, beta1=0.8, beta2=0.9, eps=0.0)
    after1 = p[0].copy()
    om.adam_step(p, [g2], m, v, 2, 0.1, beta1=0.8, beta2=0.9, eps=0.0)
    mh = (0.8 * g1 + g2) / 1.8
    vh = (0.9 * g1 ** 2 + g2 ** 2) / 1.9
    assert np.allclose(p[0] - after1, -0.1 * mh / np.sqrt(vh), rtol=1e-13)
