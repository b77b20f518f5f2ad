"""FP64 CPU oracle for the warm-start multilayer perceptron.

TEST INFRASTRUCTURE ONLY: used by the tests (gradient checks of the CUDA
training kernels) and nowhere in the product path.

The network maps a query point x to a predicted optimal dual p* (and, for
time-to-reach, T*):  n_in -> 256 -> 256 -> n_out with the exact GELU
g(a) = a (1 + erf(a / sqrt 2)) / 2 after each hidden layer.  Inputs and
targets are standardised with fixed per-feature shifts and scales that are
part of the model.  The loss is the mean squared error over a batch and
over the outputs.  The paper has no learned component; this follows the
plain definitions (chain rule, Adam of Kingma and Ba 2015).
"""
import numpy as np
from scipy.special import erf

SQRT2 = np.sqrt(2.0)


def gelu(a):
    """Exact GELU: a * Phi(a), Phi the standard normal CDF."""
    return 0.5 * a * (1.0 + erf(a / SQRT2))


def gelu_grad(a):
    """d/da [a Phi(a)] = Phi(a) + a phi(a)."""
    return 0.5 * (1.0 + erf(a / SQRT2)) + a * np.exp(-0.5 * a * a) / np.sqrt(2.0 * np.pi)


def forward(layers, x, x_shift, x_scale):
    """Returns (out, cache).  layers = [(W (out,in), b (out,)), ...]; the last
    layer is affine, the others are followed by GELU.  Output is in
    standardised units."""
    h = (np.asarray(x, dtype=np.float64) - x_shift) / x_scale
    cache = [h]
    for li, (W, b) in enumerate(layers):
        a = h @ W.T + b
        if li + 1 < len(layers):
            cache.append(a)
            h = gelu(a)
            cache.append(h)
        else:
            h = a
    return h, cache


def predict(layers, x, x_shift, x_scale, y_shift, y_scale):
    """Prediction in physical units: out * y_scale + y_shift."""
    out, _ = forward(layers, x, x_shift, x_scale)
    return out * y_scale + y_shift


def loss_and_grads(layers, x, y, x_shift, x_scale, y_shift, y_scale):
    """Mean squared error between the standardised output and the standardised
    target (y - y_shift) / y_scale, and its gradient for every W and b."""
    out, cache = forward(layers, x, x_shift, x_scale)
    t = (np.asarray(y, dtype=np.float64) - y_shift) / y_scale
    Bsz, n_out = out.shape
    diff = out - t
    loss = float(np.sum(diff * diff) / (Bsz * n_out))
    g = 2.0 * diff / (Bsz * n_out)             # d loss / d out
    grads = [None] * len(layers)
    L = len(layers)
    for li in range(L - 1, -1, -1):
        W, b = layers[li]
        h_in = cache[0] if li == 0 else cache[2 * li]
        grads[li] = (g.T @ h_in, g.sum(axis=0))
        if li > 0:
            a_prev = cache[2 * li - 1]
            g = (g @ W) * gelu_grad(a_prev)
    return loss, grads


def adam_step(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected) for a flat list of arrays, in place."""
    for i, (p, g) in enumerate(zip(params, grads)):
        m[i] = beta1 * m[i] + (1.0 - beta1) * g
        v[i] = beta2 * v[i] + (1.0 - beta2) * g * g
        mh = m[i] / (1.0 - beta1 ** step)
        vh = v[i] / (1.0 - beta2 ** step)
        p -= lr * mh / (np.sqrt(vh) + eps)
