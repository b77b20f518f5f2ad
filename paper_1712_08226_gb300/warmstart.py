"""Learned warm start: a network trained on the solver's own solutions.

The network (n -> hidden -> hidden -> n, GELU, bfloat16 weights, float32
accumulation) predicts p* from x; ``value_warm`` starts the primal-dual
iteration from the prediction and re-solves from the cold start any point the
warm solve does not certify.  Forward, backward and optimiser steps are the
library's CUDA kernels (hopf_mlp_*); this module holds the parameters in
device tensors and drives the training loop.
"""
import ctypes

import numpy as np

from . import _lib
from .api import Options, _check, _Marshal


class WarmStartNet:
    """Parameters and optimiser state of the warm-start network on one device."""

    def __init__(self, n_in, n_out, hidden=256, seed=0, device="cuda"):
        import torch
        from inputs.workloads import mlp_init
        self.torch = torch
        self.lib = _lib.load()
        self.n_in, self.hidden, self.n_out = int(n_in), int(hidden), int(n_out)
        self.count = int(self.lib.hopf_mlp_param_count(self.n_in, self.hidden, self.n_out))
        flat = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in
                               mlp_init(seed, [self.n_in, self.hidden, self.hidden, self.n_out])])
        assert flat.size == self.count
        f32 = dict(dtype=torch.float32, device=device)
        self.w = torch.tensor(flat, **f32)
        self.w_bf16 = torch.empty(self.count, dtype=torch.bfloat16, device=device)
        self.m = torch.zeros(self.count, **f32)
        self.v = torch.zeros(self.count, **f32)
        self.grad = torch.zeros(self.count, **f32)
        self.loss = torch.zeros(1, **f32)
        self.x_shift = torch.zeros(self.n_in, **f32)
        self.x_scale = torch.ones(self.n_in, **f32)
        self.y_shift = torch.zeros(self.n_out, **f32)
        self.y_scale = torch.ones(self.n_out, **f32)
        self.step = 0
        self.use_tc = True          # prediction on the tensor cores (training stays on CUDA cores)
        self.sync()

    def c_struct(self):
        p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        return _lib.HopfMlp(self.n_in, self.hidden, self.n_out, p(self.w), p(self.w_bf16), p(self.m), p(self.v),
                            p(self.x_shift), p(self.x_scale), p(self.y_shift), p(self.y_scale),
                            int(self.use_tc))

    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def sync(self):
        net = self.c_struct()
        _check(self.lib, self.lib.hopf_mlp_sync(ctypes.byref(net), self._stream()))

    def set_normalisation(self, x, y):
        """Per-feature mean and standard deviation of the training inputs/targets."""
        self.x_shift.copy_(x.mean(0))
        self.x_scale.copy_(x.std(0).clamp_min(1e-6))
        self.y_shift.copy_(y.mean(0))
        self.y_scale.copy_(y.std(0).clamp_min(1e-6))

    def forward(self, x):
        x = x.contiguous()
        y = self.torch.empty(x.shape[0], self.n_out, dtype=self.torch.float32, device=x.device)
        net = self.c_struct()
        _check(self.lib, self.lib.hopf_mlp_forward(ctypes.byref(net), x.shape[0], ctypes.c_void_p(x.data_ptr()),
                                                   ctypes.c_void_p(y.data_ptr()), self._stream()))
        return y

    def loss_grad(self, x, y):
        """Loss (device scalar) and gradient (device vector, owned by the net)."""
        net = self.c_struct()
        _check(self.lib, self.lib.hopf_mlp_loss_grad(ctypes.byref(net), x.shape[0], ctypes.c_void_p(x.data_ptr()),
                                                     ctypes.c_void_p(y.data_ptr()),
                                                     ctypes.c_void_p(self.loss.data_ptr()),
                                                     ctypes.c_void_p(self.grad.data_ptr()), self._stream()))
        return self.loss, self.grad

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        net = self.c_struct()
        _check(self.lib, self.lib.hopf_mlp_adam(ctypes.byref(net), ctypes.c_void_p(self.grad.data_ptr()), self.step,
                                                lr, beta1, beta2, eps, self._stream()))

    def fit(self, x, y, epochs=20, batch=4096, lr=2e-3, lr_final=2e-5, seed=0, log_every=0):
        """Adam with a cosine learning-rate schedule on (x, y) device tensors.
        Returns the list of per-epoch mean training losses."""
        torch = self.torch
        n = x.shape[0]
        g = torch.Generator(device=x.device)
        g.manual_seed(seed)
        steps_per_epoch = max(1, n // batch)
        total = epochs * steps_per_epoch
        hist = []
        k = 0
        for ep in range(epochs):
            perm = torch.randperm(n, device=x.device, generator=g)
            acc = torch.zeros((), device=x.device)
            for s in range(steps_per_epoch):
                idx = perm[s * batch:(s + 1) * batch]
                xb = x.index_select(0, idx).contiguous()
                yb = y.index_select(0, idx).contiguous()
                loss, _ = self.loss_grad(xb, yb)
                acc += loss[0]
                cur = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * k / max(1, total - 1)))
                self.adam(cur)
                k += 1
            hist.append(float(acc) / steps_per_epoch)
            if log_every and (ep + 1) % log_every == 0:
                print(f"epoch {ep + 1}: loss {hist[-1]:.3e}", flush=True)
        return hist


def value_warm(system, x, t, net, opts=None, max_iter_warm=None, stream=None):
    """Warm-started batched value solve (float32; device tensors, or numpy host
    arrays copied in and out inside the call).  Returns dict(phi, p, gap,
    iters, status, n_fallback)."""
    import torch
    lib = _lib.load()
    opts = opts or Options()
    mar = _Marshal(opts.precision, x)
    xx = mar.inp(x)
    P = int(xx.shape[0])
    scalar_t = np.ndim(t) == 0 and not (hasattr(t, "ndim") and t.ndim > 0)
    tt = mar.inp(np.array([float(t)]) if scalar_t else t)
    out = dict(phi=mar.out((P,)), p=mar.out((P, system.n)), gap=mar.out((P,)),
               iters=mar.out((P,), True), status=mar.out((P,), True))
    nfb = torch.zeros(1, dtype=torch.int32, device=xx.device) if mar.device else np.zeros(1, np.int32)
    prob = system.c_struct()
    o = opts.c_struct(not mar.device)
    c = net.c_struct()
    mi = opts.max_iter if max_iter_warm is None else int(max_iter_warm)
    rc = lib.hopf_value_warm(ctypes.byref(prob), ctypes.byref(o), ctypes.byref(c), P, mar.ptr(xx), mar.ptr(tt),
                             0 if scalar_t else 1, mi, mar.ptr(out["phi"]), mar.ptr(out["p"]), mar.ptr(out["gap"]),
                             mar.ptr(out["iters"]), mar.ptr(out["status"]), mar.ptr(nfb), mar.stream(stream))
    _check(lib, rc)
    out["n_fallback"] = nfb
    return out

