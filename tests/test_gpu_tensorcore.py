"""Tensor-core primitives (tcgen05 MMA into tensor memory): exact products.

Inputs are multiples of 1/4 in [-2, 2], exactly representable in tf32, so
every product and every partial sum is exact in float32 and the result must
equal the float64 matrix product bit for bit; any error in the operand layout,
the descriptors or the accumulator read-out shows up."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,K", [(16, 8), (64, 32), (256, 64), (48, 128), (208, 16)])
def test_tf32_mma_exact(N, K):
    import torch
    from paper_1712_08226_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    rng = np.random.default_rng(N * 1000 + K)
    A = rng.integers(-8, 9, (128, K)) / 4.0
    B = rng.integers(-8, 9, (N, K)) / 4.0
    tA = torch.tensor(A, dtype=torch.float32, device="cuda")
    tB = torch.tensor(B, dtype=torch.float32, device="cuda")
    tD = torch.full((128, N), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    rc = lib.hopf_tc_selftest(N, K, p(tA), p(tB), p(tD), p(err),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert np.array_equal(tD.cpu().numpy().astype(np.float64), A @ B.T)
