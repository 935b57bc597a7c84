"""The allocation-free log-likelihood entry point (sps_loglik_noalloc) against sps_loglik.

sps_loglik_noalloc exists for callers that cannot let the library allocate device memory during
a call (memory owned by another allocator, loops that cannot absorb cudaMalloc's
synchronisation); its scratch is a fixed device array shared by all calls. This file is collected
last so that a run stopping at its first failure has already run every other test. The checks:
two calls in a row with different sizes, each equal to sps_loglik within the split-precision
tolerance (1e-5 relative), so the second call sees nothing left over from the first; and a call
too large for the fixed array is refused with SPS_ERR_INVALID_ARG.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _problem(n, k, C_out, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    X = g.standard_normal((n, k))
    X[:, 0] = 1.0
    X[:, k - 3:] = (g.random((n, 3)) < 0.3).astype(float)
    y = g.integers(0, C_out, n).astype(np.int32)
    return X, y


def _noalloc(s, th, t):
    torch = pytest.importorskip("torch")
    out = torch.empty(th.shape[0], dtype=torch.float64, device="cuda")
    s.lib.sps_set_stream(s.ctx, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    st = s.lib.sps_loglik_noalloc(s.ctx, C.c_void_p(th.data_ptr()), th.shape[0], int(t), C.c_void_p(out.data_ptr()))
    torch.cuda.synchronize()
    return st, out


@pytest.mark.parametrize("C_out", [2, 3])
def test_two_calls_match_sps_loglik(torch_cuda, C_out):
    torch = torch_cuda
    from paper_1304_4333_b300 import Sps
    X, y = _problem(1500, 12, C_out, 1)
    s = Sps(X, y, C_out, prior_sd=5.0)
    D = 12 * (C_out - 1)
    g = np.random.Generator(np.random.PCG64(2))
    for P, t in ((3000, 1500), (700, 777)):
        th = torch.from_numpy(0.3 * g.standard_normal((P, D))).cuda()
        st, got = _noalloc(s, th, t)
        assert st == 0, s.lib.sps_last_error(s.ctx).decode()
        ref = s.loglik(th, t, "split")
        torch.cuda.synchronize()
        np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=1e-5)


def test_oversized_call_is_refused(torch_cuda):
    torch = torch_cuda
    from paper_1304_4333_b300 import Sps
    X, y = _problem(400, 12, 2, 3)
    s = Sps(X, y, 2, prior_sd=5.0)
    th = torch.zeros((1 << 18, 12), dtype=torch.float64, device="cuda")
    st, _ = _noalloc(s, th, 400)
    assert st == 1
    assert "static area" in s.lib.sps_last_error(s.ctx).decode()
