"""The allocation-free log-likelihood entry point (sps_loglik_noalloc).

sps_loglik_noalloc exists for callers that cannot let the library allocate device memory during
a call (memory owned by another allocator, loops that cannot absorb cudaMalloc's
synchronisation); its scratch is a fixed device array shared by all calls. This file is collected
last so that a run stopping at its first failure has already run every other test. The checks:
two calls in a row with different sizes, each bit-identical to sps_loglik (the same kernels and
summation order) and within the split-precision tolerance (1e-5 relative) of the FP64 oracle, so
the second call sees nothing left over from the first; free device memory unchanged across calls
after the first; a call too large for the fixed array refused with SPS_ERR_INVALID_ARG; and a
kernel timeout (forced by the diagnostics switch that stops the TMA producer) reported as NaN
results, after which the next call is correct again.
"""
import ctypes as C

import numpy as np
import pytest

from oracle.logit import loglik as oracle_loglik

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


def _noalloc(s, th, t, sync=True):
    torch = pytest.importorskip("torch")
    out = torch.empty(th.shape[0], dtype=torch.float64, device="cuda")
    s.lib.sps_set_stream(s.ctx, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    st = s.lib.sps_loglik_noalloc(s.ctx, C.c_void_p(th.data_ptr()), th.shape[0], int(t), C.c_void_p(out.data_ptr()))
    if sync:
        torch.cuda.synchronize()
    return st, out


@pytest.mark.parametrize("C_out", [2, 3])
def test_two_calls_match_sps_loglik_and_the_oracle(torch_cuda, C_out):
    torch = torch_cuda
    from paper_1304_4333_b300 import Sps
    X, y = _problem(1500, 12, C_out, 1)
    s = Sps(X, y, C_out, prior_sd=5.0)
    D = 12 * (C_out - 1)
    g = np.random.Generator(np.random.PCG64(2))
    for P, t in ((3000, 1500), (700, 777)):
        th_h = 0.3 * g.standard_normal((P, D))
        th = torch.from_numpy(th_h).cuda()
        st, got = _noalloc(s, th, t)
        assert st == 0, s.lib.sps_last_error(s.ctx).decode()
        ref = s.loglik(th, t, "split")
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())
        idx = np.array([0, 1, P // 2, P - 1])
        o = oracle_loglik(X, y, th_h[idx], C_out, t)
        np.testing.assert_allclose(got.cpu().numpy()[idx], o, rtol=1e-5)


def test_calls_after_the_first_allocate_no_device_memory(torch_cuda):
    torch = torch_cuda
    from paper_1304_4333_b300 import Sps
    X, y = _problem(2000, 12, 2, 4)
    s = Sps(X, y, 2, prior_sd=5.0)
    g = np.random.Generator(np.random.PCG64(5))
    ths = [torch.from_numpy(0.3 * g.standard_normal((P, 12))).cuda() for P in (3000, 700, 3000, 129)]
    outs = [torch.empty(th.shape[0], dtype=torch.float64, device="cuda") for th in ths]
    s.lib.sps_set_stream(s.ctx, C.c_void_p(torch.cuda.current_stream().cuda_stream))

    def call(i, t):
        return s.lib.sps_loglik_noalloc(s.ctx, C.c_void_p(ths[i].data_ptr()), ths[i].shape[0], t,
                                        C.c_void_p(outs[i].data_ptr()))

    assert call(0, 2000) == 0            # the first call on this device looks up the array
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for i, t in ((1, 1999), (2, 777), (3, 2000), (0, 1500)):
        assert call(i, t) == 0, s.lib.sps_last_error(s.ctx).decode()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_oversized_call_is_refused(torch_cuda):
    torch = torch_cuda
    from paper_1304_4333_b300 import Sps
    X, y = _problem(400, 12, 2, 3)
    s = Sps(X, y, 2, prior_sd=5.0)
    th = torch.zeros((1 << 18, 12), dtype=torch.float64, device="cuda")
    st, _ = _noalloc(s, th, 400)
    assert st == 1
    assert "static area" in s.lib.sps_last_error(s.ctx).decode()


def test_timeout_gives_nan_and_the_next_call_recovers(torch_cuda):
    torch = torch_cuda
    from paper_1304_4333_b300 import Sps
    X, y = _problem(1000, 12, 2, 6)
    s = Sps(X, y, 2, prior_sd=5.0)
    th_h = 0.3 * np.random.Generator(np.random.PCG64(7)).standard_normal((500, 12))
    th = torch.from_numpy(th_h).cuda()
    # the producer issues no copy: every consumer wait runs out after 20 ms
    assert s.lib.sps_set_debug(s.ctx, 1, 20_000_000) == 0
    st, got = _noalloc(s, th, 1000)
    assert st == 0
    assert np.all(np.isnan(got.cpu().numpy()))
    assert s.lib.sps_set_debug(s.ctx, 0, 0) == 0
    st, got = _noalloc(s, th, 1000)
    assert st == 0
    np.testing.assert_allclose(got.cpu().numpy(), oracle_loglik(X, y, th_h, 2, 1000), rtol=1e-5)
