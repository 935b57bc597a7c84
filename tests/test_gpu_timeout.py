"""The fused kernel's bounded waits, made to run out from the host (no GPU fault involved).

sps_set_debug stops the kernel's TMA producer before it issues any copy, so nothing is in
flight; every consumer wait (MMA thread, epilogue warps, and the relay of a CTA pair) then gives
up after the short limit, the CTAs drain, free their tensor memory and return, and the call
reports SPS_ERR_TIMEOUT. The next call on the same context must succeed and match the oracle.
Both launch forms are covered: CTA pairs (SPS_TC_CLUSTER=2) and single CTAs (SPS_TC_CLUSTER=1).
"""
import numpy as np
import pytest

from oracle.logit import loglik as oracle_loglik

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("C,mode", [(2, "2"), (2, "1"), (3, "2"), (3, "1")])
def test_stalled_producer_times_out_and_context_recovers(cuda, monkeypatch, C, mode):
    from paper_1304_4333_b300 import Sps
    from paper_1304_4333_b300._native import SpsError
    monkeypatch.setenv("SPS_TC_CLUSTER", mode)
    g = np.random.Generator(np.random.PCG64(9 + C))
    n, k = 1200, 10
    X = g.standard_normal((n, k))
    X[:, 0] = 1.0
    y = g.integers(0, C, n).astype(np.int32)
    th = 0.3 * g.standard_normal((400, k * (C - 1)))
    s = Sps(X, y, C, prior_sd=5.0)
    assert s.lib.sps_set_debug(s.ctx, 1, 20_000_000) == 0
    with pytest.raises(SpsError) as e:
        s.loglik(th, n, "split")
    assert e.value.status == 6
    assert "timed out" in str(e.value)
    assert s.lib.sps_set_debug(s.ctx, 0, 0) == 0
    got = s.loglik(th, n, "split")
    np.testing.assert_allclose(got, oracle_loglik(X, y, th, C, n), rtol=1e-5)
    s.close()
