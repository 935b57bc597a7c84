"""GPU parity of the extensions beyond Algorithm 2 against the FP64 oracle: residual
resampling (bit-exact given the same weights and uniforms), log predictive likelihoods
(FP32 exponentials of the running log weights, FP64 sums: 1e-6 absolute per observation),
Zellner's g-prior and the normalised prior (FP64, 1e-9 relative)."""
import math

import numpy as np
import pytest

import synthetic
from oracle import smc as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _gen(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _small(n=300, k=4, C=2, seed=0):
    g = _gen(seed)
    X = g.standard_normal((n, k))
    X[:, 0] = 1.0
    y = g.integers(0, C, n).astype(np.int32)
    return X, y


def _ctx(X, y, C, **kw):
    from paper_1304_4333_b300 import Sps
    return Sps(X, y, C, prior_sd=5.0, **kw)


@pytest.mark.parametrize("J,N", [(3, 64), (5, 1000), (2, 4096), (4, 7)])
def test_residual_resampling_bit_exact(cuda, J, N):
    X, y = _small()
    s = _ctx(X, y, 2)
    g = _gen(J * 1000 + N)
    w = np.exp(2.0 * g.standard_normal((J, N)))
    w[0, :] = 1.0                                   # equal weights: copies only
    if J > 2:
        w[2, :] = 0.0
        w[2, :4] = [1.0, 0.5, 0.25, 0.25]           # integral expected counts when N = 4 k
    w = w / w.max(axis=1, keepdims=True)
    u = g.random((J, N))
    got = s.resample(w.reshape(-1), u.reshape(-1), J, N, scheme="residual").reshape(J, N)
    for j in range(J):
        np.testing.assert_array_equal(got[j], OS.resample_residual(w[j], u[j]))


def test_residual_s_phase_keeps_floor_copies(cuda):
    w_ = synthetic.make_c1()
    s = _ctx(w_.X, w_.y, w_.C, resampling="residual")
    st = s.state(4, 256, seed=5)
    st.cphase()
    lw = st.get()["logw"].reshape(4, 256)
    idx = st.sphase().reshape(4, 256)
    for j in range(4):
        wj = np.exp(lw[j] - lw[j].max())
        c = np.bincount(idx[j], minlength=256)
        assert np.all(c >= np.floor(256 * wj / wj.sum() * (1 - 1e-6)))
        assert c.sum() == 256


def test_log_predictive_matches_oracle_cphase(cuda):
    w_ = synthetic.make_c1()
    s = _ctx(w_.X, w_.y, w_.C)
    st = s.state(4, 256, seed=11)
    th = st.get()["theta"]
    t_new, _, inc, lp = st.cphase(log_pred=True)
    ref = []
    t_o, _, _ = OS.cphase(w_.X, w_.y, w_.C, th, 0, 4, 256, log_pred=ref)
    assert t_new == t_o
    ref = np.array(ref)
    assert lp.shape == ref.shape
    np.testing.assert_allclose(lp, ref, atol=1e-6)
    np.testing.assert_allclose(lp.sum(axis=0), inc, atol=1e-5)


def test_run_log_predictive_sums_to_log_ml_and_is_exact_for_zero_covariates(cuda):
    w_ = synthetic.make_c1()
    s = _ctx(w_.X, w_.y, w_.C, seed=3)
    r = s.run(4, 256, log_pred=True)
    assert r.log_pred.shape == (w_.n,)
    assert np.all(np.isfinite(r.log_pred)) and np.all(r.log_pred < 0)
    assert r.log_pred.sum() == pytest.approx(r.log_ml, abs=1e-3)
    n, C = 80, 3
    X = np.zeros((n, 2))
    y = _gen(4).integers(0, C, n).astype(np.int32)
    r0 = _ctx(X, y, C, seed=1).run(4, 128, log_pred=True)
    np.testing.assert_allclose(r0.log_pred, -math.log(C), atol=1e-6)


def test_gprior_and_normalised_prior_match_oracle(cuda):
    from paper_1304_4333_b300 import prior_normalize
    for C in (2, 3):
        X, y = _small(n=500, k=5, C=C, seed=7)
        s = _ctx(X, y, C)
        for g in (1.0, 0.25):
            mean, cov = s.gprior(g)
            m_o, c_o = OS.gprior_covariance(X, C, g)
            np.testing.assert_array_equal(mean, m_o)
            np.testing.assert_allclose(cov, c_o, rtol=1e-9, atol=1e-12 * np.abs(c_o).max())
        s.set_prior(prior_cov=cov, prior_mean=mean)
        r = s.run(4, 128)
        assert np.isfinite(r.log_ml)
    g = _gen(8)
    mu = g.standard_normal((4, 3))
    A = g.standard_normal((4, 3, 3))
    Sig = np.einsum("cij,ckj->cik", A, A) + np.eye(3)[None]
    m, c = prior_normalize(mu, Sig)
    m_o, c_o = OS.normalise_prior(mu, Sig)
    np.testing.assert_allclose(m, m_o, rtol=0, atol=0)
    np.testing.assert_allclose(c, c_o, rtol=0, atol=0)


@pytest.mark.parametrize("prec", ["fp32", "split"])
def test_autograd_function_backward_is_the_gradient_kernel(cuda, prec):
    # backward is the context's gradient function (FP32 SIMT, or the tensor-core form in split
    # precision, C = 3 here); the split bound follows its BF16 hi + lo operands
    torch = cuda
    from oracle import logit as OL
    from paper_1304_4333_b300.autograd import loglik
    X, y = _small(n=600, k=6, C=3, seed=12)
    s = _ctx(X, y, 3, precision=prec)
    g = _gen(13)
    th = torch.tensor(0.3 * g.standard_normal((90, 12)), device="cuda", requires_grad=True)
    wts = torch.tensor(g.standard_normal(90), device="cuda")
    ll = loglik(th, s, 550, prec)
    (wts * ll).sum().backward()
    _, G = s.loglik_grad(th.detach(), 550)
    torch.testing.assert_close(th.grad, wts[:, None] * G, rtol=0, atol=0)
    ll_o, G_o = OL.loglik_grad(X, y, th.detach().cpu().numpy(), 3, 550)
    np.testing.assert_allclose(ll.detach().cpu().numpy(), ll_o, rtol=1e-6 if prec == "fp32" else 1e-5)
    ref = wts.cpu().numpy()[:, None] * G_o
    rel = np.max(np.abs(th.grad.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert rel < (1e-5 if prec == "fp32" else 2e-4), rel
