"""One MALA step with given randomness (sps_mala_step_given) against the oracle's MALA step.

Same normals z and uniforms u on both sides. The library forms the drift sigma g / 2 and the
proposal-density ratio with FP32 products of the FP32 Cholesky factor and the FP32 gradient,
and evaluates the log-likelihood and gradient with its split-precision (tensor-core) or FP32
kernels; the oracle is FP64 throughout. Bars: log alpha within
r (|ll(theta)| + |ll(theta')|) + 1e-4 |log alpha| + 1e-4, r the kernels' relative tolerance
(1e-5 split, 1e-6 FP32) on each log-likelihood; the same decisions wherever |log u - log alpha|
is more than twice that tolerance; the accepted particles within 1e-5 relative (+1e-5 absolute
for the FP32 drift); the returned log-likelihoods within the kernels' relative tolerance.
"""
import numpy as np
import pytest

import synthetic
from oracle import logit as OL
from oracle import smc as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _data(C):
    if C == 2:
        w = synthetic.make_c1()
        return w.X, w.y, w.theta_true
    g = np.random.Generator(np.random.PCG64(40 + C))
    n, k = 700, 6
    X = g.standard_normal((n, k))
    X[:, 0] = 1.0
    X[:, -2:] = (g.random((n, 2)) < 0.3).astype(float)
    beta = 0.4 * g.standard_normal(k * (C - 1))
    eta = np.concatenate([np.zeros((n, 1))] + [X @ beta[c * k:(c + 1) * k][:, None] for c in range(C - 1)], axis=1)
    y = np.argmax(eta + g.gumbel(size=eta.shape), axis=1).astype(np.int32)
    return X, y, beta


@pytest.mark.parametrize("C,prec", [(2, "split"), (2, "fp32"), (3, "split"), (4, "split"), (3, "fp32")])
def test_mala_step_given_randomness(cuda, C, prec):
    from paper_1304_4333_b300 import Sps
    X, y, beta = _data(C)
    D = beta.shape[0]
    s = Sps(X, y, C, prior_sd=5.0, precision=prec)
    P = 1024
    t = X.shape[0] - 37
    th = synthetic.particles_around(beta, P, 0.2, seed=17)
    prior = OS.GaussianPrior.isotropic(D, 5.0)
    Sigma = 0.3 * OS.particle_covariance(th) * (2.38 ** 2 / D)
    g = np.random.Generator(np.random.PCG64(18))
    z = g.standard_normal((P, D))
    u = g.random(P)
    ll = OL.loglik(X, y, th, C, t)
    th_o, ll_o, acc_o, la_o = OS.mala_step(X, y, C, t, th, ll, prior, Sigma, z, u)
    th_g, ll_g, la_g, acc_g = s.mala_step_given(th, t, Sigma, z, u)
    # log alpha carries the two log-likelihoods' own bars (1e-5 split, 1e-6 FP32, relative) and
    # the FP32 drift and proposal ratio (1e-4 relative)
    rtol = 1e-5 if prec == "split" else 1e-6
    # (the proposals' log-likelihoods are within 10 % of the current ones here)
    tol = rtol * 2.2 * np.abs(ll) + 1e-4 * np.abs(la_o) + 1e-4
    err = np.abs(la_g - la_o)
    print(f"C={C} {prec}: max |log alpha error| {err.max():.2e}, max tolerance {tol.max():.2e}")
    assert np.all(err <= tol), (err.max(), tol[np.argmax(err)])
    clear = np.abs(np.log(u) - la_o) > 2 * tol
    assert clear.mean() > 0.8
    np.testing.assert_array_equal(acc_g[clear], acc_o[clear])
    sel = clear & acc_o
    assert 0.05 < acc_o.mean() < 0.995 and (~acc_o[clear]).sum() >= 5   # accepts and rejects both checked
    np.testing.assert_allclose(th_g[sel], th_o[sel], rtol=1e-5, atol=1e-5)
    rej = clear & ~acc_o
    np.testing.assert_array_equal(th_g[rej], th[rej])
    np.testing.assert_allclose(ll_g[clear], ll_o[clear], rtol=rtol)
    # the drift moved the proposals: MALA and the random walk propose differently
    prop_rw = th + z @ np.linalg.cholesky(Sigma).T
    assert np.max(np.abs(th_g[sel] - prop_rw[sel])) > 1e-4
    s.close()


def test_mala_step_given_rejects_indefinite_sigma(cuda):
    from paper_1304_4333_b300 import Sps
    from paper_1304_4333_b300._native import SpsError
    X, y, beta = _data(2)
    s = Sps(X, y, 2, prior_sd=5.0)
    D = beta.shape[0]
    th = synthetic.particles_around(beta, 64, 0.2, seed=1)
    Sigma = -np.eye(D)
    with pytest.raises(SpsError) as e:
        s.mala_step_given(th, X.shape[0], Sigma, np.zeros((64, D)), np.full(64, 0.5))
    assert e.value.status == 4
    s.close()
