"""Pins for the oracle's full simulator (Algorithms 1-3) against exact results and quadrature."""
import math

import numpy as np
import pytest

from oracle.logit import loglik
from oracle.quadrature import binary_logit_posterior, mnl_intercept_posterior
from oracle.smc import DegenerateError, GaussianPrior, cphase, sps_run


def _gen(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_zero_covariates_posterior_is_prior_and_log_ml_exact():
    # X = 0: every observation has probability 1/C whatever theta, so all weights are equal,
    # ESS never drops, there is one cycle, the posterior is the prior and log ML = -n log C.
    n, k, C, J, N = 60, 2, 3, 8, 256
    X = np.zeros((n, k))
    y = _gen(1).integers(0, C, n).astype(np.int32)
    prior = GaussianPrior.isotropic(k * (C - 1), 5.0)
    res = sps_run(X, y, C, prior, J, N, _gen(2))
    assert res.n_cycles == 1
    assert res.log_ml == pytest.approx(-n * math.log(C), abs=1e-9)
    assert np.all(np.abs(res.log_ml_groups + n * math.log(C)) < 1e-9)
    D = k * (C - 1)
    z = res.moments.mean[:D] / res.moments.nse[:D]
    assert np.all(np.abs(z) < 5.0)
    np.testing.assert_allclose(res.moments.sd[:D], 5.0, rtol=0.15)


def test_dogmatic_prior_one_cycle_and_log_ml_is_loglik_at_prior_mean():
    # Sec. 4.2: a dogmatic prior gives a uniform weight function and one cycle; the marginal
    # likelihood is then the likelihood at the prior mean.
    n, k, J, N = 120, 3, 4, 128
    g = _gen(3)
    X = np.concatenate([np.ones((n, 1)), g.standard_normal((n, k - 1))], axis=1)
    y = (g.random(n) < 0.4).astype(np.int32)
    mu = np.array([0.2, -0.5, 0.3])
    prior = GaussianPrior(mu, 1e-14 * np.eye(k))
    res = sps_run(X, y, 2, prior, J, N, _gen(4))
    assert res.n_cycles == 1
    assert res.log_ml == pytest.approx(loglik(X, y, mu[None], 2)[0], abs=1e-4)


def test_cphase_stops_at_first_ess_drop():
    # Two particles with opposite signs on one covariate: the weight ratio after s observations
    # with x = 1, y = 1 is ((1+e^-a)/(1+e^a))^s; check the stop index against ESS computed by hand.
    a = 2.0
    theta = np.array([[a], [-a]])
    X = np.ones((10, 1))
    y = np.ones(10, np.int32)
    t, logw, e = cphase(X, y, 2, theta, 0, J=1, N=2, ess_fraction=0.9)
    r = (1 + math.exp(-a)) / (1 + math.exp(a))   # w_2 / w_1 per observation
    want = None
    for s in range(1, 11):
        q = r ** s
        if (1 + q) ** 2 / (1 + q * q) / 2 < 0.9:
            want = s
            break
    assert t == want


def _compare_to_quadrature(res, quad, D, tol_sd=4.0):
    nse = res.moments.nse[:D]
    z_mean = (res.moments.mean[:D] - quad["mean"]) / nse
    assert np.all(np.abs(z_mean) < tol_sd), (res.moments.mean[:D], quad["mean"], nse)
    np.testing.assert_allclose(res.moments.sd[:D], quad["sd"], rtol=0.08)
    z_ml = (res.log_ml - quad["log_ml"]) / max(res.log_ml_nse, 1e-3)
    assert abs(z_ml) < tol_sd, (res.log_ml, quad["log_ml"], res.log_ml_nse)


def test_binary_intercept_only_against_quadrature():
    n = 150
    y = (_gen(5).random(n) < 0.3).astype(np.int32)
    X = np.ones((n, 1))
    prior = GaussianPrior.isotropic(1, 5.0)
    quad = binary_logit_posterior(X, y, prior.mean, prior.cov)
    res = sps_run(X, y, 2, prior, 10, 512, _gen(6))
    _compare_to_quadrature(res, quad, 1)


def test_binary_intercept_and_slope_against_quadrature():
    n = 200
    g = _gen(7)
    X = np.concatenate([np.ones((n, 1)), g.standard_normal((n, 1))], axis=1)
    eta = -0.4 + 1.2 * X[:, 1]
    y = (g.random(n) < 1 / (1 + np.exp(-eta))).astype(np.int32)
    prior = GaussianPrior.isotropic(2, 5.0)
    quad = binary_logit_posterior(X, y, prior.mean, prior.cov, points=801)
    res = sps_run(X, y, 2, prior, 10, 512, _gen(8))
    _compare_to_quadrature(res, quad, 2)


def test_three_outcome_intercept_only_against_quadrature():
    n = 180
    y = _gen(9).choice(3, size=n, p=[0.5, 0.3, 0.2]).astype(np.int32)
    X = np.ones((n, 1))
    prior = GaussianPrior.isotropic(2, 5.0)
    quad = mnl_intercept_posterior(y, 3, prior.mean, prior.cov, points=801)
    res = sps_run(X, y, 3, prior, 10, 512, _gen(10))
    _compare_to_quadrature(res, quad, 2)


def test_two_pass_replay_follows_schedule():
    # Algorithm 3: pass 2 replays t_l, R_l and Sigma_lr of pass 1; its results agree within NSE.
    n = 120
    g = _gen(11)
    X = np.concatenate([np.ones((n, 1)), g.standard_normal((n, 1))], axis=1)
    y = (g.random(n) < 0.5).astype(np.int32)
    prior = GaussianPrior.isotropic(2, 5.0)
    p1 = sps_run(X, y, 2, prior, 8, 256, _gen(12))
    p2 = sps_run(X, y, 2, prior, 8, 256, _gen(13), schedule=p1.cycles)
    assert [c.t for c in p2.cycles] == [c.t for c in p1.cycles]
    assert [c.R for c in p2.cycles] == [c.R for c in p1.cycles]
    for c1, c2 in zip(p1.cycles, p2.cycles):
        for s1, s2 in zip(c1.sigmas, c2.sigmas):
            np.testing.assert_array_equal(s1, s2)
    comb = math.hypot(p1.log_ml_nse, p2.log_ml_nse)
    assert abs(p1.log_ml - p2.log_ml) < 5 * max(comb, 1e-3)


def test_degenerate_proposal_raises():
    # A covariance of rank < D (all particles identical) cannot be factored: step 2(c)i fails.
    from oracle.smc import rw_step
    X = np.ones((5, 2)); y = np.ones(5, np.int32)
    theta = np.ones((8, 2))
    prior = GaussianPrior.isotropic(2, 5.0)
    with pytest.raises(DegenerateError):
        rw_step(X, y, 2, 5, theta, np.zeros(8), prior, np.zeros((2, 2)), np.zeros((8, 2)), np.full(8, 0.5))
