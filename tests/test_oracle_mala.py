"""Pins for the oracle's MALA step and its pooled particle covariance (Algorithm 2 step 2(c)i).

The MALA step is pinned by a one-dimensional case computed by hand, by the antisymmetry of the
Metropolis-Hastings log ratio (the reverse move has log ratio -log alpha, which fails for a
dropped or sign-flipped proposal-density term or a wrong reverse mean), by its reduction to the
random walk when the log posterior is flat, and by the invariance of a Gaussian target under
large steps (an unadjusted Langevin step of this size inflates the variance by 60 %).
The covariance is pinned by hand-computed cases whose divisor (J N - 1) and orientation show.
"""
import numpy as np
import pytest

from oracle.logit import loglik
from oracle.smc import GaussianPrior, mala_step, particle_covariance, rw_step


def _zero_data(n, k, C):
    return np.zeros((n, k)), np.zeros(n, dtype=np.int32)


def test_mala_one_dimensional_hand_value():
    # X = 0: ell is constant and its gradient zero; prior N(0, 4); theta = 1, Sigma = 1, z = 0.5.
    # g(1) = -1/4, theta' = 1 - 1/8 + 1/2 = 1.375; log p(theta') - log p(theta) = -0.111328125;
    # log q(theta'|theta) = -0.125; g(theta') = -0.34375, reverse residual -0.203125,
    # log q(theta|theta') = -0.0206298828125; log alpha = -0.0069580078125 (all exact in binary)
    X, y = _zero_data(7, 1, 2)
    prior = GaussianPrior(np.zeros(1), np.array([[4.0]]))
    th = np.array([[1.0]])
    ll = loglik(X, y, th, 2, 7)
    out, ll2, acc, la = mala_step(X, y, 2, 7, th, ll, prior, np.array([[1.0]]), np.array([[0.5]]),
                                  np.array([0.5]))
    assert la[0] == pytest.approx(-0.0069580078125, abs=1e-15)
    assert acc[0] and out[0, 0] == pytest.approx(1.375, abs=1e-15)
    assert ll2[0] == pytest.approx(-7 * np.log(2.0), abs=1e-12)
    # u above alpha: rejected, state unchanged
    out, _, acc, _ = mala_step(X, y, 2, 7, th, ll, prior, np.array([[1.0]]), np.array([[0.5]]),
                               np.array([0.9999]))
    assert not acc[0] and out[0, 0] == 1.0


def test_mala_log_ratio_is_antisymmetric(rng):
    # forward move theta -> theta' with z; the reverse move theta' -> theta needs
    # z_rev = L^-1 (theta - theta' - Sigma g(theta') / 2), and its log ratio is -log alpha
    n, k, C = 60, 3, 3
    X = rng.standard_normal((n, k)); X[:, 0] = 1.0
    y = rng.integers(0, C, n).astype(np.int32)
    D = k * (C - 1)
    A = rng.standard_normal((D, D))
    prior = GaussianPrior(0.3 * rng.standard_normal(D), A @ A.T / D + np.eye(D))
    B = rng.standard_normal((D, D))
    Sigma = 0.02 * (B @ B.T / D + np.eye(D))
    L = np.linalg.cholesky(Sigma)
    th = 0.4 * rng.standard_normal((5, D))
    z = rng.standard_normal((5, D))
    ll = loglik(X, y, th, C, n)
    u = np.full(5, 1e-300)                       # accept everything
    prop, ll_p, acc, la = mala_step(X, y, C, n, th, ll, prior, Sigma, z, u)
    assert acc.all()
    from oracle.logit import loglik_grad
    _, gl = loglik_grad(X, y, prop, C, n)
    g_prop = gl - (prop - prior.mean[None, :]) @ prior.prec.T
    z_rev = np.linalg.solve(L, (th - prop - 0.5 * g_prop @ Sigma.T).T).T
    back, _, _, la_rev = mala_step(X, y, C, n, prop, ll_p, prior, Sigma, z_rev, u)
    np.testing.assert_allclose(back, th, rtol=0, atol=1e-12)
    np.testing.assert_allclose(la_rev, -la, rtol=0, atol=1e-9)
    assert np.max(np.abs(la)) > 0.05             # a ratio far from zero, so the check means something


def test_mala_reduces_to_random_walk_when_posterior_is_flat(rng):
    # X = 0 and a prior of variance 1e12: the drift Sigma g / 2 and the proposal-density ratio
    # vanish, so MALA takes the random walk's steps and decisions
    n, k, C = 10, 2, 3
    X, y = _zero_data(n, k, C)
    D = k * (C - 1)
    prior = GaussianPrior(np.zeros(D), 1e12 * np.eye(D))
    Sigma = np.diag([0.5, 1.0, 2.0, 0.25])
    th = rng.standard_normal((50, D))
    z = rng.standard_normal((50, D))
    u = rng.random(50)
    ll = loglik(X, y, th, C, n)
    a, la_, acc_a, lal = mala_step(X, y, C, n, th, ll, prior, Sigma, z, u)
    b, lb_, acc_b = rw_step(X, y, C, n, th, ll, prior, Sigma, z, u)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-9)
    assert np.array_equal(acc_a, acc_b)
    assert np.max(np.abs(lal)) < 1e-9


def test_mala_leaves_a_gaussian_target_invariant(rng):
    # X = 0, prior N(0, I) in two dimensions, particles drawn from it, 60 steps of size
    # Sigma = 1.5 I: the variance stays 1 (an unadjusted Langevin step of this size would drift to
    # 1.6; MC error of the variance of 20 000 draws is about 0.01)
    n, k, C = 5, 2, 2
    X, y = _zero_data(n, k, C)
    prior = GaussianPrior(np.zeros(2), np.eye(2))
    P = 20000
    th = rng.standard_normal((P, 2))
    ll = loglik(X, y, th, C, n)
    Sigma = 1.5 * np.eye(2)
    acc_rate = []
    for _ in range(60):
        th, ll, acc, _ = mala_step(X, y, C, n, th, ll, prior, Sigma, rng.standard_normal((P, 2)), rng.random(P))
        acc_rate.append(acc.mean())
    assert np.all(np.abs(th.mean(axis=0)) < 0.04)
    assert np.all(np.abs(th.var(axis=0) - 1.0) < 0.05)
    assert 0.3 < np.mean(acc_rate) < 0.99


def test_particle_covariance_hand_values():
    # three particles in two dimensions: mean (2, 3); deviations (-1,-1), (1,2), (0,-1);
    # sum of outer products [[2, 3], [3, 6]] divided by J N - 1 = 2
    th = np.array([[1.0, 2.0], [3.0, 5.0], [2.0, 2.0]])
    V = particle_covariance(th)
    np.testing.assert_array_equal(V, np.array([[1.0, 1.5], [1.5, 3.0]]))
    # one coordinate: 0, 2, 4, 6 about 3 -> 20 / 3
    V1 = particle_covariance(np.array([[0.0], [2.0], [4.0], [6.0]]))
    assert V1.shape == (1, 1) and V1[0, 0] == pytest.approx(20.0 / 3.0, rel=1e-15)
