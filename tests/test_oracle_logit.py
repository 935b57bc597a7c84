"""Pins for the oracle's log-likelihood and gradient (Eq. 1) against closed forms and library
routines -- nothing here re-types the oracle's own formula."""
import math

import numpy as np
import pytest
from scipy.special import log_expit

from oracle.logit import loglik, loglik_grad, log_prob_terms


@pytest.mark.parametrize("C", [2, 3, 4])
def test_theta_zero_gives_uniform_probabilities(C, rng):
    # theta = 0: every outcome has probability 1/C, so ell(t) = -t log C exactly (Eq. 1).
    n, k = 37, 5
    X = rng.standard_normal((n, k))
    y = rng.integers(0, C, n).astype(np.int32)
    th = np.zeros((3, k * (C - 1)))
    for t in (0, 1, 17, n):
        np.testing.assert_allclose(loglik(X, y, th, C, t), -t * math.log(C), rtol=0, atol=1e-12)


@pytest.mark.parametrize("C", [2, 4])
def test_zero_covariates_give_uniform_probabilities(C, rng):
    n, k = 29, 4
    X = np.zeros((n, k))
    y = rng.integers(0, C, n).astype(np.int32)
    th = rng.standard_normal((5, k * (C - 1))) * 3
    np.testing.assert_allclose(loglik(X, y, th, C), -n * math.log(C), rtol=0, atol=1e-12)


def test_binary_single_observation_rational():
    # x = 1, theta = ln 3: P(Y=1) = 3/4, P(Y=0) = 1/4.
    X = np.ones((1, 1))
    th = np.array([[math.log(3.0)]])
    assert loglik(X, np.array([1], np.int32), th, 2)[0] == pytest.approx(math.log(0.75), abs=1e-15)
    assert loglik(X, np.array([0], np.int32), th, 2)[0] == pytest.approx(math.log(0.25), abs=1e-15)


def test_multinomial_single_observation_rational():
    # C = 3, x = 1, theta_1 = ln 2, theta_2 = ln 3: probabilities (1, 2, 3)/6 for outcomes 0, 1, 2.
    X = np.ones((1, 1))
    th = np.array([[math.log(2.0), math.log(3.0)]])
    for c in range(3):
        v = loglik(X, np.array([c], np.int32), th, 3)[0]
        assert v == pytest.approx(math.log((c + 1) / 6.0), abs=1e-15)


def test_class_major_layout():
    # k = 2, C = 3: theta = [theta_1 | theta_2]; x = (1, 0) selects the first entry of each block.
    th = np.array([[math.log(2.0), 7.0, math.log(5.0), -3.0]])
    X = np.array([[1.0, 0.0], [0.0, 1.0]])
    y = np.array([2, 1], np.int32)
    # obs 0: utilities (0, ln2, ln5) -> P(2) = 5/8; obs 1: (0, 7, -3) -> P(1) = e^7/(1+e^7+e^-3)
    want = math.log(5 / 8) + (7.0 - math.log(1 + math.exp(7.0) + math.exp(-3.0)))
    assert loglik(X, y, th, 3)[0] == pytest.approx(want, abs=1e-13)


def test_binary_matches_scipy_log_expit(rng):
    n, k, P = 300, 6, 9
    X = rng.standard_normal((n, k))
    y = rng.integers(0, 2, n).astype(np.int32)
    th = rng.standard_normal((P, k)) * 2
    want = log_expit((th @ X.T) * (2.0 * y - 1.0)[None, :]).sum(axis=1)
    np.testing.assert_allclose(loglik(X, y, th, 2), want, rtol=1e-13, atol=1e-11)


def test_binary_label_flip_symmetry(rng):
    n, k = 80, 3
    X = rng.standard_normal((n, k))
    y = rng.integers(0, 2, n).astype(np.int32)
    th = rng.standard_normal((4, k))
    np.testing.assert_allclose(loglik(X, y, th, 2), loglik(X, 1 - y, -th, 2), rtol=1e-13)


def test_multinomial_relabelling_symmetry(rng):
    # Swapping outcomes 1 and 2 in y together with their parameter blocks leaves ell unchanged.
    n, k, C = 60, 4, 3
    X = rng.standard_normal((n, k))
    y = rng.integers(0, C, n).astype(np.int32)
    th = rng.standard_normal((3, k * 2))
    y2 = y.copy(); y2[y == 1] = 2; y2[y == 2] = 1
    th2 = np.concatenate([th[:, k:], th[:, :k]], axis=1)
    np.testing.assert_allclose(loglik(X, y, th, C), loglik(X, y2, th2, C), rtol=1e-13)


def test_three_outcomes_with_a_dead_outcome_reduce_to_binary(rng):
    # C = 3 with eta_2 = -800 (intercept column, coefficient -800): outcome 2 has probability
    # e^-800, so on y in {0, 1} the model is the binary logit of outcome 1 against 0.
    n, k = 50, 3
    X = rng.standard_normal((n, k))
    X[:, 0] = 1.0
    y = rng.integers(0, 2, n).astype(np.int32)
    th = rng.standard_normal((2, k))
    dead = np.zeros((2, k)); dead[:, 0] = -800.0
    ll3 = loglik(X, y, np.concatenate([th, dead], axis=1), 3)
    want = log_expit((th @ X.T) * (2.0 * y - 1.0)[None, :]).sum(axis=1)
    np.testing.assert_allclose(ll3, want, rtol=1e-13)


def test_extreme_linear_predictor_is_finite_and_exact():
    X = np.ones((1, 1))
    th = np.array([[800.0], [-800.0]])
    v0 = loglik(X, np.array([0], np.int32), th, 2)
    v1 = loglik(X, np.array([1], np.int32), th, 2)
    assert np.all(np.isfinite(v0)) and np.all(np.isfinite(v1))
    assert v0[0] == -800.0 and v1[0] == 0.0
    assert v0[1] == 0.0 and v1[1] == -800.0


def test_terms_sum_to_loglik(rng):
    n, k, C = 40, 3, 3
    X = rng.standard_normal((n, k))
    y = rng.integers(0, C, n).astype(np.int32)
    th = rng.standard_normal((4, k * (C - 1)))
    terms = log_prob_terms(X, y, th, C)
    assert np.all(terms <= 0)
    # each term is a log probability: the C probabilities of one observation sum to one
    tot = np.zeros((4, n))
    for c in range(C):
        tot += np.exp(log_prob_terms(X, np.full(n, c, np.int32), th, C))
    np.testing.assert_allclose(tot, 1.0, atol=1e-14)


@pytest.mark.parametrize("C", [2, 3])
def test_gradient_central_differences(C, rng):
    n, k = 70, 4
    X = rng.standard_normal((n, k))
    y = rng.integers(0, C, n).astype(np.int32)
    th = rng.standard_normal((2, k * (C - 1)))
    ll, g = loglik_grad(X, y, th, C, 50)
    np.testing.assert_allclose(ll, loglik(X, y, th, C, 50), rtol=1e-13)
    for p in range(2):
        fd = np.zeros(k * (C - 1))
        for i in range(k * (C - 1)):
            h = 1e-5 * max(1.0, abs(th[p, i]))
            e = np.zeros_like(th[p]); e[i] = h
            fd[i] = (loglik(X, y, (th[p] + e)[None], C, 50)[0] - loglik(X, y, (th[p] - e)[None], C, 50)[0]) / (2 * h)
        assert np.max(np.abs(g[p] - fd)) / np.max(np.abs(fd)) < 1e-7


@pytest.mark.parametrize("C", [2, 4])
def test_gradient_closed_form_at_zero(C, rng):
    # theta = 0: p_{s,c} = 1/C, so d ell / d theta_c = sum_s (1[y_s = c] - 1/C) x_s.
    n, k = 45, 3
    X = rng.standard_normal((n, k))
    y = rng.integers(0, C, n).astype(np.int32)
    _, g = loglik_grad(X, y, np.zeros((1, k * (C - 1))), C)
    for c in range(1, C):
        want = ((y == c).astype(float) - 1.0 / C) @ X
        np.testing.assert_allclose(g[0, (c - 1) * k:c * k], want, rtol=1e-12, atol=1e-12)
