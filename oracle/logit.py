"""Multinomial-logit log-likelihood and gradient, plain FP64 (oracle; test infrastructure only).

Model, Sec. 2.1 Eq. (1): P(Y_t = c | x_t, theta) = exp(theta_c' x_t) / sum_i exp(theta_i' x_t),
normalised by theta_0 = 0 for the base outcome 0 (the normalisation the paper allows right after
Eq. (1); Sec. 3.1 uses the same normalised parameter vector of length k(C-1)).

The likelihood of y_{1:t} is the product over observations (Sec. 2.1, the product form of
p(y_{1:T} | theta)), so the log-likelihood is the sum over s <= t of log P(Y_s = y_s | x_s, theta).

Layout: X is [n, k] row-major; y is [n] with values 0..C-1; theta is [P, k(C-1)] class-major,
theta[p, (c-1)*k + i] the coefficient of covariate i for outcome c (c = 1..C-1).
"""
from __future__ import annotations

import numpy as np

# particles per batch so that [batch, t, C] FP64 arrays stay below ~256 MB
_MAX_ELEMS = 1 << 25


def _batches(P: int, t: int, C: int):
    b = max(1, _MAX_ELEMS // max(1, t * C))
    for lo in range(0, P, b):
        yield lo, min(P, lo + b)


def linear_predictors(X: np.ndarray, theta: np.ndarray, C: int) -> np.ndarray:
    """eta[p, s, c] = theta_c' x_s with eta[p, s, 0] = 0 (Eq. 1 with theta_0 = 0): [P, n, C]."""
    X = np.asarray(X, dtype=np.float64)
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    P, D = theta.shape
    n, k = X.shape
    assert D == k * (C - 1), "theta must have k*(C-1) columns"
    eta = np.zeros((P, n, C))
    for c in range(1, C):
        eta[:, :, c] = theta[:, (c - 1) * k:c * k] @ X.T
    return eta


def log_prob_terms(X: np.ndarray, y: np.ndarray, theta: np.ndarray, C: int) -> np.ndarray:
    """log P(Y_s = y_s | x_s, theta_p) for every particle and observation: [P, n].

    Eq. (1) in logarithms: eta_{y_s} - log sum_c exp(eta_c), the log-sum-exp evaluated as
    m + log sum_c exp(eta_c - m) with m = max_c eta_c so that no exponential overflows.
    """
    eta = linear_predictors(X, theta, C)
    m = eta.max(axis=2, keepdims=True)
    lse = m[:, :, 0] + np.log(np.exp(eta - m).sum(axis=2))
    yi = np.asarray(y, dtype=np.int64)
    obs = np.take_along_axis(eta, yi[None, :, None].repeat(eta.shape[0], axis=0), axis=2)[:, :, 0]
    return obs - lse


def loglik(X: np.ndarray, y: np.ndarray, theta: np.ndarray, C: int, t: int | None = None) -> np.ndarray:
    """ell_p(t) = sum_{s<=t} log P(Y_s = y_s | x_s, theta_p): [P] FP64 (Eq. 1, product form)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    t = n if t is None else int(t)
    assert 0 <= t <= n
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    out = np.zeros(theta.shape[0])
    if t == 0:
        return out
    for lo, hi in _batches(theta.shape[0], t, C):
        out[lo:hi] = log_prob_terms(X[:t], y[:t], theta[lo:hi], C).sum(axis=1)
    return out


def loglik_grad(X: np.ndarray, y: np.ndarray, theta: np.ndarray, C: int, t: int | None = None):
    """(ell [P], grad [P, k(C-1)]) with d ell / d theta_c = sum_{s<=t} (1[y_s = c] - p_{s,c}) x_s.

    The paper prints no gradient; this is the derivative of Eq. (1) summed over observations,
    p_{s,c} = P(Y_s = c | x_s, theta) for c = 1..C-1 (the base outcome has no parameters).
    """
    X = np.asarray(X, dtype=np.float64)
    n, k = X.shape
    t = n if t is None else int(t)
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    P, D = theta.shape
    ll = np.zeros(P)
    grad = np.zeros((P, D))
    if t == 0:
        return ll, grad
    Xt = X[:t]
    yt = np.asarray(y[:t], dtype=np.int64)
    onehot = np.zeros((t, C))
    onehot[np.arange(t), yt] = 1.0
    for lo, hi in _batches(P, t, C):
        eta = linear_predictors(Xt, theta[lo:hi], C)
        m = eta.max(axis=2, keepdims=True)
        e = np.exp(eta - m)
        z = e.sum(axis=2, keepdims=True)
        prob = e / z
        lse = m[:, :, 0] + np.log(z[:, :, 0])
        obs = (eta * onehot[None, :, :]).sum(axis=2)
        ll[lo:hi] = (obs - lse).sum(axis=1)
        resid = onehot[None, :, :] - prob
        for c in range(1, C):
            grad[lo:hi, (c - 1) * k:c * k] = resid[:, :, c] @ Xt
    return ll, grad
