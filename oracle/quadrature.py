"""Brute-force grid posteriors for one- and two-parameter logits (oracle; test infrastructure).

These pin the simulator's outputs (posterior mean, SD, log marginal likelihood) by a method that
shares nothing with it: the log-likelihood is evaluated through scipy's log_expit (binary) or the
closed form with outcome counts (intercept-only multinomial), and the posterior is integrated by
the trapezoid rule on a dense grid spanning +-10 posterior SDs around the mode.

log ML = log of the integral of p(y | theta) p(theta) with the normalised Gaussian prior, the
quantity whose estimate the simulator returns.
"""
from __future__ import annotations

import numpy as np
from scipy.special import log_expit, logsumexp


def _binary_loglik_grid(X: np.ndarray, y: np.ndarray, grid: np.ndarray) -> np.ndarray:
    """grid [G, k] -> [G] log-likelihood sum_s log sigma((2 y_s - 1) x_s' theta)."""
    sgn = 2.0 * np.asarray(y, dtype=np.float64) - 1.0
    out = np.empty(grid.shape[0])
    step = max(1, (1 << 22) // max(1, X.shape[0]))
    for lo in range(0, grid.shape[0], step):
        eta = grid[lo:lo + step] @ X.T
        out[lo:lo + step] = log_expit(eta * sgn[None, :]).sum(axis=1)
    return out


def _mnl_intercept_loglik_grid(counts: np.ndarray, grid: np.ndarray) -> np.ndarray:
    """Intercept-only multinomial logit, base outcome 0: sum_c n_c a_c - n log(1 + sum_c e^{a_c})."""
    n = counts.sum()
    full = np.concatenate([np.zeros((grid.shape[0], 1)), grid], axis=1)
    return full[:, 1:] @ counts[1:] - n * logsumexp(full, axis=1)


def _log_normal_pdf(grid: np.ndarray, mean: np.ndarray, cov: np.ndarray) -> np.ndarray:
    d = grid - mean[None, :]
    prec = np.linalg.inv(cov)
    _, logdet = np.linalg.slogdet(cov)
    D = mean.shape[0]
    return -0.5 * np.einsum("gi,ij,gj->g", d, prec, d) - 0.5 * (D * np.log(2 * np.pi) + logdet)


def _integrate(logpost: np.ndarray, axes, shape):
    """Trapezoid weights on a tensor grid; returns log integral and normalised weights."""
    logw = logpost.reshape(shape).copy()
    vol = 0.0
    for d, ax in enumerate(axes):
        h = ax[1] - ax[0]
        vol += np.log(h)
        edge = [slice(None)] * len(shape)
        edge[d] = 0
        logw[tuple(edge)] += np.log(0.5)
        edge[d] = -1
        logw[tuple(edge)] += np.log(0.5)
    lz = logsumexp(logw) + vol
    wn = np.exp(logw - logsumexp(logw)).reshape(-1)
    return lz, wn


def grid_posterior(loglik_fn, prior_mean, prior_cov, center, scale, points: int = 2001):
    """Posterior mean, SD and log ML on a grid center +- 10 scale (1 or 2 dimensions)."""
    center = np.asarray(center, dtype=np.float64)
    scale = np.asarray(scale, dtype=np.float64)
    D = center.shape[0]
    axes = [np.linspace(center[d] - 10 * scale[d], center[d] + 10 * scale[d], points) for d in range(D)]
    mesh = np.meshgrid(*axes, indexing="ij")
    grid = np.stack([m.reshape(-1) for m in mesh], axis=1)
    logpost = loglik_fn(grid) + _log_normal_pdf(grid, np.asarray(prior_mean, float), np.atleast_2d(prior_cov))
    lz, wn = _integrate(logpost, axes, tuple([points] * D))
    mean = wn @ grid
    sd = np.sqrt(wn @ (grid - mean[None, :]) ** 2)
    return {"mean": mean, "sd": sd, "log_ml": float(lz)}


def _laplace_center(loglik_fn, prior_mean, prior_cov, start, iters: int = 60):
    """Mode and curvature scale by Newton steps on finite-difference derivatives (grid placement)."""
    x = np.asarray(start, dtype=np.float64).copy()
    D = x.shape[0]
    prec = np.linalg.inv(np.atleast_2d(prior_cov))
    mu = np.asarray(prior_mean, float)

    def f(v):
        d = v - mu
        return float(loglik_fn(v[None, :])[0] - 0.5 * d @ prec @ d)

    h = 1e-4
    for _ in range(iters):
        g = np.zeros(D)
        H = np.zeros((D, D))
        f0 = f(x)
        for i in range(D):
            e = np.zeros(D); e[i] = h
            g[i] = (f(x + e) - f(x - e)) / (2 * h)
            H[i, i] = (f(x + e) - 2 * f0 + f(x - e)) / (h * h)
            for j in range(i):
                e2 = np.zeros(D); e2[j] = h
                H[i, j] = H[j, i] = (f(x + e + e2) - f(x + e - e2) - f(x - e + e2) + f(x - e - e2)) / (4 * h * h)
        step = np.linalg.solve(H, g)
        x = x - step
        if np.max(np.abs(step)) < 1e-10:
            break
    cov = np.linalg.inv(-H)
    return x, np.sqrt(np.diag(cov))


def binary_logit_posterior(X, y, prior_mean, prior_cov, points: int = 2001):
    """Grid posterior of a binary logit with k = 1 or 2 covariates (log_expit likelihood)."""
    X = np.asarray(X, dtype=np.float64)
    fn = lambda g: _binary_loglik_grid(X, y, g)  # noqa: E731
    c, s = _laplace_center(fn, prior_mean, prior_cov, np.zeros(X.shape[1]))
    return grid_posterior(fn, prior_mean, prior_cov, c, s, points)


def mnl_intercept_posterior(y, C: int, prior_mean, prior_cov, points: int = 1201):
    """Grid posterior of an intercept-only multinomial logit (C - 1 = 1 or 2 parameters)."""
    counts = np.bincount(np.asarray(y, dtype=np.int64), minlength=C).astype(np.float64)
    fn = lambda g: _mnl_intercept_loglik_grid(counts, g)  # noqa: E731
    c, s = _laplace_center(fn, prior_mean, prior_cov, np.zeros(C - 1))
    return grid_posterior(fn, prior_mean, prior_cov, c, s, points)
