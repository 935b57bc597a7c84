"""The five synthetic multinomial-logit workloads, generated from numpy PCG64 streams.

Each workload stands in for the shape class of the paper's applications (Sec. 3.2, Table 1:
hundreds of observations, k <= 42 covariates, C <= 4 outcomes) and scales it up. The real data
sets are not used. Recipes:

* c1 -- binary, n = 500, k = 5 (intercept + 4 iid N(0,1)), beta = (-0.5, 1, -1, 0.5, 0.25);
  J x N = 4 x 256.
* c2 -- binary, n = 20 000, k = 30: intercept, 19 columns AR(1) across columns with rho = 0.5
  (each N(0,1)), 10 Bernoulli(0.3) dummies; beta ~ N(0, 0.3^2); J x N = 16 x 4096.
* c3 -- C = 4 outcomes (base 0), n = 50 000, k = 50: intercept, 39 N(0,1), 10 Bernoulli(0.2);
  coefficients of outcomes 1..3 ~ N(0, 0.2^2); J x N = 32 x 2048.
* c4 -- binary, n = 1 000 000, k = 100: intercept, 69 equicorrelated N(0,1) (pairwise 0.2),
  30 Bernoulli(0.1); beta ~ N(0, 0.1^2); J x N = 64 x 1024.
* c5 -- C = 3, n = 100 000, 74 columns alternating N(0,1) (even index) and Bernoulli(0.25)
  (odd index), no intercept; true coefficients non-zero on the first 20 columns only,
  N(0, 0.3^2); 24 nested models use the first k_m = 5 + 3m columns (m = 0..23);
  J x N = 16 x 1024 per model.

Every workload has the prior N(0, 5^2 I) on all k(C-1) free coefficients.

Outcomes are drawn without evaluating any likelihood: a binary y is 1[x'beta + L > 0] with L
standard logistic, a multinomial y is argmax_c (x'beta_c + G_c) with G_c standard Gumbel and
beta_0 = 0 (the Gumbel-max construction). Both give P(Y = c | x) of the multinomial logit.

Parameter vectors are laid out class-major: theta[(c-1)*k + i] is the coefficient of covariate
i for outcome c, c = 1..C-1.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

CONFIG_NAMES = ("c1", "c2", "c3", "c4", "c5")


@dataclass
class Workload:
    name: str
    X: np.ndarray            # [n, k] float64, row-major
    y: np.ndarray            # [n] int32 in 0..C-1
    C: int                   # number of outcomes, base outcome 0
    theta_true: np.ndarray   # [k*(C-1)] float64, class-major
    J: int                   # particle groups
    N: int                   # particles per group
    prior_sd: float = 5.0
    model_k: Optional[List[int]] = None   # c5: nested covariate prefixes
    recipe: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def k(self) -> int:
        return int(self.X.shape[1])

    @property
    def D(self) -> int:
        return self.k * (self.C - 1)

    @property
    def P(self) -> int:
        return self.J * self.N


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, stream])))


def _draw_outcomes(X: np.ndarray, beta: np.ndarray, C: int, rng: np.random.Generator) -> np.ndarray:
    """beta: [C-1, k]. Latent-utility draw (logistic / Gumbel-max), no likelihood arithmetic."""
    n = X.shape[0]
    util = X @ beta.T                                  # [n, C-1]
    if C == 2:
        u = rng.random(n)
        u = np.clip(u, 1e-300, 1.0 - 1e-16)
        noise = np.log(u) - np.log1p(-u)              # standard logistic
        return (util[:, 0] + noise > 0.0).astype(np.int32)
    u = rng.random((n, C))
    u = np.clip(u, 1e-300, 1.0 - 1e-16)
    gumbel = -np.log(-np.log(u))
    full = np.concatenate([np.zeros((n, 1)), util], axis=1) + gumbel
    return np.argmax(full, axis=1).astype(np.int32)


def make_c1(seed: int = 0, n: int = 500) -> Workload:
    rng = _rng(seed, 1)
    X = np.empty((n, 5))
    X[:, 0] = 1.0
    X[:, 1:] = rng.standard_normal((n, 4))
    beta = np.array([-0.5, 1.0, -1.0, 0.5, 0.25])
    y = _draw_outcomes(X, beta[None, :], 2, rng)
    return Workload("c1", X, y, 2, beta.copy(), J=4, N=256,
                    recipe="binary logit n=500 k=5 intercept+4 iid N(0,1); beta fixed; prior N(0,25I)")


def make_c2(seed: int = 0, n: int = 20_000) -> Workload:
    rng = _rng(seed, 2)
    k = 30
    X = np.empty((n, k))
    X[:, 0] = 1.0
    rho = 0.5
    e = rng.standard_normal((n, 19))
    X[:, 1] = e[:, 0]
    for j in range(1, 19):
        X[:, 1 + j] = rho * X[:, j] + np.sqrt(1.0 - rho * rho) * e[:, j]
    X[:, 20:30] = (rng.random((n, 10)) < 0.3).astype(np.float64)
    beta = rng.normal(0.0, 0.3, size=k)
    y = _draw_outcomes(X, beta[None, :], 2, rng)
    return Workload("c2", X, y, 2, beta, J=16, N=4096,
                    recipe="binary logit n=20000 k=30: intercept, 19 AR(1) rho=0.5 N(0,1), "
                           "10 Bernoulli(0.3); beta~N(0,0.3^2); prior N(0,25I)")


def make_c3(seed: int = 0, n: int = 50_000) -> Workload:
    rng = _rng(seed, 3)
    k, C = 50, 4
    X = np.empty((n, k))
    X[:, 0] = 1.0
    X[:, 1:40] = rng.standard_normal((n, 39))
    X[:, 40:50] = (rng.random((n, 10)) < 0.2).astype(np.float64)
    beta = rng.normal(0.0, 0.2, size=(C - 1, k))
    y = _draw_outcomes(X, beta, C, rng)
    return Workload("c3", X, y, C, beta.reshape(-1), J=32, N=2048,
                    recipe="multinomial logit C=4 (base 0) n=50000 k=50: intercept, 39 N(0,1), "
                           "10 Bernoulli(0.2); coefficients~N(0,0.2^2); prior N(0,25I)")


def make_c4(seed: int = 0, n: int = 1_000_000) -> Workload:
    rng = _rng(seed, 4)
    k = 100
    X = np.empty((n, k))
    X[:, 0] = 1.0
    f = rng.standard_normal((n, 1))
    X[:, 1:70] = np.sqrt(0.2) * f + np.sqrt(0.8) * rng.standard_normal((n, 69))
    X[:, 70:100] = (rng.random((n, 30)) < 0.1).astype(np.float64)
    beta = rng.normal(0.0, 0.1, size=k)
    y = _draw_outcomes(X, beta[None, :], 2, rng)
    return Workload("c4", X, y, 2, beta, J=64, N=1024,
                    recipe="binary logit n=1e6 k=100: intercept, 69 equicorrelated(0.2) N(0,1), "
                           "30 Bernoulli(0.1); beta~N(0,0.1^2); prior N(0,25I)")


def make_c5(seed: int = 0, n: int = 100_000) -> Workload:
    rng = _rng(seed, 5)
    C, kmax = 3, 74
    X = np.empty((n, kmax))
    for j in range(kmax):
        if j % 2 == 0:
            X[:, j] = rng.standard_normal(n)
        else:
            X[:, j] = (rng.random(n) < 0.25).astype(np.float64)
    beta = np.zeros((C - 1, kmax))
    beta[:, :20] = rng.normal(0.0, 0.3, size=(C - 1, 20))
    y = _draw_outcomes(X, beta, C, rng)
    model_k = [5 + 3 * m for m in range(24)]
    return Workload("c5", X, y, C, beta.reshape(-1), J=16, N=1024, model_k=model_k,
                    recipe="24 nested multinomial logits C=3 n=1e5, k_m=5+3m of 74 columns alternating "
                           "N(0,1)/Bernoulli(0.25); true coefficients on the first 20 columns N(0,0.3^2)")


_MAKERS = {"c1": make_c1, "c2": make_c2, "c3": make_c3, "c4": make_c4, "c5": make_c5}


def make_workload(name: str, seed: int = 0, n: Optional[int] = None) -> Workload:
    maker = _MAKERS[name]
    return maker(seed) if n is None else maker(seed, n=n)


def particles_around(theta_center: np.ndarray, P: int, sd: float = 0.1, seed: int = 1) -> np.ndarray:
    """P particles theta_center + sd * z, z iid N(0, 1): [P, D] float64."""
    rng = _rng(seed, 101)
    D = theta_center.shape[0]
    return theta_center[None, :] + sd * rng.standard_normal((P, D))


def prior_draws(D: int, P: int, prior_sd: float = 5.0, seed: int = 1) -> np.ndarray:
    """P draws from the N(0, prior_sd^2 I) prior: [P, D] float64."""
    rng = _rng(seed, 102)
    return prior_sd * rng.standard_normal((P, D))


def uniforms(shape, seed: int = 1, stream: int = 103) -> np.ndarray:
    """FP64 uniforms on [0, 1) with 53 random bits each."""
    return _rng(seed, stream).random(shape)


def normals(shape, seed: int = 1, stream: int = 104) -> np.ndarray:
    return _rng(seed, stream).standard_normal(shape)
