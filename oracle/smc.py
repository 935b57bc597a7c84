"""Plain FP64 sequential posterior simulator (oracle; test infrastructure only).

Follows Sec. 2 of the paper step by step:

* group means, grand mean, v-hat, NSE and RNE: Eqs. (3), (5), (6), (7), (10);
* the non-adaptive simulator's C, S and M phases: Algorithm 1, Eqs. (11)-(13);
* the adaptive simulator: Algorithm 2 (ESS rule Eq. (14), random-walk Metropolis M phase with
  Sigma = h * V, the +-0.01 step-size rule and the RNE stopping rule);
* the second pass of the two-pass simulator (Algorithm 3): a replay of a recorded schedule
  {t_l, R_l, Sigma_lr}.

Readings taken where the paper is silent or garbled (each also listed in the design notes):

* NSE (Eq. 7) is read as (v-hat / (J N))^(1/2); the printed (v-hat / J)^(1/2) does not match the
  CLT scaling of Eq. (2) nor the paper's own Table 5 figures.
* log marginal likelihood: per group, the sum over cycles of log N^-1 sum_n w_jn (the paper
  defers the estimator to another paper). Reported as the mean over groups with
  NSE = sd_j / sqrt(J); the log of the mean of the group likelihoods is also returned.
* RNE stopping rule: the monitoring set is {ell(theta; y_{1:t}), theta_c' xbar (c = 1..C-1)},
  xbar the covariate mean over all T observations; the M phase stops when the smallest RNE
  in the set reaches K, or after r_max steps.
* V is the pooled sample covariance of all J N particles with divisor J N - 1.
* "a_lr > 0.25" in Algorithm 2 is the acceptance rate alpha_lr (strict inequality).
* The S phase also runs at the end of the last cycle (s = T), then the final M phase uses K = 0.9.
* Multinomial resampling uses an integer CDF: q_n = floor(w_n 2^40) from weights normalised by
  their maximum, tau = min(floor(u Q), Q - 1), index = first n with cumulative q > tau.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .logit import log_prob_terms, loglik, loglik_grad


class DegenerateError(RuntimeError):
    """The proposal covariance h V is not positive definite (Sec. 4.2: a very diffuse prior
    leaves one unique particle per group, rank V < dim theta, and Algorithm 2 step 2(c)i fails)."""


# ----------------------------------------------------------------------------- prior

@dataclass
class GaussianPrior:
    """theta ~ N(mean, cov) on the normalised parameter vector (Eq. 16 with theta_0 = 0)."""
    mean: np.ndarray
    cov: np.ndarray

    def __post_init__(self):
        self.mean = np.asarray(self.mean, dtype=np.float64).reshape(-1)
        self.cov = np.atleast_2d(np.asarray(self.cov, dtype=np.float64))
        self.chol = np.linalg.cholesky(self.cov)
        self.prec = np.linalg.inv(self.cov)

    @staticmethod
    def isotropic(D: int, sd: float) -> "GaussianPrior":
        return GaussianPrior(np.zeros(D), (sd * sd) * np.eye(D))

    @property
    def D(self) -> int:
        return self.mean.shape[0]

    def log_kernel(self, theta: np.ndarray) -> np.ndarray:
        """-1/2 (theta - mu)' cov^-1 (theta - mu), the prior log density up to its constant."""
        d = np.atleast_2d(theta) - self.mean[None, :]
        return -0.5 * np.einsum("pi,ij,pj->p", d, self.prec, d)

    def sample(self, rng: np.random.Generator, P: int) -> np.ndarray:
        return self.mean[None, :] + rng.standard_normal((P, self.D)) @ self.chol.T


def normalise_prior(mu: np.ndarray, Sigma: np.ndarray):
    """Prior of the normalised parameters from independent class priors (Sec. 3.1, Eq. 17).

    mu: [C, k], Sigma: [C, k, k] for theta_c ~ N(mu_c, Sigma_c), c = 0..C-1 independent. With
    outcome 0 as the base (theta_j replaced by theta_j - theta_0, j = 1..C-1) the D = k (C-1)
    vector is Gaussian with block mean mu_j - mu_0, diagonal blocks Sigma_j + Sigma_0 and
    off-diagonal blocks Sigma_0. Returns (mean [D], cov [D, D]).
    """
    mu = np.asarray(mu, dtype=np.float64)
    Sigma = np.asarray(Sigma, dtype=np.float64)
    C, k = mu.shape
    mean = np.concatenate([mu[j] - mu[0] for j in range(1, C)])
    cov = np.zeros((k * (C - 1), k * (C - 1)))
    for a in range(1, C):
        for b in range(1, C):
            blk = Sigma[0].copy()
            if a == b:
                blk = blk + Sigma[a]
            cov[(a - 1) * k:a * k, (b - 1) * k:b * k] = blk
    return mean, cov


def gprior_covariance(X: np.ndarray, C: int, g: float):
    """Zellner's g-prior of the paper (Sec. 3.1, Eq. 18): mu_c = 0 and Sigma_c = g T (X'X)^-1 for
    every outcome, then normalised on outcome 0 (normalise_prior). Returns (mean, cov)."""
    X = np.asarray(X, dtype=np.float64)
    T, k = X.shape
    S = g * T * np.linalg.inv(X.T @ X)
    return normalise_prior(np.zeros((C, k)), np.broadcast_to(S, (C, k, k)))


# ----------------------------------------------------------------------------- statistics

def ess(logw: np.ndarray) -> float:
    """Eq. (14): ESS = (sum w)^2 / sum w^2 over all J N particles, from log weights.

    Weights are scaled by exp(-max log w), which cancels in the ratio.
    """
    lw = np.asarray(logw, dtype=np.float64).reshape(-1)
    w = np.exp(lw - lw.max())
    return float(w.sum() ** 2 / (w * w).sum())


def log_mean_exp(logw: np.ndarray) -> float:
    """log( N^-1 sum_n exp(logw_n) ), evaluated as m + log(mean(exp(logw - m)))."""
    lw = np.asarray(logw, dtype=np.float64).reshape(-1)
    m = lw.max()
    return float(m + np.log(np.mean(np.exp(lw - m))))


@dataclass
class GroupMoments:
    mean: np.ndarray   # grand mean, Eq. (5)
    sd: np.ndarray     # pooled posterior SD, sqrt((JN)^-1 sum sum (g - gbar)^2)
    vhat: np.ndarray   # Eq. (6)
    nse: np.ndarray    # Eq. (7), read as sqrt(vhat / (J N))
    rne: np.ndarray    # Eq. (10)
    group_means: np.ndarray  # Eq. (3), [J, m]


def group_moments(g: np.ndarray, J: int, N: int) -> GroupMoments:
    """Moments of monitoring values g [J*N, m] (particles ordered group-major).

    Eq. (3) group means, Eq. (5) grand mean, Eq. (6) v-hat = N/(J-1) sum_j (gbar_j - gbar)^2,
    Eq. (10) RNE = (JN)^-1 sum_j sum_n (g_jn - gbar)^2 / v-hat, NSE = (v-hat/(JN))^(1/2).
    """
    g = np.asarray(g, dtype=np.float64)
    if g.ndim == 1:
        g = g[:, None]
    gj = g.reshape(J, N, -1)
    gbar_j = gj.mean(axis=1)                       # Eq. (3)
    gbar = gbar_j.mean(axis=0)                     # Eq. (5)
    vhat = (N / (J - 1.0)) * ((gbar_j - gbar[None, :]) ** 2).sum(axis=0)   # Eq. (6)
    var = ((gj - gbar[None, None, :]) ** 2).sum(axis=(0, 1)) / (J * N)
    with np.errstate(divide="ignore", invalid="ignore"):
        rne = np.where(vhat > 0, var / vhat, np.inf)   # Eq. (10)
    nse = np.sqrt(vhat / (J * N))
    return GroupMoments(gbar, np.sqrt(var), vhat, nse, rne, gbar_j)


# ----------------------------------------------------------------------------- S phase

WEIGHT_BITS = 40


def resample_multinomial(w: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Multinomial resampling of one group (Algorithm 1, S phase) by an integer CDF.

    w: [N] non-negative FP64 weights with max(w) = 1 (weights divided by their maximum);
    u: [M] FP64 uniforms on [0, 1). Returns [M] int32 indices.

    q_n = floor(w_n * 2^40) (exact in FP64: w_n * 2^40 is a power-of-two scaling), c = cumulative
    sum of q in uint64, Q = c_N <= N 2^40. For each u_i: tau = min(floor(u_i * Q), Q - 1) (one
    correctly rounded FP64 product), index = the first n with c_n > tau. Each draw selects n with
    probability q_n / Q, which equals w_n / sum w up to the 2^-40 quantisation.
    """
    w = np.asarray(w, dtype=np.float64)
    q = np.floor(np.ldexp(w, WEIGHT_BITS)).astype(np.uint64)
    c = np.cumsum(q, dtype=np.uint64)
    Q = c[-1]
    if Q == 0:
        raise DegenerateError("all resampling weights quantise to zero")
    tau = np.floor(np.asarray(u, dtype=np.float64) * np.float64(Q)).astype(np.uint64)
    tau = np.minimum(tau, Q - np.uint64(1))
    return np.searchsorted(c, tau, side="right").astype(np.int32)


RESIDUAL_SHIFT = 12


def resample_residual(w: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Residual resampling of one group (the alternative to multinomial resampling that the S
    phase allows, Sec. 2.2; Chopin's condition holds for it), in integers.

    w: [N] weights with max(w) = 1; u: [N] FP64 uniforms on [0, 1), of which the first R are
    used. q_n = floor(w_n 2^40), Q = sum q. Particle n gets c_n = floor(N q_n / Q) copies
    (exact: N q_n < 2^64), placed first in particle order; the remaining R = N - sum c draws are
    multinomial on the residuals r_n = (N q_n mod Q) >> 12 (so that sum r < 2^52 stays exact in
    FP64), by the integer CDF of resample_multinomial: tau = min(floor(u_i sum r), sum r - 1),
    index = first n with cumulative r > tau. Returns [N] int32 indices.
    """
    w = np.asarray(w, dtype=np.float64)
    N = w.shape[0]
    q = [int(v) for v in np.floor(np.ldexp(w, WEIGHT_BITS))]
    Q = sum(q)
    if Q == 0:
        raise DegenerateError("all resampling weights quantise to zero")
    counts = [(N * qn) // Q for qn in q]
    resid = [((N * qn) % Q) >> RESIDUAL_SHIFT for qn in q]
    out = []
    for n, c in enumerate(counts):
        out.extend([n] * c)
    R = N - len(out)
    if R > 0:
        cr = np.cumsum(np.array(resid, dtype=np.uint64), dtype=np.uint64)
        S = cr[-1]
        tau = np.floor(np.asarray(u[:R], dtype=np.float64) * np.float64(S)).astype(np.uint64)
        tau = np.minimum(tau, S - np.uint64(1))
        out.extend(np.searchsorted(cr, tau, side="right").tolist())
    return np.array(out, dtype=np.int32)


def normalised_weights(logw: np.ndarray) -> np.ndarray:
    """exp(logw - max logw) for one group."""
    lw = np.asarray(logw, dtype=np.float64)
    return np.exp(lw - lw.max())


# ----------------------------------------------------------------------------- options / records

@dataclass
class SpsOptions:
    """The constants of Algorithm 2 that the paper calls hard-wired but user-changeable (Sec. 2.3)."""
    ess_fraction: float = 0.5      # step 1(b): ESS/(J N) < 0.5 ends the C phase
    h_init: float = 0.5            # step 2(a)ii: h_11 = 0.5
    h_step: float = 0.01           # step 2(c)ii: +- 0.01
    h_min: float = 0.1
    h_max: float = 1.0
    target_accept: float = 0.25    # step 2(c)ii: alpha_lr > 0.25
    rne_cycle: float = 0.35        # step 2(b)i: K = 0.35 if s < T
    rne_final: float = 0.9         # step 2(b)ii: K = 0.9 if s = T
    r_max: int = 200               # cap on M steps per cycle (not in the paper)
    resampling: str = "multinomial"   # or "residual" (S phase, Sec. 2.2)


@dataclass
class CycleRecord:
    t: int                      # t_l
    R: int = 0                  # R_l, M steps taken
    sigmas: List[np.ndarray] = field(default_factory=list)   # Sigma_lr = h_lr V_lr, r = 1..R_l
    hs: List[float] = field(default_factory=list)
    accept: List[float] = field(default_factory=list)
    rne_min: List[float] = field(default_factory=list)
    ess_end: float = 0.0
    logml_inc: Optional[np.ndarray] = None   # [J]
    log_pred: Optional[np.ndarray] = None    # [t_l - t_{l-1}, J] per-observation log predictive


@dataclass
class SpsResult:
    theta: np.ndarray           # [J*N, D] final particles
    ll: np.ndarray              # [J*N] log-likelihood at T
    moments: GroupMoments       # of theta coordinates then log-odds theta_c' xbar
    log_ml: float               # mean over groups of log ML_j
    log_ml_nse: float           # sd_j / sqrt(J)
    log_ml_groups: np.ndarray   # [J]
    log_ml_pooled: float        # log of the mean of ML_j over groups
    cycles: List[CycleRecord]
    log_pred_groups: Optional[np.ndarray] = None   # [T, J] log p(y_s | y_1:s-1) per group
    log_pred: Optional[np.ndarray] = None          # [T] mean over groups
    log_pred_nse: Optional[np.ndarray] = None      # [T] sd over groups / sqrt(J)

    @property
    def n_cycles(self) -> int:
        return len(self.cycles)

    @property
    def m_steps(self) -> int:
        return int(sum(c.R for c in self.cycles))


# ----------------------------------------------------------------------------- phases

def cphase(X, y, C, theta, t0: int, J: int, N: int, ess_fraction: float = 0.5,
           t_fixed: Optional[int] = None, log_pred: Optional[list] = None):
    """C phase (Algorithm 1 step 2(a), Eq. 11; end rule Algorithm 2 step 1, Eq. 14).

    Starting from w_jn(t0) = 1, multiply in p(y_s | theta_jn) for s = t0+1, t0+2, ... and stop at
    the first s with ESS(s)/(J N) < ess_fraction, or at s = T. With t_fixed given (a recorded
    schedule), stop at s = t_fixed instead. Returns (t_new, logw [J*N], ess at t_new).

    With a list given as log_pred, appends for each s the [J] log predictive likelihoods
    log p(y_s | y_1:s-1) of the groups (Sec. 6 calls them a by-product of SPS):
    log sum_n w_jn(s) - log sum_n w_jn(s-1), the weighted mean of p(y_s | theta_jn) under the
    weights before observation s. Over a cycle they sum to the log-ML increment.
    """
    T = X.shape[0]
    P = theta.shape[0]
    logw = np.zeros(P)
    prev = np.zeros(J)                       # log mean_n w_jn(t0) = 0
    s = t0
    e = float(P)
    # evaluate observation terms a block at a time; the stopping rule is still applied at each s
    block = 64
    while s < T:
        hi = min(T, s + block)
        terms = log_prob_terms(X[s:hi], y[s:hi], theta, C)      # [P, hi - s]
        for j in range(hi - s):
            logw = logw + terms[:, j]
            s += 1
            if log_pred is not None:
                cur = np.array([log_mean_exp(logw[g * N:(g + 1) * N]) for g in range(J)])
                log_pred.append(cur - prev)
                prev = cur
            e = ess(logw)
            if t_fixed is not None:
                if s == t_fixed:
                    return s, logw, e
            elif e / P < ess_fraction or s == T:
                return s, logw, e
    return s, logw, e


def sphase(theta, ll, logw, J: int, N: int, rng: np.random.Generator, scheme: str = "multinomial"):
    """S phase (Algorithm 1 step 2(b)): multinomial (or residual) resampling of each group
    independently."""
    idx = np.empty(J * N, dtype=np.int64)
    for j in range(J):
        w = normalised_weights(logw[j * N:(j + 1) * N])
        u = rng.random(N)
        pick = resample_residual(w, u) if scheme == "residual" else resample_multinomial(w, u)
        idx[j * N:(j + 1) * N] = j * N + pick
    return theta[idx].copy(), ll[idx].copy(), idx


def monitoring_values(theta: np.ndarray, ll: np.ndarray, xbar: np.ndarray, C: int) -> np.ndarray:
    """Monitoring functions for the RNE rule: ell(theta; y_1:t) and theta_c' xbar, c = 1..C-1."""
    k = xbar.shape[0]
    cols = [ll]
    for c in range(1, C):
        cols.append(theta[:, (c - 1) * k:c * k] @ xbar)
    return np.stack(cols, axis=1)


def particle_covariance(theta: np.ndarray) -> np.ndarray:
    """V: pooled sample covariance of all J N particles, divisor J N - 1 (Algorithm 2 2(c)i)."""
    return np.atleast_2d(np.cov(theta, rowvar=False, ddof=1))


def rw_step(X, y, C, t: int, theta, ll, prior: GaussianPrior, Sigma: np.ndarray,
            z: np.ndarray, u: np.ndarray):
    """One Gaussian random-walk Metropolis step (Algorithm 2 step 2(c)i) with given randomness.

    theta' = theta + L z with L L' = Sigma; log alpha = ell(theta') - ell(theta) + log p(theta')
    - log p(theta); accept when log u < log alpha. The kernel is symmetric, so it leaves the
    posterior given y_{1:t} invariant (Eq. 13). Returns (theta, ll, accepted mask).
    """
    try:
        L = np.linalg.cholesky(Sigma)
    except np.linalg.LinAlgError as exc:
        raise DegenerateError(str(exc)) from exc
    prop = theta + z @ L.T
    ll_prop = loglik(X, y, prop, C, t)
    log_alpha = ll_prop - ll + prior.log_kernel(prop) - prior.log_kernel(theta)
    with np.errstate(divide="ignore"):
        acc = np.log(u) < log_alpha
    theta = np.where(acc[:, None], prop, theta)
    ll = np.where(acc, ll_prop, ll)
    return theta, ll, acc


def mala_step(X, y, C, t: int, theta, ll, prior: GaussianPrior, Sigma: np.ndarray,
              z: np.ndarray, u: np.ndarray):
    """One Metropolis-adjusted Langevin step with given randomness (not in the paper: an exact
    Metropolis-Hastings kernel for the same posterior given y_{1:t}, Eq. 13, used beside the
    random walk of Algorithm 2 step 2(c)i).

    With g(theta) the gradient of the log posterior (log-likelihood plus log prior) and L the
    lower Cholesky factor of Sigma, the proposal density is q(theta' | theta) =
    N(theta'; theta + Sigma g(theta) / 2, Sigma), drawn as theta' = theta + Sigma g(theta) / 2 + L z.
    The acceptance ratio is the Metropolis-Hastings ratio of the posterior kernel and the two
    proposal densities (their normalising constants are equal and cancel):
        log alpha = ell(theta') + log p(theta') + log q(theta | theta')
                  - ell(theta)  - log p(theta)  - log q(theta' | theta),
    accept when log u < log alpha. Returns (theta, ll, accepted mask, log alpha).
    """
    try:
        L = np.linalg.cholesky(Sigma)
    except np.linalg.LinAlgError as exc:
        raise DegenerateError(str(exc)) from exc
    Sinv = np.linalg.inv(Sigma)
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))

    def grad_log_post(th):
        _, gl = loglik_grad(X, y, th, C, t)
        return gl - (th - prior.mean[None, :]) @ prior.prec.T

    def log_q(to, frm, g_frm):
        # log N(to; frm + Sigma g(frm) / 2, Sigma) up to the shared constant
        r = to - frm - 0.5 * g_frm @ Sigma.T
        return -0.5 * np.einsum("pi,ij,pj->p", r, Sinv, r)

    g = grad_log_post(theta)
    prop = theta + 0.5 * g @ Sigma.T + z @ L.T
    ll_prop = loglik(X, y, prop, C, t)
    g_prop = grad_log_post(prop)
    log_alpha = (ll_prop + prior.log_kernel(prop) + log_q(theta, prop, g_prop)
                 - ll - prior.log_kernel(theta) - log_q(prop, theta, g))
    with np.errstate(divide="ignore"):
        acc = np.log(u) < log_alpha
    theta = np.where(acc[:, None], prop, theta)
    ll = np.where(acc, ll_prop, ll)
    return theta, ll, acc, log_alpha


def next_h(h: float, alpha: float, opt: SpsOptions) -> float:
    """Algorithm 2 step 2(c)ii: h <- min(h + 0.01, 1) if alpha > 0.25, else max(h - 0.01, 0.1)."""
    if alpha > opt.target_accept:
        return min(h + opt.h_step, opt.h_max)
    return max(h - opt.h_step, opt.h_min)


# ----------------------------------------------------------------------------- driver

def sps_run(X: np.ndarray, y: np.ndarray, C: int, prior: GaussianPrior, J: int, N: int,
            rng: np.random.Generator, options: Optional[SpsOptions] = None,
            schedule: Optional[List[CycleRecord]] = None) -> SpsResult:
    """Adaptive SPS (Algorithm 2), or the replay of a recorded schedule (Algorithm 3 pass 2).

    Initial particles are iid prior draws (Algorithm 1 step 1). Each cycle runs the C phase to
    t_l, the S phase, then M steps r = 1, 2, ... until the smallest RNE of the monitoring set
    reaches K (0.35 before T, 0.9 at T). With a schedule, t_l, R_l and Sigma_lr are taken from it.
    """
    opt = options or SpsOptions()
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.int32)
    T, k = X.shape
    P = J * N
    xbar = X.mean(axis=0)
    theta = prior.sample(rng, P)
    ll = np.zeros(P)
    t = 0
    h = opt.h_init
    logml = np.zeros(J)
    cycles: List[CycleRecord] = []
    ell_idx = 0
    while t < T:
        fixed = schedule[ell_idx] if schedule is not None else None
        lp: list = []
        t_new, logw, e = cphase(X, y, C, theta, t, J, N, opt.ess_fraction,
                                t_fixed=None if fixed is None else fixed.t, log_pred=lp)
        inc = np.array([log_mean_exp(logw[j * N:(j + 1) * N]) for j in range(J)])
        logml += inc
        ll = ll + logw
        rec = CycleRecord(t=t_new, ess_end=e, logml_inc=inc, log_pred=np.array(lp))
        t = t_new
        theta, ll, _ = sphase(theta, ll, logw, J, N, rng, opt.resampling)
        K = opt.rne_final if t == T else opt.rne_cycle
        r = 0
        while True:
            r += 1
            if fixed is not None:
                Sigma = fixed.sigmas[r - 1]
            else:
                Sigma = h * particle_covariance(theta)
            z = rng.standard_normal((P, k * (C - 1)))
            u = rng.random(P)
            theta, ll, acc = rw_step(X, y, C, t, theta, ll, prior, Sigma, z, u)
            alpha = float(acc.mean())
            rec.sigmas.append(np.array(Sigma))
            rec.hs.append(h)
            rec.accept.append(alpha)
            if fixed is None:
                h = next_h(h, alpha, opt)
            mom = group_moments(monitoring_values(theta, ll, xbar, C), J, N)
            rmin = float(np.min(mom.rne))
            rec.rne_min.append(rmin)
            if fixed is not None:
                if r >= fixed.R:
                    break
            elif rmin >= K or r >= opt.r_max:
                break
        rec.R = r
        cycles.append(rec)
        ell_idx += 1
    g = np.concatenate([theta, monitoring_values(theta, ll, xbar, C)[:, 1:]], axis=1)
    mom = group_moments(g, J, N)
    lm = float(logml.mean())
    lm_nse = float(logml.std(ddof=1) / np.sqrt(J)) if J > 1 else float("nan")
    mx = logml.max()
    pooled = float(mx + np.log(np.mean(np.exp(logml - mx))))
    lpg = np.concatenate([c.log_pred for c in cycles], axis=0)   # [T, J]
    lp_nse = lpg.std(axis=1, ddof=1) / np.sqrt(J) if J > 1 else np.full(T, np.nan)
    return SpsResult(theta, ll, mom, lm, lm_nse, logml, pooled, cycles, lpg, lpg.mean(axis=1), lp_nse)
