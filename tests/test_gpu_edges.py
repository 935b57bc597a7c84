"""Edge cases of the log-likelihood entry points, against the FP64 oracle (Eq. 1).

* Linear predictors in the hundreds: the C > 2 epilogue's direct sum 1 + sum_c 2^u overflows FP32
  there and each such 16-column chunk takes the shifted form; the C = 2 form (|u| and 2^-|u|) is
  stable by construction; the FP32 path shifts by the maximum.
* A single particle (one ragged particle tile) and a single observation (one ragged X tile).
* One outcome observed throughout, and an intercept-only model (no continuous column, so no
  low-part MMAs).
* Arguments the library must refuse with SPS_ERR_INVALID_ARG; the context stays usable.
* The tensor-core gradient with linear predictors in the hundreds (p saturated at 0 or 1), held
  to the bound of test_gpu_grad_tc.

Tolerances as in test_gpu_loglik: every particle within the relative bar (1e-5 split, 1e-6 FP32)
plus the propagated rounding bound of its linear predictors, and the relative bar on its own for
prefixes of a whole tile or more, over the particles whose log-likelihood is not a near-perfect
fit (|ll| >= 0.1 t). Where every term is close to zero (a single observation with |eta| large,
one outcome that a particle predicts almost surely) the error is set by the rounding of eta, not
by the size of ll, and only the bound applies. With one outcome throughout, the split path's
errors in eta (hi + lo BF16 keep 16 bits of each operand's mantissa) add up instead of cancelling
as they do when the residuals y_s - p_s change sign, and for C = 2 the kernel's sum of |eta| / 2
cancels against the linear part theta . X'(y - 1/2) on well-predicted observations: the relative
error reaches a few 1e-5 (within the bound, which assumes no cancellation); that case asserts the
bound and reports the relative error.
"""
import ctypes as C

import numpy as np
import pytest

from oracle.logit import loglik as oracle_loglik

pytestmark = pytest.mark.gpu

INVALID_ARG = 1


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _mk(n, k, C_, seed, exact_cols=0):
    g = np.random.Generator(np.random.PCG64(seed))
    X = g.standard_normal((n, k))
    X[:, 0] = 1.0
    if exact_cols:
        X[:, k - exact_cols:] = (g.random((n, exact_cols)) < 0.3).astype(float)
    y = g.integers(0, C_, n).astype(np.int32)
    return X, y


def _sps(X, y, C_):
    from paper_1304_4333_b300 import Sps
    return Sps(X, y, C_, prior_sd=5.0)


def _bound(X, theta, C_, t, prec):
    """Rounding of each eta_s propagated into the sum (|d term / d eta| <= 1)."""
    k = X.shape[1]
    A = np.abs(X[:t])
    B = np.zeros(theta.shape[0])
    for c in range(C_ - 1):
        B += (np.abs(theta[:, c * k:(c + 1) * k]) @ A.T).sum(axis=1)
    return (3 * 2.0 ** -16 if prec == "split" else k * 2.0 ** -23) * B


def _check(got, ref, X, theta, C_, t, prec, rel_bar=True):
    assert np.all(np.isfinite(got))
    bar = 1e-5 if prec == "split" else 1e-6
    err = np.abs(got - ref)
    assert np.all(err <= bar * np.abs(ref) + _bound(X, theta, C_, t, prec) + 1e-9 * t), np.max(err)
    typical = np.abs(ref) >= 0.1 * t
    rel = 0.0
    if t >= 128 and np.any(typical):
        rel = float(np.max(err[typical] / np.abs(ref[typical])))
        assert rel <= bar or not rel_bar, rel
    return rel


@pytest.mark.parametrize("prec", ["split", "fp32"])
@pytest.mark.parametrize("C_", [2, 3, 4])
def test_linear_predictors_in_the_hundreds(torch_cuda, C_, prec):
    n, k = 300, 6
    X, y = _mk(n, k, C_, 11, exact_cols=2)
    g = np.random.Generator(np.random.PCG64(12))
    theta = g.standard_normal((256, k * (C_ - 1))) * 80.0
    eta_max = max(np.max(np.abs(X @ theta[:, c * k:(c + 1) * k].T)) for c in range(C_ - 1))
    assert eta_max > 200.0   # 2^(eta log2 e) overflows FP32 beyond eta = 88.7
    s = _sps(X, y, C_)
    for t in (1, 130, n):
        ref = oracle_loglik(X, y, theta, C_, t)
        rel = _check(s.loglik(theta, t, prec), ref, X, theta, C_, t, prec)
    print(f"C={C_} {prec}: |eta| up to {eta_max:.0f}, max relative error {rel:.2e}")


@pytest.mark.parametrize("prec", ["split", "fp32"])
@pytest.mark.parametrize("C_", [2, 4])
def test_single_particle_and_single_observation(torch_cuda, C_, prec):
    k = 5
    X, y = _mk(300, k, C_, 21, exact_cols=1)
    theta = np.random.Generator(np.random.PCG64(22)).standard_normal((1, k * (C_ - 1)))
    s = _sps(X, y, C_)
    for t in (0, 1, 129, 300):
        ref = oracle_loglik(X, y, theta, C_, t)
        got = s.loglik(theta, t, prec)
        assert got.shape == (1,)
        if t == 0:
            assert got[0] == 0.0
        else:
            _check(got, ref, X, theta, C_, t, prec)
    # a data set of one observation
    s1 = _sps(X[:1], y[:1], C_)
    th = np.random.Generator(np.random.PCG64(23)).standard_normal((300, k * (C_ - 1)))
    _check(s1.loglik(th, 1, prec), oracle_loglik(X[:1], y[:1], th, C_, 1), X[:1], th, C_, 1, prec)


@pytest.mark.parametrize("prec", ["split", "fp32"])
@pytest.mark.parametrize("C_", [2, 3])
def test_one_outcome_throughout(torch_cuda, C_, prec):
    n, k = 400, 8
    X, _ = _mk(n, k, C_, 31, exact_cols=3)
    theta = np.random.Generator(np.random.PCG64(32)).standard_normal((200, k * (C_ - 1)))
    for cls in (0, C_ - 1):
        y = np.full(n, cls, dtype=np.int32)
        s = _sps(X, y, C_)
        rel = _check(s.loglik(theta, n, prec), oracle_loglik(X, y, theta, C_, n), X, theta, C_, n, prec,
                     rel_bar=(prec == "fp32"))
        print(f"C={C_} {prec}, every outcome {cls}: max relative error {rel:.2e}")


@pytest.mark.parametrize("prec", ["split", "fp32"])
@pytest.mark.parametrize("C_", [2, 4])
def test_intercept_only_model(torch_cuda, C_, prec):
    n = 700
    X = np.ones((n, 1))
    y = np.random.Generator(np.random.PCG64(41)).integers(0, C_, n).astype(np.int32)
    theta = np.random.Generator(np.random.PCG64(42)).standard_normal((300, C_ - 1)) * 2.0
    s = _sps(X, y, C_)
    # closed form: counts of each outcome times the log softmax of the intercepts
    eta = np.concatenate([np.zeros((theta.shape[0], 1)), theta], axis=1)
    logp = eta - np.log(np.exp(eta).sum(axis=1, keepdims=True))
    for t in (1, 255, n):
        counts = np.bincount(y[:t], minlength=C_)
        ref = logp @ counts
        np.testing.assert_allclose(ref, oracle_loglik(X, y, theta, C_, t), rtol=1e-12)
        _check(s.loglik(theta, t, prec), ref, X, theta, C_, t, prec)


def test_invalid_arguments_are_refused_and_the_context_stays_usable(torch_cuda):
    n, k, C_ = 200, 4, 3
    X, y = _mk(n, k, C_, 51)
    s = _sps(X, y, C_)
    th = np.random.Generator(np.random.PCG64(52)).standard_normal((64, k * (C_ - 1)))
    out = np.empty(64)
    grad = np.empty(th.size)
    pt = th.ctypes.data_as(C.c_void_p)
    po = out.ctypes.data_as(C.c_void_p)
    pg = grad.ctypes.data_as(C.c_void_p)
    cases = [
        ("no particles", lambda: s.lib.sps_loglik(s.ctx, pt, 0, n, po, 0, 0)),
        ("negative prefix", lambda: s.lib.sps_loglik(s.ctx, pt, 64, -1, po, 0, 0)),
        ("prefix beyond n", lambda: s.lib.sps_loglik(s.ctx, pt, 64, n + 1, po, 0, 0)),
        ("null theta", lambda: s.lib.sps_loglik(s.ctx, None, 64, n, po, 0, 0)),
        ("null output", lambda: s.lib.sps_loglik(s.ctx, pt, 64, n, None, 0, 0)),
        ("unknown memory kind", lambda: s.lib.sps_loglik(s.ctx, pt, 64, n, po, 0, 7)),
        ("unknown precision", lambda: s.lib.sps_loglik(s.ctx, pt, 64, n, po, 9, 0)),
        ("gradient, no particles", lambda: s.lib.sps_loglik_grad(s.ctx, pt, 0, n, po, pg, 0)),
        ("gradient, prefix beyond n", lambda: s.lib.sps_loglik_grad(s.ctx, pt, 64, n + 1, po, pg, 0)),
    ]
    ref = oracle_loglik(X, y, th, C_, n)
    for name, call in cases:
        assert call() == INVALID_ARG, name
        assert s.lib.sps_last_error(s.ctx).decode(), name   # a message says what was wrong
        # the context still computes
        for prec in ("split", "fp32"):
            _check(s.loglik(th, n, prec), ref, X, th, C_, n, prec)


def _grad_bound(X, th, C_, t):
    """The tensor-core gradient's bound (as in test_gpu_grad_tc): 2^-13 sum_s (1 + |eta_s|) |x_si|
    per entry, on top of 1e-5 of the oracle gradient."""
    k = X.shape[1]
    Xt = X[:t]
    out = np.zeros_like(th)
    for c in range(C_ - 1):
        eta = th[:, c * k:(c + 1) * k] @ Xt.T
        out[:, c * k:(c + 1) * k] = (1.0 + np.abs(eta)) @ np.abs(Xt)
    return 2.0 ** -13 * out


@pytest.mark.parametrize("C_", [2, 3, 4])
def test_gradient_with_linear_predictors_in_the_hundreds(torch_cuda, C_):
    # p_s saturates at 0 or 1: the sigmoid / softmax of the gradient's epilogue must not overflow
    from oracle.logit import loglik_grad as oracle_grad
    n, k = 300, 6
    X, y = _mk(n, k, C_, 61, exact_cols=2)
    theta = np.random.Generator(np.random.PCG64(62)).standard_normal((200, k * (C_ - 1))) * 80.0
    s = _sps(X, y, C_)
    for t in (1, 130, n):
        ll, G = s.loglik_grad(theta, t)
        ll_o, G_o = oracle_grad(X, y, theta, C_, t)
        assert np.all(np.isfinite(G)) and np.all(np.isfinite(ll))
        bound = 1e-5 * np.abs(G_o) + _grad_bound(X, theta, C_, t)
        assert np.all(np.abs(G - G_o) <= bound), np.max(np.abs(G - G_o) - bound)
        _check(ll, ll_o, X, theta, C_, t, "split")
