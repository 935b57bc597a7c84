"""Batched model comparison (sps_run_batched): nested models of one data set run through the
simulator together, their M phases in lockstep with one batched log-likelihood launch per step.
Each model must behave as its own run of Algorithm 2: the log marginal likelihood and the
posterior moments agree with separate runs on X[:, :k_m] within the Monte Carlo error, and the
exact special case X = 0 gives log ML = -n log C for every model."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _nested_case(n=400, k=5, C=2, seed=4):
    g = np.random.Generator(np.random.PCG64(seed))
    X = g.standard_normal((n, k))
    X[:, 0] = 1.0
    X[:, 3:] = (X[:, 3:] > 0.2).astype(float)     # exact 0/1 columns after continuous ones
    beta = np.zeros((k, C))
    beta[:3, 1:] = 0.8 * g.standard_normal((3, C - 1))
    eta = X @ beta
    p = np.exp(eta - eta.max(axis=1, keepdims=True))
    p /= p.sum(axis=1, keepdims=True)
    y = np.array([g.choice(C, p=row) for row in p], dtype=np.int32)
    return X, y


def test_zero_covariates_every_model_exact(cuda):
    from paper_1304_4333_b300 import Sps
    n, C = 60, 3
    X = np.zeros((n, 4))
    y = np.random.Generator(np.random.PCG64(1)).integers(0, C, n).astype(np.int32)
    s = Sps(X, y, C, prior_sd=5.0, seed=3)
    rs = s.run_batched([1, 2, 4], 8, 256)
    for r in rs:
        assert r.n_cycles == 1
        assert r.log_ml == pytest.approx(-n * math.log(C), abs=1e-5)
    s.close()


@pytest.mark.parametrize("C,prec", [(2, "split"), (3, "split"), (2, "fp32")])
def test_batched_agrees_with_separate_runs(cuda, C, prec):
    from paper_1304_4333_b300 import Sps
    X, y = _nested_case(C=C)
    ks = [2, 3, 5]
    s = Sps(X, y, C, prior_sd=5.0, seed=7, precision=prec)
    rb = s.run_batched(ks, 16, 512)
    s.close()
    for km, r in zip(ks, rb):
        s1 = Sps(np.ascontiguousarray(X[:, :km]), y, C, prior_sd=5.0, seed=100 + km, precision=prec)
        r1 = s1.run(16, 512, record=False)
        s1.close()
        comb = math.hypot(r.log_ml_nse, r1.log_ml_nse)
        assert abs(r.log_ml - r1.log_ml) < 4 * max(comb, 1e-3), (km, r.log_ml, r1.log_ml, comb)
        D = km * (C - 1)
        z = (r.mean[:D] - r1.mean[:D]) / np.hypot(r.nse[:D], r1.nse[:D])
        assert np.all(np.abs(z) < 5), (km, z)
        np.testing.assert_allclose(r.sd[:D], r1.sd[:D], rtol=0.2)
        assert r.m_steps >= r.n_cycles >= 1


def test_batched_rejects_bad_models(cuda):
    from paper_1304_4333_b300 import Sps, SpsError
    X, y = _nested_case()
    s = Sps(X, y, 2, prior_sd=5.0)
    with pytest.raises(SpsError):
        s.run_batched([0, 2], 4, 64)
    with pytest.raises(SpsError):
        s.run_batched([6], 4, 64)
    s.close()


def test_batched_gprior_matches_separate_gprior_runs(cuda):
    # with g > 0 each model gets the g-prior of its own covariates, as sps_gprior + sps_set_prior
    from paper_1304_4333_b300 import Sps
    X, y = _nested_case(C=3, seed=8)
    ks = [2, 4]
    s = Sps(X, y, 3, prior_sd=5.0, seed=9)
    rb = s.run_batched(ks, 16, 512, g=0.25)
    s.close()
    for km, r in zip(ks, rb):
        s1 = Sps(np.ascontiguousarray(X[:, :km]), y, 3, prior_sd=5.0, seed=50 + km)
        gm, gc = s1.gprior(0.25)
        s1.set_prior(prior_mean=gm, prior_cov=gc)
        r1 = s1.run(16, 512, record=False)
        s1.close()
        comb = math.hypot(r.log_ml_nse, r1.log_ml_nse)
        assert abs(r.log_ml - r1.log_ml) < 4 * max(comb, 1e-3), (km, r.log_ml, r1.log_ml, comb)


def test_batched_mala_agrees_with_separate_runs(cuda):
    # MALA M phases in lockstep (each model's gradient from its own launch): the same posterior and
    # marginal likelihood as separate MALA runs within the Monte Carlo error
    from paper_1304_4333_b300 import Sps
    X, y = _nested_case(C=2, seed=12)
    ks = [2, 3, 5]
    s = Sps(X, y, 2, prior_sd=5.0, seed=13, mkernel="mala")
    rb = s.run_batched(ks, 16, 512)
    s.close()
    for km, r in zip(ks, rb):
        s1 = Sps(np.ascontiguousarray(X[:, :km]), y, 2, prior_sd=5.0, seed=60 + km, mkernel="mala")
        r1 = s1.run(16, 512, record=False)
        s1.close()
        comb = math.hypot(r.log_ml_nse, r1.log_ml_nse)
        assert abs(r.log_ml - r1.log_ml) < 4 * max(comb, 1e-3), (km, r.log_ml, r1.log_ml, comb)
        z = (r.mean[:km] - r1.mean[:km]) / np.hypot(r.nse[:km], r1.nse[:km])
        assert np.all(np.abs(z) < 5), (km, z)


def test_batched_small_nested_case_against_oracle(cuda):
    # per-model log marginal likelihoods of a batched run against the FP64 oracle simulator run on
    # each model's own columns (independent random numbers): within 4x the combined NSE
    from oracle import smc as OS
    from paper_1304_4333_b300 import Sps
    X, y = _nested_case(n=200, k=4, C=2, seed=21)
    ks = [1, 2, 4]
    s = Sps(X, y, 2, prior_sd=5.0, seed=22)
    rb = s.run_batched(ks, 8, 256)
    s.close()
    for km, r in zip(ks, rb):
        prior = OS.GaussianPrior.isotropic(km, 5.0)
        o = OS.sps_run(np.ascontiguousarray(X[:, :km]), y, 2, prior, 8, 256,
                       np.random.Generator(np.random.PCG64(23 + km)))
        comb = math.hypot(r.log_ml_nse, o.log_ml_nse)
        assert abs(r.log_ml - o.log_ml) < 4 * max(comb, 1e-3), (km, r.log_ml, o.log_ml, comb)


def _batched(X, y, C, ks, J, N, graphs, **kw):
    from paper_1304_4333_b300 import Sps
    s = Sps(X, y, C, prior_sd=5.0, seed=31, graphs=graphs, **kw)
    try:
        r = s.run_batched(ks, J, N)
        # a graph that could not be built leaves its reason here (and the run continues from the host)
        assert "not used" not in s.lib.sps_last_error(s.ctx).decode()
        return r
    finally:
        s.close()


@pytest.mark.parametrize("C,prec,mkernel", [(2, "split", "rw"), (3, "split", "rw"), (2, "fp32", "rw"),
                                            (3, "split", "mala")])
def test_batched_graph_phases_identical_to_host_steps(cuda, C, prec, mkernel):
    # the captured C and S phases (device-side ESS stopping rule and block choice) and lockstep M
    # phases (per-model conditional nodes, one batched evaluation per step, device-side step-size
    # and stopping rules) take the same decisions with the same rounding as the host-driven
    # loops: every output of every model is bit for bit the same
    X, y = _nested_case(n=300, k=5, C=C, seed=40 + C)
    ks = [1, 3, 5]
    g = _batched(X, y, C, ks, 8, 256, 1, precision=prec, mkernel=mkernel)
    h = _batched(X, y, C, ks, 8, 256, 0, precision=prec, mkernel=mkernel)
    for a, b in zip(g, h):
        assert a.n_cycles == b.n_cycles and a.m_steps == b.m_steps
        np.testing.assert_array_equal(a.log_ml_group, b.log_ml_group)
        for f in ("mean", "sd", "nse", "rne"):
            np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
        assert b.graph_steps == 0
    # most steps ran inside the graphs (every phase's first step runs on the host)
    assert sum(a.graph_steps for a in g) > 0.5 * sum(a.m_steps for a in g)
