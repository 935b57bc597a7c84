"""GPU parity of the simulator's building blocks and phases against the FP64 oracle.

Bars: bit-exact for Philox words and for resampling indices given the same FP64 weights and
uniforms; ESS within 1e-6 relative (FP32 exponentials of FP64 differences, FP64 sums);
per-group log-mean-exp within 1e-12; the particle covariance within 1e-5 relative (FP32
products of FP64-centred values); gradient within 1e-5 of the oracle gradient and 1e-4 of
central finite differences (norm-wise); one Metropolis step with given randomness: the same
accept decisions away from ties and log alpha within the log-likelihood tolerance.
"""
import math

import numpy as np
import pytest

import synthetic
from oracle import logit as OL
from oracle import smc as OS
from oracle.philox import philox_array

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _ctx(X, y, C, **kw):
    from paper_1304_4333_b300 import Sps
    return Sps(X, y, C, prior_sd=5.0, **kw)


def _small(n=300, k=4, C=2, seed=0):
    g = np.random.Generator(np.random.PCG64(seed))
    X = g.standard_normal((n, k))
    X[:, 0] = 1.0
    y = g.integers(0, C, n).astype(np.int32)
    return X, y


def test_philox_bitwise(cuda):
    X, y = _small()
    s = _ctx(X, y, 2)
    assert list(s.philox((0, 0), (0, 0, 0, 0), 1)[0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    out = s.philox((0xDEADBEEF, 0x12345678), (5, 7, 9, 11), 5000)
    ctr = np.zeros((5000, 4), np.uint32)
    ctr[:, 0] = 5 + np.arange(5000)
    ctr[:, 1:] = (7, 9, 11)
    np.testing.assert_array_equal(out, philox_array(ctr, (0xDEADBEEF, 0x12345678)))


@pytest.mark.parametrize("J,N", [(1, 3), (5, 1000), (3, 4096), (16, 256)])
def test_resample_bit_exact(cuda, J, N):
    X, y = _small()
    s = _ctx(X, y, 2)
    g = np.random.Generator(np.random.PCG64(J * 1000 + N))
    lw = g.standard_normal((J, N)) * 3
    w = np.exp(lw - lw.max(axis=1, keepdims=True))
    w[0, : min(N, 2)] = 0.0               # zero weights are never selected
    if N > 2:
        w[0, 2] = 1.0
    u = g.random((J, N))
    u[0, 0] = 0.0
    u[-1, -1] = np.nextafter(1.0, 0.0)     # the clamp tau <= Q - 1
    got = s.resample(w.reshape(-1), u.reshape(-1), J, N).reshape(J, N)
    for j in range(J):
        np.testing.assert_array_equal(got[j], OS.resample_multinomial(w[j], u[j]))


def test_resample_single_survivor(cuda):
    X, y = _small()
    s = _ctx(X, y, 2)
    w = np.zeros(64); w[37] = 1.0
    got = s.resample(w, np.linspace(0, 1, 64, endpoint=False), 1, 64)
    assert np.all(got == 37)


def test_ess_and_group_log_mean_exp(cuda):
    X, y = _small()
    s = _ctx(X, y, 2)
    g = np.random.Generator(np.random.PCG64(3))
    for J, N, scale in ((4, 256, 2.0), (16, 4096, 10.0), (2, 3, 0.0)):
        lw = g.standard_normal(J * N) * scale - 50.0
        e, lme = s.ess(lw, J)
        assert e == pytest.approx(OS.ess(lw), rel=1e-6)
        want = [OS.log_mean_exp(lw[j * N:(j + 1) * N]) for j in range(J)]
        np.testing.assert_allclose(lme, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("C,k", [(2, 5), (4, 50)])
def test_particle_covariance(cuda, C, k):
    X, y = _small(k=k, C=C)
    s = _ctx(X, y, C)
    D = k * (C - 1)
    g = np.random.Generator(np.random.PCG64(4))
    A = g.standard_normal((D, D)) * 0.1 + np.eye(D)
    th = 3.0 + g.standard_normal((5000, D)) @ A.T
    V = s.particle_cov(th)
    ref = OS.particle_covariance(th)
    assert np.max(np.abs(V - ref)) / np.max(np.abs(ref)) < 1e-5
    np.testing.assert_allclose(V, V.T)


@pytest.mark.parametrize("C", [2, 3])
def test_gradient_against_oracle_and_finite_differences(cuda, C):
    # the FP32 SIMT gradient kernel (precision fp32); the tensor-core form is in test_gpu_grad_tc.py
    X, y = _small(n=700, k=6, C=C, seed=5)
    s = _ctx(X, y, C, precision="fp32")
    D = 6 * (C - 1)
    g = np.random.Generator(np.random.PCG64(6))
    th = 0.3 * g.standard_normal((130, D))
    ll, gr = s.loglik_grad(th, 650)
    ll_o, gr_o = OL.loglik_grad(X, y, th, C, 650)
    np.testing.assert_allclose(ll, ll_o, rtol=1e-6)
    assert np.max(np.abs(gr - gr_o)) / np.max(np.abs(gr_o)) < 1e-5
    for p in (0, 77):
        fd = np.zeros(D)
        for i in range(D):
            h = 1e-5 * max(1.0, abs(th[p, i]))
            e = np.zeros(D); e[i] = h
            fd[i] = (OL.loglik(X, y, (th[p] + e)[None], C, 650)[0] - OL.loglik(X, y, (th[p] - e)[None], C, 650)[0]) / (2 * h)
        assert np.max(np.abs(gr[p] - fd)) / np.max(np.abs(fd)) < 1e-4


@pytest.mark.parametrize("prec", ["split", "fp32"])
def test_rw_step_given_randomness(cuda, prec):
    w = synthetic.make_c1()
    s = _ctx(w.X, w.y, w.C)
    P, D, t = 1024, w.D, 300
    th = synthetic.particles_around(w.theta_true, P, 0.3, seed=7)
    ll = OL.loglik(w.X, w.y, th, w.C, t)
    prior = OS.GaussianPrior.isotropic(D, 5.0)
    Sigma = 0.5 * OS.particle_covariance(th)
    g = np.random.Generator(np.random.PCG64(8))
    z = g.standard_normal((P, D))
    u = g.random(P)
    th_o, ll_o, acc_o = OS.rw_step(w.X, w.y, w.C, t, th, ll, prior, Sigma, z, u)
    L = np.linalg.cholesky(Sigma)
    prop = th + z @ L.T
    la_o = OL.loglik(w.X, w.y, prop, w.C, t) - ll + prior.log_kernel(prop) - prior.log_kernel(th)
    th_g, ll_g, la_g, acc_g = s.rw_step_given(th, ll, t, Sigma, z, u, prec)
    np.testing.assert_allclose(la_g, la_o, atol=2e-3, rtol=1e-4)
    clear = np.abs(np.log(u) - la_o) > 1e-2
    np.testing.assert_array_equal(acc_g[clear], acc_o[clear])
    sel = clear & acc_o
    np.testing.assert_allclose(th_g[sel], th_o[sel], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(ll_g[sel], ll_o[sel], rtol=1e-5)
    assert 0.05 < acc_g.mean() < 0.95


def test_cphase_matches_oracle(cuda):
    w = synthetic.make_c1()
    s = _ctx(w.X, w.y, w.C)
    st = s.state(4, 256, seed=11)
    th = st.get()["theta"]
    t_new, ess, inc = st.cphase()
    t_o, logw_o, ess_o = OS.cphase(w.X, w.y, w.C, th, 0, 4, 256)
    assert t_new == t_o
    assert ess == pytest.approx(ess_o, rel=1e-5)
    want = [OS.log_mean_exp(logw_o[j * 256:(j + 1) * 256]) for j in range(4)]
    np.testing.assert_allclose(inc, want, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(st.get()["logw"], logw_o, rtol=1e-5, atol=1e-5)


def test_sphase_gathers_selected_particles(cuda):
    w = synthetic.make_c1()
    s = _ctx(w.X, w.y, w.C)
    st = s.state(4, 256, seed=12)
    before = st.get()
    st.cphase()
    lw = st.get()["logw"]
    u = np.random.Generator(np.random.PCG64(13)).random(1024)
    idx = st.sphase(u)
    after = st.get()
    for j in range(4):
        sl = slice(j * 256, (j + 1) * 256)
        ww = np.exp(lw[sl] - lw[sl].max())
        ref = OS.resample_multinomial(ww, u[sl])
        # the weights are exponentiated on the device; indices agree except where an ulp of exp
        # moves a CDF boundary across a uniform, which these seeds do not hit
        np.testing.assert_array_equal(idx[sl], ref)
        np.testing.assert_array_equal(after["theta"][sl], before["theta"][sl][idx[sl]])


def test_degenerate_particles_raise(cuda):
    from paper_1304_4333_b300 import SpsError
    w = synthetic.make_c1()
    s = _ctx(w.X, w.y, w.C)
    st = s.state(2, 64, seed=1)
    st.set(np.tile(w.theta_true, (128, 1)), None, 100)
    with pytest.raises(SpsError) as e:
        st.mstep()
    assert e.value.status == 4   # SPS_ERR_DEGENERATE


def test_zero_covariates_log_ml_exact(cuda):
    n, k, C = 60, 2, 3
    X = np.zeros((n, k))
    y = np.random.Generator(np.random.PCG64(1)).integers(0, C, n).astype(np.int32)
    s = _ctx(X, y, C, seed=3)
    r = s.run(8, 256)
    assert r.n_cycles == 1
    assert r.log_ml == pytest.approx(-n * math.log(C), abs=1e-5)
    D = k * (C - 1)
    assert np.all(np.abs(r.mean[:D] / r.nse[:D]) < 5)
    np.testing.assert_allclose(r.sd[:D], 5.0, rtol=0.15)


def _quad_case():
    from oracle.quadrature import binary_logit_posterior
    n = 200
    g = np.random.Generator(np.random.PCG64(7))
    X = np.concatenate([np.ones((n, 1)), g.standard_normal((n, 1))], axis=1)
    eta = -0.4 + 1.2 * X[:, 1]
    y = (g.random(n) < 1 / (1 + np.exp(-eta))).astype(np.int32)
    quad = binary_logit_posterior(X, y, np.zeros(2), 25.0 * np.eye(2), points=801)
    return X, y, quad


@pytest.mark.parametrize("prec", ["split", "fp32"])
def test_sps_run_against_quadrature(cuda, prec):
    X, y, quad = _quad_case()
    s = _ctx(X, y, 2, seed=21, precision=prec)
    r = s.run(16, 1024)
    z = (r.mean[:2] - quad["mean"]) / r.nse[:2]
    assert np.all(np.abs(z) < 4), (r.mean[:2], quad["mean"], r.nse[:2])
    np.testing.assert_allclose(r.sd[:2], quad["sd"], rtol=0.05)
    assert abs(r.log_ml - quad["log_ml"]) < 4 * max(r.log_ml_nse, 1e-3), (r.log_ml, quad["log_ml"], r.log_ml_nse)
    assert r.schedule.t[-1] == len(y) and r.schedule.R.sum() == r.m_steps


def test_sps_run_c1_against_oracle(cuda):
    # config c1 end to end: GPU and oracle (independent random numbers) agree within 4x the
    # combined NSE on the moments and the log marginal likelihood
    w = synthetic.make_c1()
    s = _ctx(w.X, w.y, w.C, seed=5)
    r = s.run(w.J, w.N)
    prior = OS.GaussianPrior.isotropic(w.D, 5.0)
    o = OS.sps_run(w.X, w.y, w.C, prior, w.J, w.N, np.random.Generator(np.random.PCG64(5)))
    m = w.D + w.C - 1
    comb = np.hypot(r.nse[:m], o.moments.nse[:m])
    assert np.all(np.abs(r.mean[:m] - o.moments.mean[:m]) < 4 * comb + 1e-9)
    comb_ml = math.hypot(r.log_ml_nse, o.log_ml_nse)
    assert abs(r.log_ml - o.log_ml) < 4 * comb_ml
    np.testing.assert_allclose(r.sd[:m], o.moments.sd[:m], rtol=0.2)


def test_two_pass_replay(cuda):
    X, y, quad = _quad_case()
    s = _ctx(X, y, 2, seed=31)
    p1 = s.run(8, 512)
    s2 = _ctx(X, y, 2, seed=32)
    p2 = s2.run(8, 512, schedule=p1.schedule)
    np.testing.assert_array_equal(p2.schedule.t, p1.schedule.t)
    np.testing.assert_array_equal(p2.schedule.R, p1.schedule.R)
    np.testing.assert_allclose(p2.schedule.sigma, p1.schedule.sigma)
    assert abs(p1.log_ml - p2.log_ml) < 5 * max(math.hypot(p1.log_ml_nse, p2.log_ml_nse), 1e-3)


def test_two_pass_replay_against_oracle_replay(cuda):
    # Algorithm 3: the oracle replays the schedule recorded by the library's adaptive pass (its t_l,
    # R_l and Sigma_lr, with its own random numbers); both replays follow the schedule exactly
    # and their log marginal likelihoods agree within 4x the combined NSE
    X, y, quad = _quad_case()
    s = _ctx(X, y, 2, seed=41)
    p1 = s.run(8, 512)
    sch = p1.schedule
    cycles, r0 = [], 0
    for tl, Rl in zip(sch.t, sch.R):
        cycles.append(OS.CycleRecord(t=int(tl), R=int(Rl), sigmas=[sch.sigma[r0 + r] for r in range(int(Rl))]))
        r0 += int(Rl)
    prior = OS.GaussianPrior.isotropic(2, 5.0)
    o = OS.sps_run(X, y, 2, prior, 8, 512, np.random.Generator(np.random.PCG64(42)), schedule=cycles)
    assert [c.t for c in o.cycles] == list(sch.t)
    assert [c.R for c in o.cycles] == list(sch.R)
    s2 = _ctx(X, y, 2, seed=43)
    p2 = s2.run(8, 512, schedule=sch)
    np.testing.assert_array_equal(p2.schedule.t, sch.t)
    comb = math.hypot(p2.log_ml_nse, o.log_ml_nse)
    assert abs(p2.log_ml - o.log_ml) < 4 * comb, (p2.log_ml, o.log_ml, comb)
    z = (p2.mean[:2] - o.moments.mean[:2]) / np.hypot(p2.nse[:2], o.moments.nse[:2])
    assert np.all(np.abs(z) < 4)
    assert abs(o.log_ml - quad["log_ml"]) < 4 * max(o.log_ml_nse, 1e-3)


def test_mala_leaves_the_prior_invariant_when_x_is_zero(cuda):
    # X = 0: the likelihood is constant, the posterior is the N(0, 25 I) prior and the MALA drift
    # comes from the prior alone. An exact MH kernel keeps prior draws distributed as the prior;
    # an error in the proposal-density ratio shows up as a drift of the variance.
    n, k = 40, 3
    X = np.zeros((n, k))
    y = (np.arange(n) % 2).astype(np.int32)
    s = _ctx(X, y, 2, seed=5)
    st = s.state(16, 1024, seed=7)
    t_new, _, _ = st.cphase()
    assert t_new == n
    st.sphase()
    accs = [st.mstep("mala")["accept"] for _ in range(60)]
    th = st.get()["theta"]
    assert 0.2 < np.mean(accs) < 0.99
    P = th.shape[0]
    # after resampling particles are duplicated; 60 steps decorrelate them, allow 6 sigma
    np.testing.assert_allclose(th.mean(axis=0), 0.0, atol=6 * 5.0 / np.sqrt(P / 4))
    np.testing.assert_allclose(th.var(axis=0), 25.0, rtol=0.1)


def test_sps_run_mala_against_quadrature(cuda):
    X, y, quad = _quad_case()
    s = _ctx(X, y, 2, seed=23, mkernel="mala")
    r = s.run(16, 1024)
    z = (r.mean[:2] - quad["mean"]) / r.nse[:2]
    assert np.all(np.abs(z) < 4), (r.mean[:2], quad["mean"], r.nse[:2])
    np.testing.assert_allclose(r.sd[:2], quad["sd"], rtol=0.05)
    assert abs(r.log_ml - quad["log_ml"]) < 4 * max(r.log_ml_nse, 1e-3)


@pytest.mark.parametrize("kernel", ["rw", "mala"])
def test_cycle_without_host_outputs_is_bitwise_the_same(cuda, kernel):
    # cphase(outputs=False), sphase(indices=False) and mstep(sigma_used=False) only skip copies
    # to the host (and the C phase's per-block ESS reads when its target is known): the state
    # after each cycle is identical bit for bit
    w = synthetic.make_c1()
    s = _ctx(w.X, w.y, w.C)
    a = s.state(4, 256, seed=21)
    b = s.state(4, 256, seed=21)
    for t in (40, 130, 131, 300):
        ta, _, inc = a.cphase(t)
        a.sphase()
        ia = a.mstep(kernel)
        tb, ess_b, inc_b = b.cphase(t, outputs=False)
        assert inc_b is None and math.isnan(ess_b)
        assert b.sphase(indices=False) is None
        ib = b.mstep(kernel, sigma_used=False)
        assert ib["sigma"] is None
        assert ta == tb == t
        assert ia["accept"] == ib["accept"] and ia["h_next"] == ib["h_next"]
        ga, gb = a.get(), b.get()
        for key in ("theta", "ll"):
            np.testing.assert_array_equal(ga[key], gb[key])


def _mnl_case(n=600, k=4, C=3, seed=61):
    g = np.random.Generator(np.random.PCG64(seed))
    X = g.standard_normal((n, k))
    X[:, 0] = 1.0
    beta = 0.5 * g.standard_normal((k, C - 1))
    eta = np.concatenate([np.zeros((n, 1)), X @ beta], axis=1)
    y = np.argmax(eta + g.gumbel(size=eta.shape), axis=1).astype(np.int32)
    return X, y


@pytest.mark.parametrize("C", [2, 3])
def test_step_rules_and_outputs_on_identical_inputs(cuda, C):
    # the library's acceptance rate, step-size rule and RNE of one M step (Algorithm 2 step
    # 2(c)ii-iii), and the run outputs of a state (Eqs. 5-7, 10, 15 and the log ML of the groups),
    # against the oracle's functions applied to the same particles and log-likelihoods
    if C == 2:
        w = synthetic.make_c1()
        X, y = w.X, w.y
    else:
        X, y = _mnl_case()
    J, N = 8, 256
    s = _ctx(X, y, C)
    st = s.state(J, N, seed=19)
    theta0 = st.get()["theta"]
    t_new, _, inc = st.cphase()
    st.sphase()
    before = st.get()
    info = st.mstep("rw")
    after = st.get()
    moved = np.any(after["theta"] != before["theta"], axis=1)
    assert info["accept"] == moved.mean()
    assert 0.0 < info["accept"] < 1.0
    assert info["h_next"] == OS.next_h(info["h"], info["accept"], OS.SpsOptions())
    # the library evaluates the log-odds theta_c' xbar as an FP32 dot product (a monitoring
    # function needs no more): 1e-7 relative per value, about 1e-6 on the moments built from them
    xbar = X.mean(axis=0)
    mon = OS.group_moments(OS.monitoring_values(after["theta"], after["ll"], xbar, C), J, N)
    assert info["rne_min"] == pytest.approx(mon.rne.min(), rel=1e-5)
    r = st.result()
    g = np.concatenate([after["theta"], OS.monitoring_values(after["theta"], after["ll"], xbar, C)[:, 1:]], axis=1)
    mom = OS.group_moments(g, J, N)
    D = after["theta"].shape[1]
    # theta's own coordinates: FP64 sums of FP64 values
    np.testing.assert_allclose(r.mean[:D], mom.mean[:D], rtol=1e-12, atol=1e-14)
    for f in ("sd", "nse", "rne"):
        np.testing.assert_allclose(getattr(r, f)[:D], getattr(mom, f)[:D], rtol=1e-9)
    np.testing.assert_allclose(r.mean[D:], mom.mean[D:], rtol=1e-6, atol=1e-7)
    for f in ("sd", "nse", "rne"):
        np.testing.assert_allclose(getattr(r, f)[D:], getattr(mom, f)[D:], rtol=1e-5)
    # the groups' log ML after one cycle: the C phase's increments, which follow the oracle's
    # C phase on the same initial particles (FP32 terms: 1e-5)
    np.testing.assert_array_equal(r.log_ml_group, inc)
    _, logw_o, _ = OS.cphase(X, y, C, theta0, 0, J, N)
    want = np.array([OS.log_mean_exp(logw_o[j * N:(j + 1) * N]) for j in range(J)])
    np.testing.assert_allclose(r.log_ml_group, want, rtol=1e-5, atol=1e-5)
    assert r.log_ml == pytest.approx(inc.mean(), rel=1e-14)
    assert r.log_ml_nse == pytest.approx(inc.std(ddof=1) / np.sqrt(J), rel=1e-12)
    assert r.log_ml_pooled == pytest.approx(inc.max() + np.log(np.mean(np.exp(inc - inc.max()))), rel=1e-12)
    assert r.n_cycles == 1 and r.m_steps == 1
    s.close()
