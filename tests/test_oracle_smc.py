"""Pins for the oracle's ESS (Eq. 14), group moments (Eqs. 3-10), resampling and Philox."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle.philox import philox4x32_10, philox_array, uniform53
from oracle.smc import (DegenerateError, ess, group_moments, log_mean_exp, next_h,
                        resample_multinomial, SpsOptions)


# ----------------------------------------------------------------------------- ESS (Eq. 14)

def test_ess_equal_weights_is_particle_count():
    assert ess(np.zeros(4096)) == pytest.approx(4096.0, rel=1e-14)


def test_ess_single_nonzero_weight_is_one():
    lw = np.full(100, -np.inf); lw[17] = -3.0
    assert ess(lw) == pytest.approx(1.0, rel=1e-15)


def test_ess_hand_value():
    # w = (1, 1, 0.5, 0) -> (2.5)^2 / 2.25
    lw = np.log(np.array([1.0, 1.0, 0.5, 1e-300]))
    assert ess(lw) == pytest.approx(2.5 ** 2 / 2.25, rel=1e-12)


def test_ess_bounds_and_shift_invariance(rng):
    lw = rng.standard_normal(1000) * 3
    e = ess(lw)
    assert 1.0 <= e <= 1000.0
    assert ess(lw + 123.456) == pytest.approx(e, rel=1e-12)
    assert log_mean_exp(lw + 7.0) == pytest.approx(log_mean_exp(lw) + 7.0, rel=1e-14)


def test_log_mean_exp_hand_value():
    assert log_mean_exp(np.log([1.0, 3.0])) == pytest.approx(math.log(2.0), abs=1e-15)


# ----------------------------------------------------------------------------- moments

def test_group_moments_hand_values():
    # J = 2, N = 2, g = (1, 3 | 5, 7): group means (2, 6), grand mean 4,
    # vhat = N/(J-1) * ((2-4)^2 + (6-4)^2) = 16, pooled var = (9+1+1+9)/4 = 5,
    # RNE = 5/16, NSE = sqrt(16/4) = 2.
    m = group_moments(np.array([1.0, 3.0, 5.0, 7.0]), J=2, N=2)
    assert m.mean[0] == 4.0 and m.vhat[0] == 16.0
    assert m.sd[0] == pytest.approx(math.sqrt(5.0))
    assert m.rne[0] == pytest.approx(5.0 / 16.0)
    assert m.nse[0] == pytest.approx(2.0)


def test_rne_near_one_for_iid_draws(rng):
    # iid draws: vhat estimates the variance, so RNE ~ 1 (chi2(J-1)/(J-1) spread).
    J, N = 64, 512
    g = rng.standard_normal(J * N)
    m = group_moments(g, J, N)
    assert 0.6 < m.rne[0] < 1.6
    assert m.nse[0] == pytest.approx(1.0 / math.sqrt(J * N), rel=0.35)


def test_step_size_rule():
    opt = SpsOptions()
    assert next_h(0.5, 0.26, opt) == pytest.approx(0.51)
    assert next_h(0.5, 0.25, opt) == pytest.approx(0.49)   # strict > 0.25
    assert next_h(1.0, 0.9, opt) == 1.0
    assert next_h(0.1, 0.0, opt) == 0.1


# ----------------------------------------------------------------------------- resampling

def test_resample_equal_weights_hand_case():
    w = np.ones(4)
    u = np.array([0.0, 0.25, 0.5, 0.75, 0.2499999999, 0.9999999999999999])
    np.testing.assert_array_equal(resample_multinomial(w, u), [0, 1, 2, 3, 0, 3])


def test_resample_unequal_hand_case():
    # w = (1, 0.5, 0.25, 0.25): CDF boundaries at 1/2, 3/4, 7/8 of the total.
    w = np.array([1.0, 0.5, 0.25, 0.25])
    u = np.array([0.49, 0.5, 0.74, 0.75, 0.874, 0.875, 0.99])
    np.testing.assert_array_equal(resample_multinomial(w, u), [0, 1, 1, 2, 2, 3, 3])


def test_resample_single_nonzero_weight():
    w = np.zeros(50); w[31] = 1.0
    u = np.linspace(0, 1, 200, endpoint=False)
    assert np.all(resample_multinomial(w, u) == 31)


def test_resample_all_zero_is_an_error():
    with pytest.raises(DegenerateError):
        resample_multinomial(np.zeros(8), np.array([0.5]))


def test_resample_offspring_unbiased(rng):
    # Multinomial resampling: E[O_n] = N w_n / sum w (the unbiasedness behind Chopin's CLT,
    # Sec. 2.2). Check with a chi-square test over replications.
    N, R = 16, 20000
    w = np.exp(rng.standard_normal(N))
    w = w / w.max()
    counts = np.zeros(N)
    for _ in range(R):
        idx = resample_multinomial(w, rng.random(N))
        c = np.bincount(idx, minlength=N)
        assert c.sum() == N
        counts += c
    expected = R * N * w / w.sum()
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert stats.chi2.sf(chi2, N - 1) > 1e-4


# ----------------------------------------------------------------------------- Philox

def test_philox_known_answers():
    # Known-answer vectors published with Philox4x32-10.
    assert philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]) == \
        [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_philox_vectorised_matches_scalar(rng):
    ctr = rng.integers(0, 2 ** 32, size=(50, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x12345678, 0x9ABCDEF0)
    out = philox_array(ctr, key)
    for i in range(50):
        assert list(out[i]) == philox4x32_10(ctr[i], key)


def test_uniform53_range_and_moments():
    ctr = np.zeros((100000, 4), np.uint32)
    ctr[:, 0] = np.arange(100000)
    u = uniform53(philox_array(ctr, (7, 11))[:, :2])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / 1e5)
    assert stats.kstest(u, "uniform").pvalue > 1e-4
