"""Oracle pins: CCD photon and readout noise against Poisson / normal laws."""
import math

import numpy as np
import pytest

from oracle import ccd


@pytest.mark.parametrize("lam", [0.3, 3.0, 12.0, 29.5, 50.0, 400.0])
def test_poisson_moments(lam):
    """Mean lambda and variance lambda (both branches), within 5 standard
    errors over 4000 pixels."""
    n = 4000
    k = np.array([ccd.poisson_count(lam, p, 7, 12345) for p in range(n)], dtype=np.float64)
    assert abs(k.mean() - lam) < 5 * math.sqrt(lam / n)
    # standard error of the sample variance of a Poisson variable
    se_var = math.sqrt((lam + 2 * lam * lam) / n)
    assert abs(k.var() - lam) < 5 * se_var
    assert np.all(k == np.round(k)) and k.min() >= 0


def test_zero_probability_and_zero_flux():
    lam, n = 0.7, 6000
    k = np.array([ccd.poisson_count(lam, p, 3, 99) for p in range(n)])
    p0 = math.exp(-lam)
    assert abs((k == 0).mean() - p0) < 5 * math.sqrt(p0 * (1 - p0) / n)
    assert all(ccd.poisson_count(0.0, p, 3, 99) == 0 for p in range(200))


def test_readout_noise_and_determinism():
    det = np.zeros((40, 40), dtype=np.float32)
    a = ccd.ccd_read(det, 1.0, 2.5, 77, 0).astype(np.float64)
    assert abs(a.mean()) < 5 * 2.5 / 40 and abs(a.std() - 2.5) < 5 * 2.5 / math.sqrt(2 * 1600)
    assert np.array_equal(a, ccd.ccd_read(det, 1.0, 2.5, 77, 0))
    assert not np.array_equal(a, ccd.ccd_read(det, 1.0, 2.5, 77, 1))
    b = ccd.ccd_read(np.full((8, 8), 5.0, dtype=np.float32), 2.0, 0.0, 77, 0)
    assert np.all(b == np.round(b))


def test_branch_switch_is_continuous_in_law():
    """Just below and above the switch the two samplers agree in mean and
    variance (the normal branch approximates Poisson(lambda) at large lambda)."""
    n = 4000
    lo = np.array([ccd.poisson_count(29.9, p, 1, 5) for p in range(n)], dtype=np.float64)
    hi = np.array([ccd.poisson_count(30.1, p, 1, 5) for p in range(n)], dtype=np.float64)
    assert abs(lo.mean() - hi.mean()) < 0.2 + 5 * math.sqrt(2 * 30 / n)
    assert abs(lo.var() - hi.var()) < 5 * math.sqrt(2 * (30 + 2 * 900) / n)


def test_exp_threshold_accuracy():
    """The float32 threshold T(lambda/64)^64 against exp(-lambda): relative
    error below 1e-5 over [0, 30] (it only shifts Poisson probabilities)."""
    for lam in np.linspace(0.0, 30.0, 301):
        v = float(ccd.exp_neg_f32(lam))
        assert abs(v / math.exp(-lam) - 1.0) < 1e-5, lam


def test_irwin_hall_moments():
    g = np.array([ccd.irwin_hall(p, 2, 11, 0) for p in range(6000)])
    assert abs(g.mean()) < 5 / math.sqrt(6000)
    assert abs(g.var() - 1.0) < 5 * math.sqrt(2.0 / 6000)
    assert np.abs(g).max() <= 6.0
