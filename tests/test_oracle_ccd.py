"""Oracle pins: CCD photon and readout noise against the Poisson and normal
laws the model states (moments, zero-count probability, chi-squared against
the probability mass functions, Kolmogorov-Smirnov for the readout normal)."""
import math

import numpy as np
import pytest

from oracle import ccd


def _counts(lam, n, frame, seed):
    return np.array([ccd.poisson_count(lam, p, frame, seed) for p in range(n)], dtype=np.int64)


def _chi2_pvalue(k, pmf, kmax):
    """Chi-squared test of integer samples k against pmf(0..kmax); bins with
    fewer than 5 expected samples are merged into their neighbours."""
    from scipy import stats
    n = k.size
    probs = np.array([pmf(j) for j in range(kmax + 1)])
    probs = np.append(probs, max(0.0, 1.0 - probs.sum()))        # the tail above kmax
    obs = np.bincount(np.minimum(k, kmax + 1), minlength=kmax + 2).astype(np.float64)
    exp_, ob, acc_e, acc_o = [], [], 0.0, 0.0
    for e, o in zip(probs * n, obs):
        acc_e += e
        acc_o += o
        if acc_e >= 5.0:
            exp_.append(acc_e)
            ob.append(acc_o)
            acc_e = acc_o = 0.0
    exp_[-1] += acc_e
    ob[-1] += acc_o
    exp_, ob = np.array(exp_), np.array(ob)
    chi2 = float(((ob - exp_) ** 2 / exp_).sum())
    return float(stats.chi2.sf(chi2, len(exp_) - 1))


def _poisson_pmf(lam):
    return lambda j: math.exp(-lam + j * math.log(lam) - math.lgamma(j + 1)) if lam > 0 else float(j == 0)


def _rounded_normal_pmf(lam):
    """P(floor(lam + sqrt(lam) g + 1/2) = j), g standard normal (j >= 1; j = 0
    takes the whole lower tail)."""
    s = math.sqrt(lam)
    cdf = lambda x: 0.5 * math.erfc(-x / math.sqrt(2.0))
    return lambda j: (cdf((j + 0.5 - lam) / s) - (cdf((j - 0.5 - lam) / s) if j > 0 else 0.0))


@pytest.mark.parametrize("lam", [0.3, 3.0, 12.0, 29.5, 50.0, 400.0])
def test_poisson_moments(lam):
    """Mean lambda and variance lambda (both branches), within 5 standard
    errors over 4000 pixels."""
    n = 4000
    k = _counts(lam, n, 7, 12345).astype(np.float64)
    assert abs(k.mean() - lam) < 5 * math.sqrt(lam / n)
    # standard error of the sample variance of a Poisson variable
    se_var = math.sqrt((lam + 2 * lam * lam) / n)
    assert abs(k.var() - lam) < 5 * se_var
    assert k.min() >= 0


@pytest.mark.parametrize("lam", [0.3, 3.0, 12.0, 29.5])
def test_multiplicative_branch_is_poisson(lam):
    """The multiplicative method draws exactly from Poisson(lambda): chi-squared
    against the Poisson mass function over 4000 pixels.  An off-by-one in the
    count, a non-strict comparison or a wrong threshold shifts the law by a
    whole unit and fails this."""
    k = _counts(lam, 4000, 2, 777)
    assert _chi2_pvalue(k, _poisson_pmf(lam), int(lam + 8 * math.sqrt(lam) + 8)) > 1e-3


@pytest.mark.parametrize("lam", [45.0, 400.0])
def test_normal_branch_is_the_rounded_normal(lam):
    """Above the switch the count is the rounded normal of mean and variance
    lambda: chi-squared against that law."""
    k = _counts(lam, 4000, 2, 4242)
    assert _chi2_pvalue(k, _rounded_normal_pmf(lam), int(lam + 6 * math.sqrt(lam))) > 1e-3


def test_zero_probability_and_zero_flux():
    lam, n = 0.7, 6000
    k = _counts(lam, n, 3, 99)
    p0 = math.exp(-lam)
    assert abs((k == 0).mean() - p0) < 5 * math.sqrt(p0 * (1 - p0) / n)
    assert all(ccd.poisson_count(0.0, p, 3, 99) == 0 for p in range(200))


def test_readout_noise_is_standard_normal():
    """On a dark detector the read is ron g: moments, and a Kolmogorov-Smirnov
    test of g against the standard normal."""
    from scipy import stats
    ron = 2.5
    det = np.zeros((60, 60), dtype=np.float32)
    a = ccd.ccd_read(det, 1.0, ron, 77, 0).astype(np.float64)
    g = a.ravel() / ron
    assert abs(g.mean()) < 5 / 60 and abs(g.std() - 1.0) < 5 / math.sqrt(2 * 3600)
    assert stats.kstest(g, "norm").pvalue > 1e-3


def test_readout_and_photon_noise_add():
    det = np.full((30, 30), 4.0, dtype=np.float32)
    a = ccd.ccd_read(det, 2.0, 1.5, 5, 1).astype(np.float64)
    k = np.array([ccd.poisson_count(8.0, p, 1, 5) for p in range(900)], dtype=np.float64)
    g = np.array([ccd.normals(p, 1, 5)[1] for p in range(900)])
    assert np.all(np.abs(a.ravel() - (k + 1.5 * g)) <= 2.0 ** -23 * np.abs(k + 1.5 * g))


def test_determinism_and_frames():
    det = np.full((8, 8), 5.0, dtype=np.float32)
    a = ccd.ccd_read(det, 2.0, 0.0, 77, 0)
    assert np.array_equal(a, ccd.ccd_read(det, 2.0, 0.0, 77, 0))
    assert not np.array_equal(a, ccd.ccd_read(det, 2.0, 0.0, 77, 1))
    assert np.all(a == np.round(a))


def test_branch_switch_is_continuous_in_law():
    """Just below and above the switch the two samplers agree in mean and
    variance (the normal branch approximates Poisson(lambda) at large lambda)."""
    n = 4000
    lo = _counts(29.9, n, 1, 5).astype(np.float64)
    hi = _counts(30.1, n, 1, 5).astype(np.float64)
    assert abs(lo.mean() - hi.mean()) < 0.2 + 5 * math.sqrt(2 * 30 / n)
    assert abs(lo.var() - hi.var()) < 5 * math.sqrt(2 * (30 + 2 * 900) / n)


def test_box_muller_pair_definition():
    """The pair is the polar form of two independent normals: r^2 = -2 ln u0
    is exponential with mean 2 and the angle is uniform (checked on 3000
    pixels)."""
    from scipy import stats
    pairs = np.array([ccd.normals(p, 9, 31) for p in range(3000)])
    r2 = (pairs ** 2).sum(axis=1)
    assert stats.kstest(r2, "expon", args=(0, 2.0)).pvalue > 1e-3
    ang = np.arctan2(pairs[:, 1], pairs[:, 0])
    assert stats.kstest(ang, "uniform", args=(-math.pi, 2 * math.pi)).pvalue > 1e-3
