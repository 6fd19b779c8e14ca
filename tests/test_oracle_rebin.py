"""Oracle pins: area-weighted detector rebinning (non-integer pixel ratio)."""
from fractions import Fraction

import numpy as np

from oracle import pyramid


def _overlap(a0, a1, b0, b1):
    return max(Fraction(0), min(a1, b1) - max(a0, b0))


def test_weights_against_exact_interval_overlaps():
    """Each weight is the overlap of [i, i+1) with [I n_in/n_out, (I+1)
    n_in/n_out), written with exact rational interval arithmetic."""
    for n_in, n_out in ((5, 3), (7, 4), (12, 5), (3, 7), (6, 6)):
        W = pyramid.rebin_weights(n_in, n_out)
        b = Fraction(n_in, n_out)
        for I in range(n_out):
            for i in range(n_in):
                assert W[I, i] == float(_overlap(Fraction(i), Fraction(i + 1), I * b, (I + 1) * b))


def test_integer_ratio_is_block_binning():
    rng = np.random.default_rng(1)
    img = rng.random((24, 24))
    for b in (1, 2, 3, 4, 6):
        assert np.allclose(pyramid.rebin_area(img, 24 // b), pyramid.bin_image(img, b),
                           rtol=1e-14, atol=0)


def test_flux_and_constant_image():
    rng = np.random.default_rng(2)
    img = rng.random((30, 30))
    for n_out in (7, 11, 13, 29, 45):
        D = pyramid.rebin_area(img, n_out)
        assert abs(D.sum() - img.sum()) <= 1e-12 * img.sum()
        C = pyramid.rebin_area(np.ones((30, 30)), n_out)
        assert np.allclose(C, (30 / n_out) ** 2, rtol=1e-13)


def test_point_source_spreads_by_overlap():
    """A single bright grid pixel lands in the detector pixels it overlaps,
    in proportion to the overlap areas."""
    img = np.zeros((5, 5))
    img[2, 3] = 1.0
    D = pyramid.rebin_area(img, 3)          # b = 5/3: pixel 2 splits 1/3 | 2/3 ... in y
    # y: grid row 2 = [2, 3) overlaps detector rows [5/3, 10/3) fully -> row 1 gets 1
    # x: grid column 3 = [3, 4) overlaps [5/3, 10/3) by 1/3 and [10/3, 5) by 2/3
    assert np.allclose(D, [[0, 0, 0], [0, 1 / 3, 2 / 3], [0, 0, 0]], atol=1e-15)
