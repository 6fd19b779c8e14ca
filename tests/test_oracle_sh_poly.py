"""Oracle pins of the polychromatic Shack-Hartmann reading: the overlap
matrix against a brute-force count on a common refinement of both pixel
lattices, the monochromatic case, flux conservation of a spot inside the
window, and the spot width scaling with wavelength."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import geometry, sh


def _weights_brute(n, r: Fraction):
    """Count cells of side h = 1 / (2 p) (r = p / q): every boundary of both
    lattices, o - n/2 +- 1/2 and (j - n/2 +- 1/2) q / p, is a multiple of h."""
    p, q = r.numerator, r.denominator
    h = Fraction(1, 2 * p)
    lo_all = min(Fraction(-n, 2) - Fraction(1, 2), (Fraction(-n, 2) - Fraction(1, 2)) / r)
    hi_all = max(Fraction(n, 2) + Fraction(1, 2), (Fraction(n, 2) + Fraction(1, 2)) / r)
    W = np.zeros((n, n))
    k0, k1 = int(lo_all / h) - 1, int(hi_all / h) + 1
    for k in range(k0, k1):
        c = (k + Fraction(1, 2)) * h                       # cell centre
        o = c + Fraction(n, 2) + Fraction(1, 2)            # detector pixel: floor(o)
        j = c * r + Fraction(n, 2) + Fraction(1, 2)        # spot pixel: floor(j)
        oi, ji = int(np.floor(float(o))), int(np.floor(float(j)))
        if 0 <= oi < n and 0 <= ji < n:
            W[oi, ji] += float(h)
    return W


@pytest.mark.parametrize("n,r", [(16, Fraction(2)), (16, Fraction(2, 3)), (24, Fraction(3, 2)),
                                 (24, Fraction(5, 4)), (16, Fraction(1))])
def test_weights_against_refinement(n, r):
    assert np.allclose(sh.poly_weights(n, float(r)), _weights_brute(n, r), rtol=0, atol=1e-12)


def _case(n_sub=6, sub_pix=8, fft_n=16, seed=3):
    n = n_sub * sub_pix
    amp = geometry.pupil_mask(n, 0.0).astype(np.float64)
    valid = geometry.valid_subaps(amp.astype(np.uint8), n_sub)
    ph = np.random.default_rng(seed).standard_normal((n, n)) * 0.3
    return amp, ph, valid, n_sub, sub_pix, fft_n


def test_single_reference_band_is_the_mono_spots():
    amp, ph, valid, ns, sp_, nf = _case()
    mono = sh.sh_spots(amp, ph, ns, sp_, nf, valid)
    assert np.array_equal(sh.sh_spots_poly(amp, ph, ns, sp_, nf, valid, [1.0], [1.0]), mono)
    # weights are linear
    two = sh.sh_spots_poly(amp, ph, ns, sp_, nf, valid, [1.0, 1.0], [0.25, 0.5])
    assert np.allclose(two, 0.75 * mono, rtol=1e-15, atol=0)


def test_flux_of_a_uniform_spot():
    """A uniform spot of n^2 pixels at r = 1.5 covers n / 1.5 reference
    pixels: the detector holds all of its flux, interior pixels r^2 each."""
    n, r = 24, 1.5
    W = sh.poly_weights(n, r)
    D = r * r * W @ np.ones((n, n)) @ W.T
    assert abs(D.sum() - n * n) < 1e-9
    assert np.allclose(D[n // 2 - 4:n // 2 + 4, n // 2 - 4:n // 2 + 4], r * r)


def test_flat_wavefront_spot_width_scales_with_wavelength():
    """A flat subaperture's spot at a shorter wavelength (r > 1) is narrower
    on the detector by about 1 / r and keeps its flux."""
    amp, _, valid, ns, sp_, nf = _case(n_sub=4, sub_pix=12, fft_n=24)
    flat = np.zeros_like(amp)
    ref = sh.sh_spots(amp, flat, ns, sp_, nf, valid)
    blue = sh.sh_spots_poly(amp, flat, ns, sp_, nf, valid, [1.5], [1.0])
    x = np.arange(nf) - nf / 2.0

    def width(s):
        m = s.sum(axis=0)                       # profile along x
        return np.sqrt((m * x * x).sum() / m.sum())

    k = len(valid) // 2
    assert abs(blue[k].sum() - ref[k].sum()) < 1e-3 * ref[k].sum()
    assert 0.55 < width(blue[k]) / width(ref[k]) < 0.8
