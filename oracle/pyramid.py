"""Modulated four-face pyramid wavefront sensor (FP64).

Follows ModulatedPyramid (App. A, Tab. 4) with the parameters of App. B,
Listing 2 (``pup_diam``, ``pup_dist``, ``mod_amp`` in lambda/D,
``output_resolution``) and the CCD integration with noise off (Listing 2:
``photon_noise``/``readout_noise`` False).  Step order per frame, for each
modulation point m = 0..n_mod-1:

  1. tilt:  E_m(x, y) = A exp(i phi) exp(2 pi i r (x cos t_m + y sin t_m) / Np)
     with x, y the centred pupil coordinates in pixels and r = ``mod_amp``
     (a tilt of r cycles across the pupil moves the focal spot by r lambda/D);
  2. pad:   place E_m centred in an N x N zero grid, N = pad * Np;
  3. FFT:   F = centred forward DFT (unnormalised);
  4. mask:  F(u, v) *= exp(-2 pi i c (|u| + |v|) / N), c = pup_dist / 2, so each
            face adds the tilt that moves its pupil image by (+-c, +-c) pixels;
            the (+, +) face images into the (+x, +y) quadrant;
  5. IFFT:  O = centred inverse DFT (1/N^2);
  6. accumulate I += |O|^2 / n_mod.
Then the N x N intensity is binned in b x b blocks, b = Np / n_sub, to the
pad n_sub detector (area-weighted rebinning where b is fractional, see
``detector``).

Readings (the paper prints no formula): centred grids (see ``dft``); amplitude
1 per in-pupil pixel, so the detector sums to the number of pupil pixels;
pup_dist = Np so the four images tile the padded grid exactly.

Shifted-mask form (a second discretisation of the same modulation).  The
tilt of step 1 is exp(2 pi i (s_x x + s_y y) / N) on the padded grid, with
s = r pad (cos t_m, sin t_m) frequency bins, so the spectrum of step 3 is the
field's spectrum moved by s.  Moving the mask instead, by -s, gives the same
image up to a phase that vanishes in |O|^2:

  F = centred DFT of the padded field (once per frame);
  O_m = centred inverse DFT of M(u + s_x, v + s_y) F(u, v);
  I = sum over m of |O_m|^2 / n_mod,

with M the analytic mask exp(-2 pi i c (|u + s_x| + |v + s_y|) / N)
evaluated at the shifted frequencies.  The two forms agree exactly when the
field's spectrum vanishes wherever u + s_x or v + s_y leaves the centred
frequency range (whole-bin shifts of a band-limited field); for a pupil-
limited field they differ where the spectrum wraps: the shifted form applies
the non-periodic mask to the spectrum's far wings instead of wrapping them.
"""
import numpy as np

from .dft import centred_coords, centred_dft2, centred_idft2
from .geometry import mod_angles


def pyramid_mask(N: int, pup_dist: float) -> np.ndarray:
    """exp(-2 pi i c (|u| + |v|) / N) on the centred N x N frequency grid."""
    c = pup_dist / 2.0
    u = np.abs(centred_coords(N))
    m1 = np.exp(-2j * np.pi * c * u / N)
    return m1[:, None] * m1[None, :]


def pwfs_intensity(amp: np.ndarray, phase: np.ndarray, pad: int, n_mod: int,
                   mod_amp: float, pup_dist: float, mask=None, points=None) -> np.ndarray:
    """Modulation-averaged N x N intensity (steps 1-6).  points: the subset of
    modulation points to image (None: all); the sum is still divided by
    n_mod, so subsets that partition the points add up to the full image."""
    Np = amp.shape[0]
    N = pad * Np
    off = (N - Np) // 2
    x = centred_coords(Np)
    E = amp * np.exp(1j * phase)
    M = pyramid_mask(N, pup_dist) if mask is None else mask
    cs, sn = mod_angles(n_mod)
    I = np.zeros((N, N))
    for m in (range(n_mod) if points is None else points):
        tilt = np.exp(2j * np.pi * mod_amp
                      * (x[None, :] * cs[m] + x[:, None] * sn[m]) / Np)
        P = np.zeros((N, N), dtype=np.complex128)
        P[off:off + Np, off:off + Np] = E * tilt
        O = centred_idft2(centred_dft2(P) * M)
        I += np.abs(O) ** 2
    return I / n_mod


def bin_image(I: np.ndarray, b: int) -> np.ndarray:
    """Sum of b x b blocks (CCD binning, noise off)."""
    n = I.shape[0]
    assert n % b == 0
    k = n // b
    return I.reshape(k, b, k, b).sum(axis=(1, 3))


def rebin_weights(n_in: int, n_out: int) -> np.ndarray:
    """W[I, i] = length of [i, i + 1) inside [I b, (I + 1) b), b = n_in / n_out
    (grid-pixel units): the share of grid pixel i that detector pixel I
    collects.  Computed exactly in units of 1 / n_out, then divided."""
    I = np.arange(n_out)[:, None]
    i = np.arange(n_in)[None, :]
    lo = np.maximum(i * n_out, I * n_in)
    hi = np.minimum((i + 1) * n_out, (I + 1) * n_in)
    return np.maximum(hi - lo, 0).astype(np.float64) / n_out


def rebin_area(img: np.ndarray, n_out: int) -> np.ndarray:
    """Area-weighted rebinning of a square image (n_in x n_in, intensity
    constant over each grid pixel) to n_out x n_out detector pixels that tile
    the same field: D = W img W^T.  Flux is kept; an integer ratio is b x b
    binning.  This is the detector sampling a pyramid's output_resolution
    asks for when it is not a whole fraction of the padded grid (Listing 2)."""
    W = rebin_weights(img.shape[-1], n_out)
    return W @ np.asarray(img, dtype=np.float64) @ W.T


def detector(I: np.ndarray, n_det: int) -> np.ndarray:
    """The N x N intensity sampled onto the n_det x n_det detector: b x b
    binning for a whole ratio b = N / n_det, area-weighted rebinning
    otherwise (a pixel of Np / n_sub grid pixels, e.g. 220 / 40 = 5.5 for
    the SOUL example's output_resolution 120 on a 660 grid)."""
    N = I.shape[0]
    return bin_image(I, N // n_det) if N % n_det == 0 else rebin_area(I, n_det)


def pwfs_image(amp, phase, pad, n_mod, mod_amp, n_sub, pup_dist):
    """Detector image pad n_sub x pad n_sub (2 n_sub x 2 n_sub with pad = 2
    and pup_dist = Np, the quadrant layout)."""
    I = pwfs_intensity(amp, phase, pad, n_mod, mod_amp, pup_dist)
    return detector(I, pad * n_sub)


def shift_bins(n_mod: int, mod_amp: float, pad: int):
    """Spectrum shift of each modulation point in frequency bins:
    s = r pad (cos t_m, sin t_m) (a tilt of r cycles across Np pupil pixels
    is r pad cycles across the N = pad Np grid)."""
    cs, sn = mod_angles(n_mod)
    return mod_amp * pad * cs, mod_amp * pad * sn


def tilted_intensity(P: np.ndarray, sx, sy, pup_dist: float) -> np.ndarray:
    """Steps 1-6 on a padded N x N field P: per point, the tilt
    exp(2 pi i (s_x x + s_y y) / N) on the centred grid, DFT, mask, inverse
    DFT, |.|^2, averaged over the points."""
    N = P.shape[0]
    x = centred_coords(N)
    M = pyramid_mask(N, pup_dist)
    I = np.zeros((N, N))
    for a, b in zip(sx, sy):
        tilt = np.exp(2j * np.pi * (x[None, :] * a + x[:, None] * b) / N)
        I += np.abs(centred_idft2(centred_dft2(P * tilt) * M)) ** 2
    return I / len(sx)


def shifted_mask(N: int, pup_dist: float, sx: float, sy: float) -> np.ndarray:
    """exp(-2 pi i c (|u + s_x| + |v + s_y|) / N) on the centred grid."""
    c = pup_dist / 2.0
    u = centred_coords(N)
    mx = np.exp(-2j * np.pi * c * np.abs(u + sx) / N)
    my = np.exp(-2j * np.pi * c * np.abs(u + sy) / N)
    return my[:, None] * mx[None, :]


def shifted_mask_intensity(P: np.ndarray, sx, sy, pup_dist: float) -> np.ndarray:
    """Shifted-mask form on a padded field: one DFT, then per point the mask
    at the shifted frequencies, inverse DFT, |.|^2, averaged."""
    N = P.shape[0]
    F = centred_dft2(P)
    I = np.zeros((N, N))
    for a, b in zip(sx, sy):
        I += np.abs(centred_idft2(F * shifted_mask(N, pup_dist, a, b))) ** 2
    return I / len(sx)


def pwfs_intensity_shifted(amp, phase, pad, n_mod, mod_amp, pup_dist) -> np.ndarray:
    """Modulation-averaged N x N intensity in the shifted-mask form."""
    Np = amp.shape[0]
    N = pad * Np
    off = (N - Np) // 2
    P = np.zeros((N, N), dtype=np.complex128)
    P[off:off + Np, off:off + Np] = amp * np.exp(1j * phase)
    sx, sy = shift_bins(n_mod, mod_amp, pad)
    return shifted_mask_intensity(P, sx, sy, pup_dist)


def pwfs_image_shifted(amp, phase, pad, n_mod, mod_amp, n_sub, pup_dist):
    """Detector image of the shifted-mask form."""
    Np = amp.shape[0]
    I = pwfs_intensity_shifted(amp, phase, pad, n_mod, mod_amp, pup_dist)
    return bin_image(I, Np // n_sub)


def pwfs_image_poly(amp, phase, pad, n_mod, mod_amp, n_sub, pup_dist, ratios, weights):
    """Polychromatic image (PolyCromPyramid, App. A, Tab. 4): the weighted sum
    over wavelengths of the monochromatic image, phase and modulation radius
    (in lambda / D) scaled by ratio = lambda_ref / lambda_i; the pupil
    images' separation is geometric (the same at every wavelength).
    Reading: the paper gives the object, not its model."""
    det = None
    for r, w in zip(ratios, weights):
        d = w * pwfs_image(amp, phase * r, pad, n_mod, mod_amp * r, n_sub, pup_dist)
        det = d if det is None else det + d
    return det
