"""Shack-Hartmann spots (FP64).

Follows SH and the Lenslet / SubapData data objects (App. A, Tabs. 3-4); the
workload sizes follow Sect. 6, Tab. 2 (per-subaperture FFTs).  Reading (the
paper prints no formula): each valid subaperture's s x s block of the pupil
field is placed centred in an n x n zero grid (n = ``fft_n``, typically 2 s,
so the spot is Nyquist sampled: pixel = lambda / (2 d)); the spot is
    spot = |centred DFT of the padded block|^2 / n^2,
which sums to the block's sum |E|^2 (Parseval).  Spots are returned in the
order of the valid-subaperture list.

Polychromatic spots (PolyChromSH, App. A, Tab. 4, named only; reading): the
spots of wavelength lambda_i are the monochromatic spots with the phase
scaled by r = lambda_ref / lambda_i at the same n, so a spot pixel is
lambda_i / (n d) = 1 / r reference pixels.  The detector, whose pixels are
the reference spot pixels, integrates each wavelength's spot taken as
constant over its own pixels: with W[o, j] the length of reference pixel o,
[o - n/2 - 1/2, o - n/2 + 1/2), inside spot pixel j, [(j - n/2 - 1/2) / r,
(j - n/2 + 1/2) / r) (both lattices centred on the zero frequency), the
wavelength contributes weight r^2 W S W^T (r^2: a spot pixel's value spread
over its area 1 / r^2).  Light outside a subaperture's n x n window is
dropped (a field stop per subaperture).
"""
import numpy as np

from .dft import centred_dft2


def sh_spots(amp: np.ndarray, phase: np.ndarray, n_sub: int, sub_pix: int,
             fft_n: int, valid: np.ndarray) -> np.ndarray:
    """(n_valid, fft_n, fft_n) float64 spot images."""
    s, n = sub_pix, fft_n
    assert amp.shape[0] == n_sub * s
    off = (n - s) // 2
    E = amp * np.exp(1j * phase)
    out = np.zeros((len(valid), n, n))
    for k, idx in enumerate(valid):
        a, b = divmod(int(idx), n_sub)
        P = np.zeros((n, n), dtype=np.complex128)
        P[off:off + s, off:off + s] = E[a * s:(a + 1) * s, b * s:(b + 1) * s]
        out[k] = np.abs(centred_dft2(P)) ** 2 / (n * n)
    return out


def poly_weights(n: int, r: float) -> np.ndarray:
    """W[o, j]: overlap of reference pixel o with the spot pixel j of a
    wavelength whose pixel is 1 / r reference pixels (float64)."""
    o = np.arange(n)[:, None] - n / 2.0
    j = np.arange(n)[None, :] - n / 2.0
    lo = np.maximum(o - 0.5, (j - 0.5) / r)
    hi = np.minimum(o + 0.5, (j + 0.5) / r)
    return np.maximum(hi - lo, 0.0)


def sh_spots_poly(amp, phase, n_sub, sub_pix, fft_n, valid, ratios, weights):
    """Weighted sum over wavelengths of the spots integrated on the reference
    lattice: sum_i w_i r_i^2 W_i S_i W_i^T."""
    out = np.zeros((len(valid), fft_n, fft_n))
    for r, w in zip(ratios, weights):
        S = sh_spots(amp, np.asarray(phase, dtype=np.float64) * r, n_sub, sub_pix, fft_n, valid)
        W = poly_weights(fft_n, r)
        out += w * r * r * np.einsum("oj,kjl,pl->kop", W, S, W)
    return out
