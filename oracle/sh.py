"""Shack-Hartmann spots (FP64).

Follows SH and the Lenslet / SubapData data objects (App. A, Tabs. 3-4); the
workload sizes follow Sect. 6, Tab. 2 (per-subaperture FFTs).  Reading (the
paper prints no formula): each valid subaperture's s x s block of the pupil
field is placed centred in an n x n zero grid (n = ``fft_n``, typically 2 s,
so the spot is Nyquist sampled: pixel = lambda / (2 d)); the spot is
    spot = |centred DFT of the padded block|^2 / n^2,
which sums to the block's sum |E|^2 (Parseval).  Spots are returned in the
order of the valid-subaperture list.
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
