"""Detector noise of the CCD object (App. A, Tab. 4; App. B, Listing 2:
``photon_noise``, ``readout_noise``, ``readout_level``, ``quantum_eff``) in
FP64.  Test infrastructure only: the product path never imports this module.

Readings (the paper prints no noise model): the noise-free detector image
(summing to the number of pupil pixels) times ``scale`` = photons per frame x
quantum efficiency / pupil pixels gives each pixel's expected photo-electron
count lambda; the pixel reads k + ron g with k ~ Poisson(lambda) and g a
standard normal.  The draws come from Philox4x32-10 (see ``philox``) with the
counter (pixel, frame, block, stream) and key (seed low, seed high); the
uniform of a word x is (x + 1/2) / 2^32.

* lambda <= LAMBDA_SWITCH: k by the multiplicative method (Knuth, TAOCP
  vol. 2, 3.4.1): k is the number of uniforms u_0, u_1, ... whose running
  product stays above exp(-lambda), at most KMAX draws; uniform j is word
  j mod 4 of block j // 4 of stream 2.  Everything in float64.
* lambda > LAMBDA_SWITCH: the normal approximation of the Poisson law,
  rounded: k = max(0, floor(lambda + sqrt(lambda) g0 + 1/2)), g0 the first
  Box-Muller normal of block 0 of stream 3.
* the readout normal g is the second Box-Muller normal of that block:
  (g0, g) = sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1) with u0, u1 the
  uniforms of its words 0 and 1.

k + ron g is summed in float64 and rounded once to float32.
"""
import math

import numpy as np

from .philox import philox4x32_10, uniform

LAMBDA_SWITCH = 30.0
KMAX = 1000
STREAM_KNUTH = 2
STREAM_NORMAL = 3


def _block(pix, frame, block, stream, seed):
    seed = int(seed)
    c = [np.array([v], dtype=np.uint32) for v in (pix, frame, block, stream)]
    x = philox4x32_10(*c, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return [w[0] for w in x]


def normals(pix: int, frame: int, seed: int):
    """The Box-Muller pair of block 0 of stream 3 (float64)."""
    x = _block(pix, frame, 0, STREAM_NORMAL, seed)
    u0, u1 = float(uniform(x[0])), float(uniform(x[1]))
    r = math.sqrt(-2.0 * math.log(u0))
    t = 2.0 * math.pi * u1
    return r * math.cos(t), r * math.sin(t)


def poisson_count(lam: float, pix: int, frame: int, seed: int) -> int:
    """The photo-electron count of one pixel (see the module docstring)."""
    if lam > LAMBDA_SWITCH:
        g0, _ = normals(pix, frame, seed)
        return min(max(0, int(math.floor(lam + math.sqrt(lam) * g0 + 0.5))), 2147483647)
    L = math.exp(-lam)
    p = 1.0
    k = 0
    words = None
    for j in range(KMAX + 1):
        if j % 4 == 0:
            words = _block(pix, frame, j // 4, STREAM_KNUTH, seed)
        p *= float(uniform(words[j % 4]))
        if not p > L:
            break
        k += 1
    return min(k, KMAX)


def ccd_read(det: np.ndarray, scale: float, ron: float, seed: int, frame: int) -> np.ndarray:
    """Noisy read of a detector image (float32 out)."""
    flat = np.asarray(det).ravel()
    out = np.empty(flat.size, dtype=np.float32)
    for pix in range(flat.size):
        lam = float(flat[pix]) * scale
        k = poisson_count(lam, pix, frame, seed)
        rd = ron * normals(pix, frame, seed)[1] if ron > 0 else 0.0
        out[pix] = np.float32(float(k) + rd)
    return out.reshape(np.shape(det))
