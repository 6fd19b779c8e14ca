"""Detector noise of the CCD object (App. A, Tab. 4; App. B, Listing 2:
``photon_noise``, ``readout_noise``, ``readout_level``, ``quantum_eff``) in
FP64, test infrastructure only.

Readings (the paper prints no noise model): the noise-free detector image
(summing to the number of pupil pixels) times ``scale`` = photons per frame x
quantum efficiency / pupil pixels gives each pixel's expected photo-electron
count lambda; the pixel reads k + ron g with k ~ Poisson(lambda) and g a
standard normal.  The draws come from Philox4x32-10 (see ``philox``) with the
counter (pixel, frame, block, stream) and key (seed low, seed high).  Every
step is a chain of IEEE basic operations (no library function), so a
reimplementation with the same operations decides the same counts:

* lambda <= LAMBDA_SWITCH: k by the multiplicative method (Knuth, TAOCP
  vol. 2, 3.4.1): k is the number of uniforms u_0 u_1 ... (each rounded to
  float32) whose running float32 product stays above L, at most KMAX draws;
  uniform j is word j mod 4 of the block j // 4 of stream 2;
  L = exp(-lambda) as (T(lambda / 64))^64 in float32, T the degree-9 Taylor
  polynomial of exp(-x) by Horner's rule (relative error ~4e-6 at lambda =
  30, which shifts the Poisson probabilities by as much);
* lambda > LAMBDA_SWITCH: k = max(0, floor(lambda + sqrt(lambda) g0 + 1/2))
  in float64, g0 an Irwin-Hall normal: the sum of the twelve uniforms of
  blocks 0-2 of stream 3, minus 6 (mean 0, variance 1, tails cut at 6);
* the readout normal g is the Irwin-Hall normal of blocks 3-5 of stream 3.

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


_TAYLOR = [np.float32(1.0 / math.factorial(k)) for k in range(10)]


def exp_neg_f32(lam: float) -> np.float32:
    """exp(-lambda) for 0 <= lambda <= 30: float32 Horner evaluation of the
    degree-9 Taylor polynomial at x = lambda / 64, then six squarings."""
    x = np.float32(np.float32(lam) / np.float32(64.0))
    p = _TAYLOR[9]
    for k in range(8, -1, -1):
        p = np.float32(np.float32(p * -x) + _TAYLOR[k])
    for _ in range(6):
        p = np.float32(p * p)
    return p


def irwin_hall(pix, frame, seed, first_block):
    """Sum of the twelve uniforms of blocks first_block .. +2 of stream 3,
    minus 6, in float64, left to right."""
    acc = 0.0
    for b in range(3):
        for w in _block(pix, frame, first_block + b, STREAM_NORMAL, seed):
            acc = acc + float(uniform(w))
    return acc - 6.0


def poisson_count(lam: float, pix: int, frame: int, seed: int) -> int:
    """The photo-electron count of one pixel (see the module docstring)."""
    if lam > LAMBDA_SWITCH:
        g0 = irwin_hall(pix, frame, seed, 0)
        return min(max(0, int(np.floor(lam + np.sqrt(lam) * g0 + 0.5))), 2147483647)
    L = exp_neg_f32(lam)
    p = np.float32(1.0)
    k = 0
    words = None
    for j in range(KMAX + 1):
        if j % 4 == 0:
            words = _block(pix, frame, j // 4, STREAM_KNUTH, seed)
        p = np.float32(p * np.float32(uniform(words[j % 4])))
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
        rd = ron * irwin_hall(pix, frame, seed, 3) if ron > 0 else 0.0
        out[pix] = np.float32(float(k) + rd)
    return out.reshape(np.shape(det))
