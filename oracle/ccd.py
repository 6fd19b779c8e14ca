"""Detector noise of the CCD object (App. A, Tab. 4; App. B, Listing 2:
``photon_noise``, ``readout_noise``, ``readout_level``, ``quantum_eff``) in
FP64, test infrastructure only.

Readings (the paper prints no noise model): the noise-free detector image
(summing to the number of pupil pixels) times ``scale`` = photons per frame x
quantum efficiency / pupil pixels gives each pixel's expected photo-electron
count lambda; the pixel reads k + ron g with k ~ Poisson(lambda) and g a
standard normal.  The draws come from Philox4x32-10 (see ``philox``) with the
counter (pixel, frame, block, stream) and key (seed low, seed high):

* lambda <= LAMBDA_SWITCH: k by the multiplicative method (Knuth, TAOCP
  vol. 2, 3.4.1): k is the number of uniforms u_0 u_1 ... whose running
  product stays above exp(-lambda), in float64, at most KMAX draws; uniform j
  is word j mod 4 of the block j // 4 of stream 2;
* lambda > LAMBDA_SWITCH: k = max(0, floor(lambda + sqrt(lambda) g0 + 1/2))
  (at most 2^31 - 1) with g0 the first Box-Muller normal of block 0 of
  stream 3;
* the readout normal g is the second normal of that block.

Both the integer decision and the sum are taken in float64; the result is
rounded once to float32.
"""
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


def _normals(pix, frame, seed):
    x = _block(pix, frame, 0, STREAM_NORMAL, seed)
    u0, u1 = uniform(x[0]), uniform(x[1])
    r = np.sqrt(-2.0 * np.log(u0))
    t = 2.0 * np.pi * u1
    return float(r * np.cos(t)), float(r * np.sin(t))


def poisson_count(lam: float, pix: int, frame: int, seed: int) -> int:
    """The photo-electron count of one pixel (see the module docstring)."""
    if lam > LAMBDA_SWITCH:
        g0, _ = _normals(pix, frame, seed)
        return min(max(0, int(np.floor(lam + np.sqrt(lam) * g0 + 0.5))), 2147483647)
    L = np.exp(-lam)
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
        _, g1 = _normals(pix, frame, seed)
        out[pix] = np.float32(float(k) + ron * g1)
    return out.reshape(np.shape(det))
