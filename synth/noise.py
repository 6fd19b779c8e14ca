"""Seeded random draws (NumPy PCG64).  No simulation arithmetic lives here."""
import numpy as np


def screen_noise(seed: int, side: int) -> np.ndarray:
    """Complex white noise for one FFT phase screen.

    Returns a (side, side) complex128 array c with Re c and Im c independent
    standard normals, drawn as two C-ordered (side, side) blocks (real part
    first) from ``numpy.random.default_rng(seed)``.  Element [ky, kx] belongs to
    the spatial-frequency sample with FFT indices (ky, kx).
    """
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((side, side))
    im = rng.standard_normal((side, side))
    return re + 1j * im


def subharmonic_noise(seed: int, levels: int = 3) -> np.ndarray:
    """Complex noise for the subharmonic frequencies of one screen.

    Shape (levels, 3, 3) complex128, element [p, b, a] for level p+1 and the
    frequency offset (a-1, b-1) in units of that level's spacing.  Drawn from a
    generator seeded with ``seed + 7919`` so that it is independent of
    :func:`screen_noise` for the same seed.
    """
    rng = np.random.default_rng(seed + 7919)
    re = rng.standard_normal((levels, 3, 3))
    im = rng.standard_normal((levels, 3, 3))
    return re + 1j * im


def uniform_draws(seed: int, shape, low=0.0, high=1.0) -> np.ndarray:
    """Float64 uniform draws in [low, high) from PCG64(seed)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(low, high, size=shape)


def normal_draws(seed: int, shape) -> np.ndarray:
    """Float64 standard-normal draws from PCG64(seed)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=shape)
