"""Centred discrete Fourier transforms (FP64).

Both wavefront sensors image a pupil-plane field onto a focal plane and the
pyramid images it back (App. A, Tab. 4: ModulatedPyramid, SH).  The transforms
are taken on centred grids: for a side n, sample i sits at x_i = i - (n-1)/2
and frequency k at u_k = k - (n-1)/2, so that a real, centro-symmetric field
has a real, centro-symmetric spectrum and the spot of a flat wavefront sits
exactly between the four central pixels.  (Reading: the paper fixes no grid
convention.)

    F[v, u] = sum_{y, x} a[y, x] exp(-2 pi i (u x + v y) / n)
    a[y, x] = 1/n^2 sum_{v, u} F[v, u] exp(+2 pi i (u x + v y) / n)

The fast versions factor exp(-2 pi i (k - c)(i - c)/n), c = (n-1)/2, into an
input phase, an unshifted FFT, an output phase and a constant; ``numpy.fft``
is the library primitive.  ``brute_centred_dft2`` evaluates the sums as written
and exists only to pin the fast versions.
"""
import numpy as np


def centred_coords(n: int) -> np.ndarray:
    """x_i = i - (n-1)/2 for i = 0..n-1 (exact half-integers or integers)."""
    return np.arange(n, dtype=np.float64) - (n - 1) / 2.0


def _half_phase(n: int, sign: float) -> np.ndarray:
    """exp(sign * 2 pi i c k / n) for k = 0..n-1, c = (n-1)/2.

    2 c k / n = (n-1) k / n; the integer (n-1) k is reduced modulo 2n first so
    that the angle pi ((n-1) k mod 2n) / n stays below 2 pi.
    """
    k = np.arange(n, dtype=np.int64)
    red = ((n - 1) * k) % (2 * n)
    return np.exp(sign * 1j * np.pi * red.astype(np.float64) / n)


def _const_phase(n: int, sign: float) -> complex:
    """exp(sign * 2 pi i c^2 / n), c = (n-1)/2, i.e. angle pi (n-1)^2 / (2n)."""
    red = ((n - 1) * (n - 1)) % (4 * n)
    return np.exp(sign * 1j * np.pi * red / (2.0 * n))


def centred_dft2(a: np.ndarray) -> np.ndarray:
    """Forward centred 2-D DFT (unnormalised) of a square complex array."""
    n = a.shape[-1]
    assert a.shape[-2] == n
    p = _half_phase(n, +1.0)
    c = _const_phase(n, -1.0)
    f = np.fft.fft2(a * p[:, None] * p[None, :])
    return f * p[:, None] * p[None, :] * (c * c)


def centred_idft2(f: np.ndarray) -> np.ndarray:
    """Inverse centred 2-D DFT with the 1/n^2 normalisation."""
    n = f.shape[-1]
    assert f.shape[-2] == n
    q = _half_phase(n, -1.0)
    c = _const_phase(n, +1.0)
    a = np.fft.ifft2(f * q[:, None] * q[None, :])
    return a * q[:, None] * q[None, :] * (c * c)


def brute_centred_dft2(a: np.ndarray, inverse: bool = False) -> np.ndarray:
    """The defining double sum, O(n^4); tiny n only (pin for the fast path)."""
    n = a.shape[0]
    x = centred_coords(n)
    sign = 1.0 if inverse else -1.0
    out = np.zeros((n, n), dtype=np.complex128)
    for v in range(n):
        for u in range(n):
            acc = 0.0 + 0.0j
            for y in range(n):
                for xx in range(n):
                    ang = sign * 2.0 * np.pi * (x[u] * x[xx] + x[v] * x[y]) / n
                    acc += a[y, xx] * complex(np.cos(ang), np.sin(ang))
            out[v, u] = acc
    if inverse:
        out /= n * n
    return out
