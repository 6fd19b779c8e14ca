"""Modal basis and modal projection (FP64).

Follows the modal objects of the paper — ModalAnalysis (projects a wavefront
onto modes), IFunc / M2C and the KL basis of the SOUL example (App. A,
Tabs. 3-4; App. B, Listing 2 `ifunc_inv_object`, `ifunc_object`).  The KL
basis files are not public (paper, "Code and Data Availability"), so the
reading here is a Zernike basis in Noll order without piston, j = 2 ..
n_modes + 1:

    Z_j(rho, theta) = sqrt(n + 1) R_n^0(rho)                 (m = 0)
                    = sqrt(2 (n + 1)) R_n^|m|(rho) cos(|m| theta)   (m != 0, j even)
                    = sqrt(2 (n + 1)) R_n^|m|(rho) sin(|m| theta)   (m != 0, j odd)
    R_n^m(rho) = sum_{s=0}^{(n-m)/2} (-1)^s (n-s)! / (s! ((n+m)/2-s)! ((n-m)/2-s)!) rho^(n-2s)

sampled at pupil pixel centres, rho = |(x, y)| / (n_pix / 2) with centred
pixel coordinates, theta = atan2(y, x); zero outside the pupil stop.  A mode of
unit coefficient has unit RMS over the full unit disk (radians).

The "true modal coefficients" of a phase are its least-squares projection on
the sampled basis over the pupil pixels.
"""
import math

import numpy as np

from .geometry import pupil_mask


def noll_to_nm(j: int):
    """Noll index j >= 1 -> (n, m); m > 0 cosine, m < 0 sine."""
    n = 0
    while (n + 1) * (n + 2) // 2 < j:
        n += 1
    k = j - n * (n + 1) // 2 - 1          # position within radial order n
    if n % 2 == 0:
        mabs = 2 * ((k + 1) // 2)
    else:
        mabs = 2 * (k // 2) + 1
    m = mabs if (mabs == 0 or j % 2 == 0) else -mabs
    return n, m


def radial(n: int, m: int, rho):
    m = abs(m)
    out = np.zeros_like(np.asarray(rho, dtype=np.float64))
    for s in range((n - m) // 2 + 1):
        c = ((-1) ** s * math.factorial(n - s)
             / (math.factorial(s) * math.factorial((n + m) // 2 - s)
                * math.factorial((n - m) // 2 - s)))
        out = out + c * rho ** (n - 2 * s)
    return out


def radial_mp(n: int, m: int, rho, dps: int = 60) -> float:
    """R_n^|m|(rho) from the same factorial sum with exact integer
    coefficients, evaluated with dps significant digits (mpmath).  In float64
    the alternating sum loses every digit to cancellation beyond radial order
    ~40; at 60 digits it stays exact to float64 precision up to order ~100,
    which the high-order pins of a 4000-mode basis need."""
    import mpmath
    m = abs(m)
    with mpmath.workdps(dps):
        x = mpmath.mpf(rho)
        acc = mpmath.mpf(0)
        for s in range((n - m) // 2 + 1):
            c = ((-1) ** s * math.factorial(n - s)
                 // (math.factorial(s) * math.factorial((n + m) // 2 - s)
                     * math.factorial((n - m) // 2 - s)))
            acc += c * x ** (n - 2 * s)
        return float(acc)


def zernike_mp(j: int, rho: float, theta: float) -> float:
    """One Zernike value through radial_mp (high radial orders)."""
    n, m = noll_to_nm(j)
    r = radial_mp(n, m, rho)
    if m == 0:
        return math.sqrt(n + 1) * r
    ang = math.cos(abs(m) * theta) if m > 0 else math.sin(abs(m) * theta)
    return math.sqrt(2 * (n + 1)) * r * ang


def zernike(j: int, rho, theta):
    n, m = noll_to_nm(j)
    r = radial(n, m, rho)
    if m == 0:
        return math.sqrt(n + 1) * r
    ang = np.cos(abs(m) * theta) if m > 0 else np.sin(abs(m) * theta)
    return math.sqrt(2 * (n + 1)) * r * ang


def pupil_polar(n_pix: int):
    c = np.arange(n_pix, dtype=np.float64) - (n_pix - 1) / 2.0
    x = c[None, :] * np.ones((n_pix, 1))
    y = c[:, None] * np.ones((1, n_pix))
    rho = np.sqrt(x * x + y * y) / (n_pix / 2.0)
    theta = np.arctan2(y, x)
    return rho, theta


def modal_basis(n_pix: int, obsc: float, n_modes: int) -> np.ndarray:
    """(n_modes, n_pix, n_pix) float64: Z_2 .. Z_{n_modes+1} times the stop."""
    mask = pupil_mask(n_pix, obsc).astype(np.float64)
    rho, theta = pupil_polar(n_pix)
    return np.stack([zernike(j, rho, theta) * mask for j in range(2, n_modes + 2)])


def project(basis: np.ndarray, phase: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """Least-squares modal coefficients of `phase` (..., n, n) over the pupil."""
    sel = mask.astype(bool).ravel()
    Z = basis.reshape(basis.shape[0], -1)[:, sel].T          # (n_pix_in, n_modes)
    ph = np.asarray(phase, dtype=np.float64).reshape(-1, mask.size)[:, sel]
    c, *_ = np.linalg.lstsq(Z, ph.T, rcond=None)
    return c.T if np.ndim(phase) > 2 else c[:, 0]
