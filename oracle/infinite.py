"""Infinite phase screens (FP64): the InfinitePhaseScreen data object (Tab. 3)
and the AtmoInfiniteEvolution processing object (Tab. 4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper names these objects but does not give their construction.  This
module follows the published method of Assemat, Wilson and Gendron (Optics
Express 14, 988, 2006).  A screen grows one line (a row or a column of
`side` pixels) at a time.  Each new line Z is drawn from its Gaussian
distribution conditioned on a stencil X: the n_st lines next to it, nearest
first, full width.

    Z = A X + B b,   A = C_ZX C_XX^+,   B B^T = C_ZZ - A C_XZ,   b ~ N(0, I)

* Covariances come from the phase covariance of the von Karman spectrum that
  the FFT screens use (``screens.vk_psd``: 0.023 r0^-5/3 (f^2 + L0^-2)^-11/6,
  rad^2 at 500 nm).  Its Hankel transform is, in closed form,
      C(r) = 0.023 (2 pi / (2^(5/6) Gamma(11/6))) (L0/r0)^(5/3) x^(5/6) K_5/6(x),
      x = 2 pi r / L0,
  with C(0) = the limit x^(5/6) K_5/6(x) -> 2^(-1/6) Gamma(5/6).  A finite L0
  is required.
* C_XX^+ keeps the eigenvalues above rcond times the largest one.
  B is the symmetric (principal) square root of C_ZZ - A C_XZ, with negative
  round-off eigenvalues set to zero.  It is the one square root that both
  sides can compute independently.
* Geometry: pixel p of a line sits at p pitch along the line.  Stencil line d
  (d = 1 .. n_st) lies d pitch behind the new line.  Index k = (d - 1) side + p
  orders X.
* Ring storage: the screen is `side` x `side` with line L stored at slot
  L mod side.  Rows (axis 0) are screen[slot, :]; columns (axis 1) are
  screen[:, slot].  Growing in direction dir = +1 writes line `head` from
  lines head - 1, head - 2, ...; dir = -1 writes line `head` from lines
  head + 1, head + 2, ....  The covariance is isotropic, so the same (A, B)
  serves both axes and both directions.
* Noise: element p of line L of stream s is normal (p mod 4) of the Philox
  counter (p // 4, L low 32 bits, L high 32 bits, s) (``philox.normals4``),
  scaled by b_scale.  With b_scale = (r0_ref / r0)^(5/6), one (A, B) built for
  r0_ref serves every r0, because A does not depend on r0 and B scales as
  r0^(-5/6).
"""
import math

import numpy as np
from scipy import special

from . import philox

NU = 5.0 / 6.0
PSD_CONST = 0.023          # the FFT screens' spectrum constant (screens.vk_psd)


def vk_covariance(r, r0: float, L0: float):
    """C(r) in rad^2 at 500 nm for distances r [m] (array)."""
    if not math.isfinite(L0):
        raise ValueError("the phase covariance needs a finite outer scale")
    r = np.asarray(r, dtype=np.float64)
    scale = PSD_CONST * 2.0 * math.pi / (2.0 ** NU * math.gamma(11.0 / 6.0)) \
        * (L0 / r0) ** (5.0 / 3.0)
    x = 2.0 * math.pi * r / L0
    out = np.empty_like(x)
    z = x == 0
    out[z] = 2.0 ** (NU - 1.0) * math.gamma(NU)
    out[~z] = x[~z] ** NU * special.kv(NU, x[~z])
    return scale * out


def stencil_covariances(side: int, n_st: int, pitch: float, r0: float, L0: float):
    """(C_XX, C_ZX, C_ZZ) for a new line and its n_st stencil lines."""
    p = np.arange(side, dtype=np.float64)
    pos_z = np.stack([p, np.zeros(side)], axis=1)               # (along, across)
    pos_x = np.concatenate([np.stack([p, np.full(side, float(d))], axis=1)
                            for d in range(1, n_st + 1)])

    def cov(a, b):
        d = a[:, None, :] - b[None, :, :]
        return vk_covariance(pitch * np.sqrt((d ** 2).sum(axis=2)), r0, L0)

    return cov(pos_x, pos_x), cov(pos_z, pos_x), cov(pos_z, pos_z)


def line_operators(side: int, n_st: int, pitch: float, r0: float, L0: float,
                   rcond: float = 1e-12):
    """(A [side, n_st side], B [side, side]) of the conditional draw."""
    Cxx, Czx, Czz = stencil_covariances(side, n_st, pitch, r0, L0)
    lam, V = np.linalg.eigh(Cxx)
    keep = lam > rcond * lam.max()
    inv = np.where(keep, 1.0 / np.where(keep, lam, 1.0), 0.0)
    A = Czx @ (V * inv) @ V.T
    BBt = Czz - A @ Czx.T
    BBt = 0.5 * (BBt + BBt.T)
    mu, W = np.linalg.eigh(BBt)
    B = (W * np.sqrt(np.maximum(mu, 0.0))) @ W.T
    return A, B


def line_noise(seed: int, stream: int, line: int, side: int) -> np.ndarray:
    """The side standard normals of line `line` (signed) of noise stream `stream`."""
    u = line & 0xFFFFFFFFFFFFFFFF
    nq = (side + 3) // 4
    g = philox.normals4(np.arange(nq, dtype=np.uint32), np.full(nq, u & 0xFFFFFFFF, np.uint32),
                        np.full(nq, u >> 32, np.uint32), np.full(nq, stream, np.uint32), seed)
    return np.stack(g, axis=1).reshape(-1)[:side].astype(np.float64)


def get_line(screen: np.ndarray, axis: int, line: int) -> np.ndarray:
    s = line % screen.shape[0]
    return screen[s, :].copy() if axis == 0 else screen[:, s].copy()


def set_line(screen: np.ndarray, axis: int, line: int, values: np.ndarray) -> None:
    s = line % screen.shape[0]
    if axis == 0:
        screen[s, :] = values
    else:
        screen[:, s] = values


def add_line(screen: np.ndarray, A, B, axis: int, direction: int, head: int,
             noise: np.ndarray, b_scale: float = 1.0) -> None:
    """Write line `head` on `axis`, conditioned on the n_st lines behind it."""
    side = screen.shape[0]
    n_st = A.shape[1] // side
    X = np.concatenate([get_line(screen, axis, head - direction * d)
                        for d in range(1, n_st + 1)])
    set_line(screen, axis, head, A @ X + b_scale * (B @ noise))


def extend(screen: np.ndarray, A, B, axis: int, direction: int, head: int, n_new: int,
           seed: int, stream: int, b_scale: float = 1.0) -> int:
    """Append n_new lines starting at line `head`, moving in `direction`, with
    the Philox line noise; returns the next head."""
    side = screen.shape[0]
    for k in range(n_new):
        L = head + direction * k
        add_line(screen, A, B, axis, direction, L, line_noise(seed, stream, L, side), b_scale)
    return head + direction * n_new


def structure_function(screen_lines: np.ndarray, lag: int) -> float:
    """Mean (phi(y + lag) - phi(y))^2 along axis 0 of a (n_lines, side) strip."""
    d = screen_lines[lag:] - screen_lines[:-lag]
    return float(np.mean(d * d))
