"""Slope computers (FP64): PyrSlopec and ShSlopec (App. A, Tab. 4), Slopes data
object (App. A, Tab. 3).

Output layout: all x slopes of the valid subapertures, then all y slopes.
"""
import numpy as np

from .geometry import pyr_quadrant_index


def pyr_slopes(det: np.ndarray, n_sub: int, valid: np.ndarray,
               ref=None) -> np.ndarray:
    """Pyramid slopes normalised by the mean subaperture flux.

    For valid subaperture k with quadrant values Q1 (+x,+y), Q2 (-x,+y),
    Q3 (-x,-y), Q4 (+x,-y) (see ``geometry.pyr_quadrant_index``):
        Sx = ((Q1 + Q4) - (Q2 + Q3)) / T,   Sy = ((Q1 + Q2) - (Q3 + Q4)) / T,
        T  = mean over valid k of (Q1 + Q2 + Q3 + Q4)
    (reading: global-mean normalisation).  ``ref`` (reference slopes of a flat
    wavefront) is subtracted when given.
    """
    q = pyr_quadrant_index(valid, n_sub)
    d = det.ravel()
    q1, q2, q3, q4 = (d[q[i]] for i in range(4))
    T = np.mean(q1 + q2 + q3 + q4)
    sx = ((q1 + q4) - (q2 + q3)) / T
    sy = ((q1 + q2) - (q3 + q4)) / T
    s = np.concatenate([sx, sy])
    if ref is not None:
        s = s - ref
    return s


def pyr_slopes_maps(det: np.ndarray, maps: np.ndarray, ref=None) -> np.ndarray:
    """The same slopes from explicit detector indices of the four pupil
    images (``geometry.pyr_image_index``): maps[0..3] = Q1..Q4."""
    d = det.ravel()
    q1, q2, q3, q4 = (d[maps[i]] for i in range(4))
    T = np.mean(q1 + q2 + q3 + q4)
    s = np.concatenate([((q1 + q4) - (q2 + q3)) / T, ((q1 + q2) - (q3 + q4)) / T])
    return s - ref if ref is not None else s


def sh_slopes(spots: np.ndarray, ref=None) -> np.ndarray:
    """Centre-of-gravity slopes in pixels over the whole n x n window:
    Sx = sum x I / sum I, Sy = sum y I / sum I with x = j - (n-1)/2 (no
    threshold).  ``spots``: (n_valid, n, n)."""
    n = spots.shape[-1]
    c = np.arange(n, dtype=np.float64) - (n - 1) / 2.0
    tot = spots.sum(axis=(1, 2))
    sx = (spots * c[None, None, :]).sum(axis=(1, 2)) / tot
    sy = (spots * c[None, :, None]).sum(axis=(1, 2)) / tot
    s = np.concatenate([sx, sy])
    if ref is not None:
        s = s - ref
    return s
