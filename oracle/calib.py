"""Calibration (FP64): push-pull interaction matrix and truncated pseudo-inverse.

Follows ImCalibrator, RecCalibrator and PushPullGenerator (App. A, Tab. 4) and
the Intmat / Recmat data objects (Tab. 3).  Readings (the paper gives no
formula):

* interaction matrix, one column per mode j of the modal basis:
      IM[:, j] = (s(+a Z_j) - s(-a Z_j)) / (2 a)
  with s the reference-free pyramid slopes of a flat wavefront plus the
  pushed mode (a in radians at the WFS wavelength; 0.1 rad by default);
* reconstructor R = pinv(IM) with singular values below rcond * sigma_max
  discarded:  IM = U S V^T,  R = V S_k^-1 U_k^T.
"""
import numpy as np

from . import pyramid, slopes


def push_pull_im(amp, basis, a, pad, n_mod, mod_amp, n_sub, pup_dist, valid):
    """(n_slopes, n_modes) float64 interaction matrix."""
    n_modes = basis.shape[0]
    cols = []
    for j in range(n_modes):
        sp = slopes.pyr_slopes(
            pyramid.pwfs_image(amp, a * basis[j], pad, n_mod, mod_amp, n_sub, pup_dist),
            n_sub, valid)
        sm = slopes.pyr_slopes(
            pyramid.pwfs_image(amp, -a * basis[j], pad, n_mod, mod_amp, n_sub, pup_dist),
            n_sub, valid)
        cols.append((sp - sm) / (2.0 * a))
    return np.stack(cols, axis=1)


def pinv_truncated(A: np.ndarray, rcond: float):
    """Truncated Moore-Penrose inverse by SVD; returns (R, rank)."""
    U, s, Vt = np.linalg.svd(np.asarray(A, dtype=np.float64), full_matrices=False)
    keep = s > rcond * s[0]
    R = (Vt[keep].T / s[keep]) @ U[:, keep].T
    return R, int(keep.sum())


def singular_values(A: np.ndarray) -> np.ndarray:
    return np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False)
