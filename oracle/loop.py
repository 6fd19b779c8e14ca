"""Closed adaptive-optics loop (FP64), test infrastructure only.

Follows the closed-loop objects of the paper's SOUL example (App. B,
Listing 2): the atmosphere propagated to the sensor, a deformable mirror
whose shape is subtracted from it (DM with a modal influence-function basis),
the pyramid sensor, slope computer and modal reconstructor (Modalrec), and an
integrator (IirFilter with integrator gains) whose output reaches the mirror
one step later through a delayed connection (the ``:-1`` input of Sect. 2.2).
Readings (the paper prints no loop equations):

  residual_k = phi_atm(t_k) - B^T c_{k-1}          (c_{-1} = 0)
  m_k        = R (slopes(residual_k) - reference)
  c_k        = (1 - leak) c_{k-1} + gain m_k

B [n_modes][n_pix^2] is the modal basis (zero outside the pupil), c the
commands in modal coefficients (radians at the sensor wavelength).  Per step
the loop reports the residual's RMS over the pupil pixels with its piston
removed, and the Strehl ratio at the science wavelength from the pupil-plane
field: SR = |sum_p A_p exp(i r_p lambda_wfs / lambda_sci)|^2 / (sum_p A_p)^2
(the on-axis value of the PSF relative to the diffraction-limited one).

``sensor`` is any callable residual -> modal measurement, so the loop logic
can be pinned with an ideal linear sensor independently of the pyramid.
"""
import numpy as np

from . import atmo, pyramid, recon, slopes


def residual_stats(amp: np.ndarray, resid: np.ndarray, wfs_over_sci: float):
    """(piston-removed RMS over the pupil, Strehl ratio at the science
    wavelength) of a residual phase in radians at the sensor wavelength."""
    w = amp.astype(np.float64).ravel()
    r = resid.astype(np.float64).ravel()
    sw = w.sum()
    mean = (w * r).sum() / sw
    rms = np.sqrt((w * (r - mean) ** 2).sum() / sw)
    e = (w * np.exp(1j * r * wfs_over_sci)).sum()
    return rms, float(np.abs(e) ** 2 / sw ** 2)


def dm_shape(basis: np.ndarray, cmd: np.ndarray) -> np.ndarray:
    """B^T c: the mirror's phase over the pupil grid."""
    nm = basis.shape[0]
    return (cmd[:, None] * basis.reshape(nm, -1)).sum(axis=0).reshape(basis.shape[1:])


def run_loop(atm_phases, amp, basis, sensor, gain, leak, wfs_over_sci):
    """Iterate the loop over the given atmospheric phases (one per step).
    Returns per-step (rms, strehl), the commands after every step and the
    last residual."""
    nm = basis.shape[0]
    c = np.zeros(nm)
    stats, cmds = [], []
    resid = None
    for phi in atm_phases:
        resid = phi - dm_shape(basis, c)
        stats.append(residual_stats(amp, resid, wfs_over_sci))
        m = sensor(resid)
        c = (1.0 - leak) * c + gain * m
        cmds.append(c.copy())
    return np.array(stats), np.array(cmds), resid


def pyramid_sensor(amp, pad, n_mod, mod_amp, n_sub, pup_dist, valid, R):
    """residual -> R (pyramid slopes - flat-wavefront reference)."""
    flat = pyramid.pwfs_image(amp, np.zeros_like(amp), pad, n_mod, mod_amp, n_sub, pup_dist)
    ref = slopes.pyr_slopes(flat, n_sub, valid)

    def sense(resid):
        det = pyramid.pwfs_image(amp, resid, pad, n_mod, mod_amp, n_sub, pup_dist)
        return recon.mvm(R, slopes.pyr_slopes(det, n_sub, valid, ref=ref))
    return sense


def atmosphere(screens, layers, source, n_pix, pitch, times):
    """The atmospheric phase at the sensor for each step time."""
    return [atmo.atmo_extract(screens, layers, source, n_pix, pitch, t) for t in times]
