"""Multi-sensor system (FP64): every sensor's chain, slopes concatenated.

Test infrastructure only (see oracle/__init__.py).

A multi-sensor simulation (Sect. 6, Tab. 2; App. A, Tab. 4) runs, for each
wavefront sensor, AtmoPropagation along its own guide star, its sensor (SH or
ModulatedPyramid), its slope computer (ShSlopec or PyrSlopec), and feeds the
slope vectors of all sensors to one Modalrec.  This module only composes the
single-sensor oracle functions in that order: per sensor the phase, the image
(SH spots or the binned pyramid detector) and the slopes minus those of a flat
wavefront; the system's slope vector is the sensors' vectors concatenated in
sensor order, each all x then all y.
"""
import numpy as np

from . import atmo, geometry, pyramid, slopes, sh


def _valid(sensor):
    amp = geometry.pupil_mask(sensor.pupil.n_pix, sensor.pupil.obsc_frac)
    n_sub = sensor.pwfs.n_sub if sensor.kind == "pwfs" else sensor.sh.n_sub
    return amp.astype(np.float64), geometry.valid_subaps(amp.astype(np.uint8), n_sub)


def sensor_image(sensor, amp, phase, valid):
    """SH spots (n_valid, n, n) or the pyramid detector (2 n_sub, 2 n_sub)."""
    if sensor.kind == "sh":
        g = sensor.sh
        return sh.sh_spots(amp, phase, g.n_sub, g.sub_pix, g.fft_n, valid)
    g = sensor.pwfs
    return pyramid.pwfs_image(amp, phase, g.pad, g.n_mod, g.mod_amp, g.n_sub, g.pup_dist_px)


def sensor_slopes(sensor, image, valid, ref=None):
    if sensor.kind == "sh":
        return slopes.sh_slopes(image, ref)
    return slopes.pyr_slopes(image, sensor.pwfs.n_sub, valid, ref=ref)


def sensor_chain(screens, layers, sensor, t):
    """dict(phase, image, slopes, ref, valid) of one sensor at time t; slopes
    are reference-subtracted (flat-wavefront slopes in `ref`)."""
    amp, valid = _valid(sensor)
    n = sensor.pupil.n_pix
    phase = atmo.atmo_extract(screens, layers, sensor.source, n, sensor.pupil.pitch_m, t)
    image = sensor_image(sensor, amp, phase, valid)
    flat = sensor_image(sensor, amp, np.zeros((n, n)), valid)
    ref = sensor_slopes(sensor, flat, valid)
    return {"phase": phase, "image": image, "ref": ref, "valid": valid,
            "slopes": sensor_slopes(sensor, image, valid, ref=ref)}


def system_slopes(screens, layers, sensors, t):
    """(concatenated reference-subtracted slopes, per-sensor chains)."""
    chains = [sensor_chain(screens, layers, s, t) for s in sensors]
    return np.concatenate([c["slopes"] for c in chains]), chains


def slope_offsets(sensors):
    """Offset of each sensor's block in the concatenated vector, and the total."""
    offs, o = [], 0
    for s in sensors:
        _, valid = _valid(s)
        offs.append(o)
        o += 2 * len(valid)
    return offs, o
