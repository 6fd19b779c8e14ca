"""Oracle pins: the multi-sensor composition (zero slopes for flat screens,
identical SH slopes under a linear ramp, laser-star cone scaling, block
layout)."""
import math
from types import SimpleNamespace as NS

import numpy as np

from oracle import geometry, system

M, PITCH = 128, 0.25


def _layer(h=0.0, vx=0.0, vy=0.0):
    return NS(side=M, pitch_m=PITCH, height_m=h, vx_mps=vx, vy_mps=vy)


def _sh(H=math.inf, tx=0.0, ty=0.0, obsc=0.0):
    return NS(kind="sh", pupil=NS(n_pix=32, pitch_m=PITCH, obsc_frac=obsc),
              source=NS(theta_x_rad=tx, theta_y_rad=ty, height_m=H, wavelength_nm=589.0),
              sh=NS(n_sub=4, sub_pix=8, fft_n=16), pwfs=None)


def _pyr(tx=0.0, ty=0.0):
    return NS(kind="pwfs", pupil=NS(n_pix=16, pitch_m=2 * PITCH, obsc_frac=0.0),
              source=NS(theta_x_rad=tx, theta_y_rad=ty, height_m=math.inf, wavelength_nm=750.0),
              pwfs=NS(pad=2, n_mod=4, mod_amp=2.0, n_sub=4, pup_dist_px=16), sh=None)


def _ramp(al, be):
    jj, ii = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    return al * ii + be * jj


def test_flat_screens_give_zero_slopes():
    sensors = [_sh(90e3, 1e-5, 0.0, 0.2), _pyr(0.0, 2e-5), _sh()]
    scr = [np.zeros((M, M)), np.zeros((M, M))]
    s, chains = system.system_slopes(scr, [_layer(), _layer(5000.0, 3.0, -2.0)], sensors, 0.05)
    assert s.shape == (system.slope_offsets(sensors)[1],)
    assert np.all(s == 0.0)


def test_ramp_gives_equal_sh_slopes_in_full_subapertures():
    sen = _sh()
    amp = geometry.pupil_mask(32, 0.0)
    valid = geometry.valid_subaps(amp, 4)
    full = [k for k, idx in enumerate(valid)
            if amp[8 * (idx // 4):8 * (idx // 4) + 8, 8 * (idx % 4):8 * (idx % 4) + 8].all()]
    assert len(full) >= 4
    s, _ = system.system_slopes([_ramp(0.02, -0.01)], [_layer()], [sen], 0.0)
    nv = len(valid)
    sx, sy = s[:nv][full], s[nv:][full]
    assert np.ptp(sx) < 1e-10 and np.ptp(sy) < 1e-10
    # a phase increasing along +x moves the spot to +x
    assert sx[0] > 0 and sy[0] < 0


def test_laser_star_cone_equals_scaled_ramp_on_the_ground():
    """A layer at height h seen from a laser star at H: the pupil phase is the
    ramp scaled by 1 - h/H plus a constant, so its SH slopes equal those of
    the scaled ramp on a ground layer seen by a natural star."""
    h, H, al, be = 6000.0, 90e3, 0.03, 0.012
    sc = 1.0 - h / H
    s_lgs, _ = system.system_slopes([_ramp(al, be)], [_layer(h, 4.0, -1.0)],
                                    [_sh(H, 1e-5, -2e-5)], 0.01)
    s_ngs, _ = system.system_slopes([_ramp(al * sc, be * sc)], [_layer()], [_sh()], 0.0)
    assert np.max(np.abs(s_lgs - s_ngs)) < 1e-9


def test_blocks_are_the_single_sensor_chains():
    rng = np.random.default_rng(9)
    scr = [rng.standard_normal((M, M)) * 0.3, rng.standard_normal((M, M)) * 0.2]
    layers = [_layer(0.0, 2.0, 1.0), _layer(3000.0, -5.0, 4.0)]
    sensors = [_pyr(1e-5, 0.0), _sh(90e3, 0.0, 1.5e-5), _pyr(-2e-5, 1e-5)]
    s, chains = system.system_slopes(scr, layers, sensors, 0.02)
    offs, tot = system.slope_offsets(sensors)
    assert tot == s.size
    for k, sen in enumerate(sensors):
        one = system.sensor_chain(scr, layers, sen, 0.02)
        blk = s[offs[k]:offs[k] + one["slopes"].size]
        assert np.array_equal(blk, one["slopes"])
        assert np.array_equal(chains[k]["phase"], one["phase"])
    # different guide-star directions see different phases
    assert not np.allclose(chains[0]["phase"], chains[2]["phase"])
