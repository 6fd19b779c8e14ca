"""Oracle pins: frozen-flow extraction (exact rolls, linear ramps, geometry)."""
import math
from types import SimpleNamespace as NS

import numpy as np

from oracle import atmo

NP, PITCH, M = 16, 0.5, 64


def _layer(h=0.0, vx=0.0, vy=0.0, side=M, pitch=PITCH):
    return NS(side=side, pitch_m=pitch, height_m=h, vx_mps=vx, vy_mps=vy)


def _src(tx=0.0, ty=0.0, H=math.inf, lam=500.0):
    return NS(theta_x_rad=tx, theta_y_rad=ty, height_m=H, wavelength_nm=lam)


def test_integer_shift_is_exact_window_and_roll():
    rng = np.random.default_rng(3)
    S = rng.standard_normal((M, M))
    # x_i / pitch = i - 7.5; u = i - 7.5 - vx t / pitch + 32 is integral when
    # vx t = -0.5 pitch (mod pitch)
    for k in range(3):
        t = 1.0
        vx = -(0.5 + k) * PITCH
        phi = atmo.atmo_extract([S], [_layer(vx=vx, vy=-0.5 * PITCH)], _src(),
                                NP, PITCH, t)
        x0 = 32 - 7 + k
        y0 = 32 - 7
        assert np.array_equal(phi, S[y0:y0 + NP, x0:x0 + NP])


def test_periodic_wrap():
    rng = np.random.default_rng(4)
    S = rng.standard_normal((M, M))
    t = 1.0
    vx = -(0.5 + 40) * PITCH      # window starts at column 65 -> wraps to 1
    phi = atmo.atmo_extract([S], [_layer(vx=vx, vy=-0.5 * PITCH)], _src(),
                            NP, PITCH, t)
    cols = (np.arange(NP) + 32 - 7 + 40) % M
    assert np.array_equal(phi, S[25:25 + NP][:, cols])


def test_bilinear_reproduces_linear_ramp_and_geometry():
    al, be, ga = 0.3, -0.7, 2.0
    jj, ii = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    S = al * ii + be * jj + ga
    h, H, tx, ty, vx, vy, t = 4000.0, 90e3, 2e-5, -1e-5, 7.0, -3.0, 0.013
    phi = atmo.atmo_extract([S], [_layer(h=h, vx=vx, vy=vy)],
                            _src(tx, ty, H, 750.0), NP, PITCH, t)
    x = (np.arange(NP) - (NP - 1) / 2) * PITCH
    s = 1 - h / H
    u = (x * s + h * tx - vx * t) / PITCH + M / 2
    v = (x * s + h * ty - vy * t) / PITCH + M / 2
    ref = (al * u[None, :] + be * v[:, None] + ga) * 500.0 / 750.0
    assert np.max(np.abs(phi - ref)) < 1e-12
    # LGS cone: the footprint gradient shrinks by (1 - h/H)
    gx = np.diff(phi, axis=1).mean()
    assert abs(gx - al * s * 500 / 750) < 1e-12


def test_layers_add():
    rng = np.random.default_rng(5)
    S1, S2 = rng.standard_normal((M, M)), rng.standard_normal((M, M))
    L1, L2 = _layer(vx=1.3), _layer(h=1000.0, vy=-2.1)
    src = _src(1e-5, 3e-6, math.inf, 600.0)
    a = atmo.atmo_extract([S1], [L1], src, NP, PITCH, 0.2)
    b = atmo.atmo_extract([S2], [L2], src, NP, PITCH, 0.2)
    ab = atmo.atmo_extract([S1, S2], [L1, L2], src, NP, PITCH, 0.2)
    assert np.allclose(ab, a + b, atol=1e-13)


def test_wind_moves_pattern_downstream():
    rng = np.random.default_rng(6)
    S = rng.standard_normal((M, M))
    L = _layer(vx=PITCH, vy=0.0)     # one screen pixel per second along +x
    phi0 = atmo.atmo_extract([S], [L], _src(), NP, PITCH, 0.25)
    phi1 = atmo.atmo_extract([S], [L], _src(), NP, PITCH, 1.25)
    # what pixel i saw at t0 is seen by pixel i+1 one second later
    assert np.allclose(phi1[:, 1:], phi0[:, :-1], atol=1e-13)
