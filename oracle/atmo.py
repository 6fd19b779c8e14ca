"""Frozen-flow layer extraction along a source direction (FP64).

Follows AtmoEvolution + AtmoPropagation (App. A, Tab. 4; parameters in App. B,
Listing 2: ``heights``, wind speed/direction, ``pixel_pupil``,
``pixel_pitch``, source ``polar_coordinates``, ``wavelengthInNm``).  The
propagation is geometric: the pupil phase is the sum over layers of each
layer's screen sampled along the line of sight.  The paper gives no formula;
the reading here:

* pupil pixel (j, i) sits at x_i = (i - (Np-1)/2) * pitch, y_j likewise;
* layer l (screen S_l of side M_l, pitch D_l, height h_l, wind v_l) is seen at
      X = x * (1 - h_l / H) + h_l * theta_x - v_lx * t
  (H = guide-star height, inf for a natural star: the cone compression), and
  at fractional screen index u = X / D_l + M_l / 2, likewise v for y;
* the screen is sampled bilinearly with periodic wrap;
* screens hold radians at 500 nm; the sum is scaled by 500 / lambda.

The integer part floor(u) is decided in float64 with the operation order
        u = ((x * s) + ((h * theta) - (v * t))) / D + M / 2,
    x = (i - (Np - 1) / 2) * pitch,  s = 1 - h / H,
which the CUDA path reproduces operation by operation.
"""
import math

import numpy as np


def layer_coords(n_pix: int, pitch: float, side: int, delta: float,
                 height: float, theta: float, wind: float, H: float, t: float):
    """Per-pixel (floor, frac) of the fractional screen index along one axis."""
    s = 1.0 - height / H
    i = np.arange(n_pix, dtype=np.float64)
    x = (i - (n_pix - 1) / 2.0) * pitch
    off = height * theta - wind * t
    u = (x * s + off) / delta + side / 2.0
    u0 = np.floor(u)
    return u0.astype(np.int64), u - u0


def atmo_extract(screens, layers, source, n_pix: int, pitch: float,
                 t: float) -> np.ndarray:
    """Pupil phase [rad at the source wavelength], (n_pix, n_pix) float64.

    ``screens``: sequence of (M_l, M_l) arrays (row = y); ``layers``: objects
    with side, pitch_m, height_m, vx_mps, vy_mps; ``source``: theta_x_rad,
    theta_y_rad, height_m, wavelength_nm.
    """
    phi = np.zeros((n_pix, n_pix))
    for S, L in zip(screens, layers):
        S = np.asarray(S, dtype=np.float64)
        M = L.side
        ix, fx = layer_coords(n_pix, pitch, M, L.pitch_m, L.height_m,
                              source.theta_x_rad, L.vx_mps, source.height_m, t)
        iy, fy = layer_coords(n_pix, pitch, M, L.pitch_m, L.height_m,
                              source.theta_y_rad, L.vy_mps, source.height_m, t)
        x0 = ix % M
        x1 = (ix + 1) % M
        y0 = iy % M
        y1 = (iy + 1) % M
        s00 = S[np.ix_(y0, x0)]
        s01 = S[np.ix_(y0, x1)]
        s10 = S[np.ix_(y1, x0)]
        s11 = S[np.ix_(y1, x1)]
        gx = fx[None, :]
        gy = fy[:, None]
        phi += ((1 - gx) * (1 - gy) * s00 + gx * (1 - gy) * s01
                + (1 - gx) * gy * s10 + gx * gy * s11)
    return phi * (500.0 / source.wavelength_nm)
