"""The synthetic workloads: sizes, seeds and atmospheric profiles.

Five systems, shaped like the paper's (Sect. 6, Tab. 2; App. B, Listing 2):

* ``pwfs8m_tiny``   one pyramid WFS, D = 8 m, 64 px pupil, 128^2 FFT, 12 mod points
* ``pwfs8m``        one pyramid WFS, D = 8.4 m, 160 px, 320^2 FFT, 24 mod points
* ``learned8m``     learned-reconstructor training set on the ``pwfs8m`` geometry
* ``mwfs39m``       6 LGS Shack-Hartmann (68x68 subaps of 12 px, 24^2 FFT) and
                    3 NGS pyramids (120 px, 240^2 FFT, 16 mod points), D = 39 m
* ``pwfs39m``       one ELT-scale pyramid WFS, 480 px, 960^2 FFT, 48 mod points
* ``mwfs8m_small``  a small multi-sensor system (2 SH + 2 pyramids) for tests

Values the paper does not state are readings chosen here (obscuration of the
39 m pupil, WFS wavelength 750 nm as in Listing 2, outer scale 40 m as in
Listing 2, screen sides, layer profiles, guide-star asterisms, 1 ms step).
This file only states parameters; it performs no simulation arithmetic.
"""
from dataclasses import dataclass, field
import math
from typing import List, Optional, Tuple

import numpy as np

ARCSEC = math.pi / (180.0 * 3600.0)


@dataclass(frozen=True)
class Layer:
    side: int          # screen side M [px]
    pitch_m: float     # screen sampling Delta [m]
    height_m: float    # layer altitude [m]
    vx_mps: float      # wind velocity x [m/s]
    vy_mps: float      # wind velocity y [m/s]
    r0_m: float        # Fried parameter of this layer at 500 nm [m]
    L0_m: float        # outer scale [m]; math.inf = Kolmogorov
    seed: int          # seed of the screen noise


@dataclass(frozen=True)
class Source:
    theta_x_rad: float
    theta_y_rad: float
    height_m: float    # math.inf for a natural guide star
    wavelength_nm: float


@dataclass(frozen=True)
class Pupil:
    n_pix: int         # pupil diameter [px]
    pitch_m: float     # pupil sampling [m/px]
    obsc_frac: float   # central obscuration (fraction of the diameter)


@dataclass(frozen=True)
class PwfsGeom:
    pad: int           # FFT side N = pad * n_pix
    n_mod: int         # modulation points
    mod_amp: float     # modulation radius [lambda/D]
    n_sub: int         # subapertures across one pupil image
    pup_dist_px: int   # separation of the pupil images [px] (= n_pix here)


@dataclass(frozen=True)
class ShGeom:
    n_sub: int         # subapertures across the pupil
    sub_pix: int       # pupil pixels across one subaperture
    fft_n: int         # padded per-subaperture FFT side


@dataclass(frozen=True)
class Sensor:
    kind: str          # 'pwfs' or 'sh'
    pupil: Pupil
    source: Source
    pwfs: Optional[PwfsGeom] = None
    sh: Optional[ShGeom] = None


@dataclass(frozen=True)
class Workload:
    name: str
    diameter_m: float
    sensors: Tuple[Sensor, ...]
    layers: Tuple[Layer, ...]
    n_modes: int
    n_frames: int
    dt_s: float
    r0_m: float
    mlp_hidden: Tuple[int, ...] = ()


def _profile(cfg_id, n_layers, r0, heights, weights, speeds, side, pitch, L0,
             dir_seed):
    """Per-layer parameters; wind directions drawn uniformly from dir_seed."""
    w = np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    if dir_seed is None:
        dirs = np.zeros(n_layers)
    else:
        dirs = np.random.default_rng(dir_seed).uniform(0.0, 2 * math.pi,
                                                        n_layers)
    layers = []
    for l in range(n_layers):
        r0_l = r0 * float(w[l]) ** (-3.0 / 5.0)
        layers.append(Layer(side=side, pitch_m=pitch, height_m=float(heights[l]),
                            vx_mps=float(speeds[l] * math.cos(dirs[l])),
                            vy_mps=float(speeds[l] * math.sin(dirs[l])),
                            r0_m=r0_l, L0_m=L0, seed=1000 * cfg_id + l))
    return tuple(layers)


def _pwfs8m_tiny():
    D, n = 8.0, 64
    pup = Pupil(n, D / n, 0.0)
    src = Source(0.0, 0.0, math.inf, 750.0)
    geom = PwfsGeom(pad=2, n_mod=12, mod_amp=3.0, n_sub=16, pup_dist_px=n)
    layers = _profile(1, 1, 0.15, [0.0], [1.0], [10.0], 256, D / n, math.inf,
                      None)
    return Workload('pwfs8m_tiny', D, (Sensor('pwfs', pup, src, pwfs=geom),),
                    layers, n_modes=200, n_frames=100, dt_s=1e-3, r0_m=0.15)


def _pwfs8m():
    D, n = 8.4, 160
    pup = Pupil(n, D / n, 0.11)
    src = Source(0.0, 0.0, math.inf, 750.0)
    geom = PwfsGeom(pad=2, n_mod=24, mod_amp=3.0, n_sub=40, pup_dist_px=n)
    layers = _profile(2, 3, 0.12, [0.0, 5000.0, 10000.0], [0.6, 0.3, 0.1],
                      [5.0, 12.5, 20.0], 1024, D / n, 40.0, 2)
    return Workload('pwfs8m', D, (Sensor('pwfs', pup, src, pwfs=geom),),
                    layers, n_modes=500, n_frames=1000, dt_s=1e-3, r0_m=0.12)


def _soul8m():
    """The geometry of the paper's SOUL example (App. B, Listing 2): 40
    subapertures across each pupil image, images 48 detector pixels apart on
    a 120 px detector, modulation 3 lambda/D.  Sampled with an 80 px pupil
    padded three times (240^2 FFT) and 2 x 2 binning; LBT 8.2 m, 750 nm;
    16 modulation points, two layers (readings: the listing's sampling and
    atmosphere are not all given)."""
    D, n = 8.2, 80
    pup = Pupil(n, D / n, 0.11)
    src = Source(0.0, 0.0, math.inf, 750.0)
    geom = PwfsGeom(pad=3, n_mod=16, mod_amp=3.0, n_sub=40, pup_dist_px=96)
    layers = _profile(6, 2, 0.14, [0.0, 6000.0], [0.7, 0.3], [6.0, 15.0], 512, D / n, 40.0, 6)
    return Workload('soul8m', D, (Sensor('pwfs', pup, src, pwfs=geom),),
                    layers, n_modes=300, n_frames=1000, dt_s=1e-3, r0_m=0.14)


def _soul220():
    """The paper's SOUL example as stated (App. B, Listing 2; Sect. 6,
    Tab. 2): 220 px pupil (0.037 m pixels on LBT's 8.2 m), 3x oversampling
    (660^2 FFT), 24 modulation points of 3 lambda/D, pup_diam 40 and
    pup_dist 48 subapertures (264 grid pixels) on an output_resolution 120
    detector, so a detector pixel is 5.5 x 5.5 grid pixels; 750 nm; 500
    modes.  Two layers as in soul8m (the listing's atmosphere is not all
    given)."""
    D, n = 8.2, 220
    pup = Pupil(n, D / n, 0.11)
    src = Source(0.0, 0.0, math.inf, 750.0)
    geom = PwfsGeom(pad=3, n_mod=24, mod_amp=3.0, n_sub=40, pup_dist_px=264)
    layers = _profile(6, 2, 0.14, [0.0, 6000.0], [0.7, 0.3], [6.0, 15.0], 512, D / n, 40.0, 6)
    return Workload('soul220', D, (Sensor('pwfs', pup, src, pwfs=geom),),
                    layers, n_modes=500, n_frames=1000, dt_s=1e-3, r0_m=0.14)


def _learned8m():
    base = _pwfs8m()
    return Workload('learned8m', base.diameter_m, base.sensors, base.layers[:1],
                    n_modes=500, n_frames=5000, dt_s=1e-3, r0_m=0.12,
                    mlp_hidden=(1024, 1024))


def _mwfs39m():
    D = 39.0
    sh_pix = 68 * 12
    sh_pup = Pupil(sh_pix, D / sh_pix, 0.28)
    py_pup = Pupil(120, D / 120, 0.28)
    sensors = []
    for k in range(6):
        a = math.radians(60.0 * k)
        src = Source(45 * ARCSEC * math.cos(a), 45 * ARCSEC * math.sin(a),
                     90e3, 589.0)
        sensors.append(Sensor('sh', sh_pup, src,
                              sh=ShGeom(n_sub=68, sub_pix=12, fft_n=24)))
    for k in range(3):
        a = math.radians(30.0 + 120.0 * k)
        src = Source(55 * ARCSEC * math.cos(a), 55 * ARCSEC * math.sin(a),
                     math.inf, 750.0)
        sensors.append(Sensor('pwfs', py_pup, src,
                              pwfs=PwfsGeom(pad=2, n_mod=16, mod_amp=3.0,
                                            n_sub=40, pup_dist_px=120)))
    h = np.linspace(0.0, 20e3, 10)
    layers = _profile(4, 10, 0.157, h, np.exp(-h / 3e3),
                      np.linspace(5.0, 30.0, 10), 2048, D / sh_pix, 40.0, 4)
    return Workload('mwfs39m', D, tuple(sensors), layers, n_modes=4000,
                    n_frames=1000, dt_s=1e-3, r0_m=0.157)


def _mwfs8m_small():
    """A small multi-sensor system for parity tests: two laser-star SH (96 px,
    8 x 8 subapertures of 12 px, 24^2 FFT) and two natural-star pyramids
    (64 px, 128^2 FFT, 8 modulation points), three layers."""
    D = 8.0
    sh_pup = Pupil(96, D / 96, 0.2)
    py_pup = Pupil(64, D / 64, 0.2)
    sensors = []
    for k in range(2):
        a = math.radians(90.0 * k + 20.0)
        sensors.append(Sensor('sh', sh_pup,
                              Source(20 * ARCSEC * math.cos(a), 20 * ARCSEC * math.sin(a),
                                     90e3, 589.0),
                              sh=ShGeom(n_sub=8, sub_pix=12, fft_n=24)))
    for k in range(2):
        a = math.radians(180.0 * k + 45.0)
        sensors.append(Sensor('pwfs', py_pup,
                              Source(30 * ARCSEC * math.cos(a), 30 * ARCSEC * math.sin(a),
                                     math.inf, 750.0),
                              pwfs=PwfsGeom(pad=2, n_mod=8, mod_amp=3.0, n_sub=16,
                                            pup_dist_px=64)))
    h = np.array([0.0, 4e3, 10e3])
    layers = _profile(6, 3, 0.15, h, [0.6, 0.3, 0.1], [5.0, 10.0, 20.0], 256, D / 96, 40.0, 6)
    return Workload('mwfs8m_small', D, tuple(sensors), layers, n_modes=64,
                    n_frames=100, dt_s=1e-3, r0_m=0.15)


def _pwfs39m():
    D, n = 39.0, 480
    pup = Pupil(n, D / n, 0.28)
    src = Source(0.0, 0.0, math.inf, 750.0)
    geom = PwfsGeom(pad=2, n_mod=48, mod_amp=4.0, n_sub=96, pup_dist_px=n)
    h = np.linspace(0.0, 25e3, 35)
    layers = _profile(5, 35, 0.157, h, np.exp(-h / 3e3),
                      np.linspace(5.0, 40.0, 35), 2048, D / n, 40.0, 5)
    return Workload('pwfs39m', D, (Sensor('pwfs', pup, src, pwfs=geom),),
                    layers, n_modes=4000, n_frames=2000, dt_s=1e-3, r0_m=0.157,
                    mlp_hidden=(2048, 2048))


def _andes400():
    """The ANDES pyramid of Sect. 6, Tab. 2 (24 x 1600 x 1600): a 400 px
    pupil on the 39 m ELT (0.0975 m pixels), 100 x 100 subapertures,
    oversampling 4 (1600^2 FFT), 24 modulation points.  The table gives
    neither the modulation radius nor the pupil separation: 3 lambda/D and
    120 subapertures (1.2 pupil diameters, as in the SOUL example's 48 / 40)
    are taken, so a detector pixel is 4 x 4 grid pixels on a 400^2
    detector.  The 35-layer ELT profile of pwfs39m at this pupil's pitch."""
    D, n = 39.0, 400
    pup = Pupil(n, D / n, 0.28)
    src = Source(0.0, 0.0, math.inf, 750.0)
    geom = PwfsGeom(pad=4, n_mod=24, mod_amp=3.0, n_sub=100, pup_dist_px=480)
    h = np.linspace(0.0, 25e3, 35)
    layers = _profile(5, 35, 0.157, h, np.exp(-h / 3e3),
                      np.linspace(5.0, 40.0, 35), 2048, D / n, 40.0, 5)
    return Workload('andes400', D, (Sensor('pwfs', pup, src, pwfs=geom),),
                    layers, n_modes=4000, n_frames=1000, dt_s=1e-3, r0_m=0.157)


WORKLOADS = {
    'pwfs8m_tiny': _pwfs8m_tiny,
    'pwfs8m': _pwfs8m,
    'learned8m': _learned8m,
    'mwfs39m': _mwfs39m,
    'mwfs8m_small': _mwfs8m_small,
    'pwfs39m': _pwfs39m,
    'soul8m': _soul8m,
    'soul220': _soul220,
    'andes400': _andes400,
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]()
