"""Shared helpers of the GPU parity tests (imported by tests/test_gpu_*.py)."""
import math

import numpy as np
import pytest

import synth
from oracle import atmo, geometry, screens


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def load_pkg():
    from paper_2602_06688_gb300 import build
    build.build()
    import paper_2602_06688_gb300 as sp
    sp.lib()
    return sp


def close_checked(sp, ctx):
    """Close a test module's context after checking that no kernel wrote into
    the guard band past any library workspace."""
    n_checked, n_bad = sp.specula_check_guards(ctx)
    ctx.close()
    assert n_bad == 0, f"{n_bad} of {n_checked} workspace guard bands overwritten"


def norm_intensity_error(got, ref):
    """max |I/sum I - I_ref/sum I_ref| / max(I_ref/sum I_ref): the normalised-
    intensity relative error (per-pixel relative error is meaningless at dark
    pixels, so the error is relative to the brightest pixel)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    a = got / got.sum()
    b = ref / ref.sum()
    return float(np.max(np.abs(a - b)) / np.max(b))


def kolmogorov_phase(n_pix, pitch, r0, seed, wavelength_nm=750.0, side=None):
    """A realistic pupil phase [rad at the WFS wavelength] built by the oracle:
    an FFT screen (seeded noise from synth) sampled on the pupil grid."""
    side = side or max(64, 1 << int(math.ceil(math.log2(2 * n_pix))))
    scr = screens.fft_screen(side, pitch, r0, 40.0, synth.screen_noise(seed, side),
                             synth.subharmonic_noise(seed))
    lay = type("L", (), dict(side=side, pitch_m=pitch, height_m=0.0, vx_mps=0.0,
                             vy_mps=0.0))()
    src = type("S", (), dict(theta_x_rad=0.0, theta_y_rad=0.0, height_m=math.inf,
                             wavelength_nm=wavelength_nm))()
    return atmo.atmo_extract([scr], [lay], src, n_pix, pitch, 0.0)


def pupil_amp(n_pix, obsc):
    return geometry.pupil_mask(n_pix, obsc).astype(np.float64)
