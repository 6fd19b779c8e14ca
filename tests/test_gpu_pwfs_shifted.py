"""GPU parity: the pyramid's shifted-mask form against its FP64 oracle.

Same tolerance as the tilt form: normalised-intensity max relative error
<= 1e-5 on the binned detector (one forward and one inverse transform per
point in FP32; the tilt form does two forward and one inverse)."""
import numpy as np
import pytest

from gpu_common import close_checked, kolmogorov_phase, load_pkg, need_gpu, norm_intensity_error
from oracle import pyramid

pytestmark = pytest.mark.gpu

EPS = 1e-5

# (n_pix, n_mod, mod_amp, obsc, n_sub, n_batch)
CASES = [
    (32, 8, 3.0, 0.2, 8, 2),      # N = 64
    (64, 12, 3.0, 0.0, 16, 2),    # N = 128
    (120, 16, 3.0, 0.28, 40, 1),  # N = 240
    (160, 24, 2.5, 0.11, 40, 1),  # N = 320
]


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


def _image(torch, sp, ctx, n_pix, n_mod, r, obsc, n_sub, phases, form):
    pu = sp.PupilDesc(n_pix, 0.1, obsc)
    pw = sp.PwfsDesc(2, n_mod, n_sub, n_pix, r)
    sp.specula_pwfs_plan(ctx, pu, pw)
    sp.specula_pwfs_set_form(ctx, pu, pw, form)
    amp = torch.empty(n_pix, n_pix, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    ph = torch.tensor(np.stack(phases).astype(np.float32), device="cuda")
    det = torch.full((len(phases), 2 * n_sub, 2 * n_sub), float("nan"), device="cuda")
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
    torch.cuda.synchronize()
    return amp.cpu().numpy().astype(np.float64), det.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{2 * c[0]}")
def test_shifted_form_parity(env, case):
    torch, sp, ctx = env
    n_pix, n_mod, r, obsc, n_sub, nb = case
    phases = [kolmogorov_phase(n_pix, 8.0 / n_pix, 0.15, seed=11 + k) for k in range(nb)]
    amp, det = _image(torch, sp, ctx, n_pix, n_mod, r, obsc, n_sub, phases, sp.PWFS_FORM_SHIFTED)
    for k in range(nb):
        ref = pyramid.pwfs_image_shifted(amp, phases[k].astype(np.float32).astype(np.float64), 2,
                                         n_mod, r, n_sub, n_pix)
        assert norm_intensity_error(det[k], ref) <= EPS, k


def test_shifted_form_full_size(env):
    """The 39 m pupil: 480 px, 960^2 transforms, 48 points."""
    torch, sp, ctx = env
    n_pix, n_mod, r, n_sub = 480, 48, 3.0, 96
    ph = kolmogorov_phase(n_pix, 39.0 / n_pix, 0.15, seed=5)
    amp, det = _image(torch, sp, ctx, n_pix, n_mod, r, 0.28, n_sub, [ph], sp.PWFS_FORM_SHIFTED)
    ref = pyramid.pwfs_image_shifted(amp, ph.astype(np.float32).astype(np.float64), 2, n_mod, r,
                                     n_sub, n_pix)
    assert norm_intensity_error(det[0], ref) <= EPS


def test_form_switch_and_errors(env):
    """Switching back gives the tilt form again; the two forms differ by the
    wrapped wings (more than the parity tolerance); bad values are refused."""
    torch, sp, ctx = env
    n_pix, n_mod, r, obsc, n_sub = 64, 12, 3.0, 0.0, 16
    ph = [kolmogorov_phase(n_pix, 8.0 / n_pix, 0.15, seed=2)]
    amp, d_s = _image(torch, sp, ctx, n_pix, n_mod, r, obsc, n_sub, ph, sp.PWFS_FORM_SHIFTED)
    _, d_t = _image(torch, sp, ctx, n_pix, n_mod, r, obsc, n_sub, ph, sp.PWFS_FORM_TILT)
    p64 = ph[0].astype(np.float32).astype(np.float64)
    assert norm_intensity_error(d_t, pyramid.pwfs_image(amp, p64, 2, n_mod, r, n_sub, n_pix)) <= EPS
    assert norm_intensity_error(d_s, d_t) > 100 * EPS
    pu = sp.PupilDesc(n_pix, 0.1, obsc)
    pw = sp.PwfsDesc(2, n_mod, n_sub, n_pix, r)
    with pytest.raises(sp.SpeculaError) as e:      # forms 0-3 exist
        sp.specula_pwfs_set_form(ctx, pu, pw, 7)
    assert e.value.status == sp.EINVAL
    sp.specula_pwfs_set_form(ctx, pu, pw, sp.PWFS_FORM_SHIFTED)
    at = torch.tensor(amp.astype(np.float32), device="cuda")
    pt = torch.tensor(p64.astype(np.float32)[None], device="cuda")
    det = torch.empty(1, 2 * n_sub, 2 * n_sub, device="cuda")
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_pwfs_autotune(ctx, pu, pw, at, pt, det)
    assert e.value.status == sp.EUNSUPPORTED
    sp.specula_pwfs_set_form(ctx, pu, pw, sp.PWFS_FORM_TILT)
