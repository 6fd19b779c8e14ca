"""GPU parity: the polychromatic pyramid image (weighted sum over wavelengths
of the image with phase and modulation radius scaled by lambda_ref /
lambda_i) against the FP64 oracle; normalised-intensity error <= 1e-5 as for
the monochromatic image; both modulation forms; batch of two."""
import numpy as np
import pytest

from gpu_common import close_checked, kolmogorov_phase, load_pkg, need_gpu, norm_intensity_error
from oracle import pyramid

pytestmark = pytest.mark.gpu

RATIOS = [1.3, 1.0, 0.75]
WEIGHTS = [0.25, 0.45, 0.3]


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


@pytest.mark.parametrize("n_pix,n_mod,r,obsc,n_sub,form", [
    (64, 12, 3.0, 0.0, 16, 0), (120, 16, 3.0, 0.28, 40, 0), (64, 12, 3.0, 0.0, 16, 1)])
def test_poly_parity(env, n_pix, n_mod, r, obsc, n_sub, form):
    torch, sp, ctx = env
    pu = sp.PupilDesc(n_pix, 0.1, obsc)
    pw = sp.PwfsDesc(2, n_mod, n_sub, n_pix, r)
    sp.specula_pwfs_plan_poly(ctx, pu, pw, RATIOS)
    for q in RATIOS:
        sp.specula_pwfs_set_form(ctx, pu, sp._pwfs_at(pw, q), form)
    amp = torch.empty(n_pix, n_pix, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    phases = [kolmogorov_phase(n_pix, 8.0 / n_pix, 0.15, seed=21 + k).astype(np.float32)
              for k in range(2)]
    ph = torch.tensor(np.stack(phases), device="cuda")
    det = torch.full((2, 2 * n_sub, 2 * n_sub), float("nan"), device="cuda")
    sp.specula_pwfs_image_poly(ctx, pu, pw, RATIOS, WEIGHTS, amp, ph, det)
    torch.cuda.synchronize()
    a64 = amp.cpu().numpy().astype(np.float64)
    img = pyramid.pwfs_image_poly if form == 0 else None
    for k in range(2):
        p64 = phases[k].astype(np.float64)
        if form == 0:
            ref = img(a64, p64, 2, n_mod, r, n_sub, n_pix, RATIOS, WEIGHTS)
        else:
            ref = sum(w * pyramid.pwfs_image_shifted(a64, p64 * q, 2, n_mod, r * q, n_sub, n_pix)
                      for q, w in zip(RATIOS, WEIGHTS))
        assert norm_intensity_error(det[k].cpu().numpy(), ref) <= 1e-5, k
    for q in RATIOS:
        sp.specula_pwfs_set_form(ctx, pu, sp._pwfs_at(pw, q), sp.PWFS_FORM_TILT)


def test_poly_needs_every_plan(env):
    torch, sp, ctx = env
    n_pix, n_sub = 32, 8
    pu = sp.PupilDesc(n_pix, 0.1, 0.2)
    pw = sp.PwfsDesc(2, 8, n_sub, n_pix, 3.0)
    sp.specula_pwfs_plan(ctx, pu, pw)                        # the reference only
    amp = torch.empty(n_pix, n_pix, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    det = torch.zeros(1, 2 * n_sub, 2 * n_sub, device="cuda")
    ph = torch.zeros(1, n_pix, n_pix, device="cuda")
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_pwfs_image_poly(ctx, pu, pw, [1.0, 0.7], [0.5, 0.5], amp, ph, det)
    assert e.value.status == sp.ENOPLAN
    # one wavelength at the reference equals the plain image
    sp.specula_pwfs_image_poly(ctx, pu, pw, [1.0], [1.0], amp, ph, det)
    plain = torch.empty_like(det)
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph, plain)
    torch.cuda.synchronize()
    assert torch.equal(det, plain)
