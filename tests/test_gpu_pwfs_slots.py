"""GPU parity of the pyramid image over a subset of modulation slots (the
modulation-point partition of one frame): each partial detector against the
oracle imaging the same points, partials summing to the full image, batched
elements, the full range restored bit for bit, and the refused forms.

Tolerances: a partial is checked against the oracle's partial to 1e-5 of the
full image's brightest pixel (the full image's normalised-intensity bound);
the sum of the partials against the full GPU image to 2e-6 of that pixel
(the same float32 terms summed in another order)."""
import numpy as np
import pytest

from gpu_common import close_checked, kolmogorov_phase, load_pkg, need_gpu
from oracle import geometry, pyramid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


@pytest.mark.parametrize("n,nsub,n_mod,world", [(160, 40, 24, 3), (480, 96, 48, 4), (64, 16, 7, 2)])
def test_partial_images_match_the_oracle_and_sum_to_the_full(env, n, nsub, n_mod, world):
    torch, sp, ctx = env
    from paper_2602_06688_gb300.sharding import slot_points, slot_ranges
    pu = sp.PupilDesc(n, 8.0 / n, 0.11)
    pw = sp.PwfsDesc(2, n_mod, nsub, n, 3.0)
    sp.specula_pwfs_plan(ctx, pu, pw)
    sp.specula_pwfs_set_tiles(ctx, pu, pw, 8, 1, 2)
    amp = torch.empty(n, n, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    nb = 3
    phs = np.stack([kolmogorov_phase(n, 8.0 / n, 0.15, seed=20 + k) for k in range(nb)])
    ph = torch.tensor(phs.astype(np.float32), device="cuda")
    d = 2 * nsub
    full = torch.empty(nb, d, d, device="cuda")
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph, full)
    parts = []
    for a, b in slot_ranges(n_mod, world):
        sp.specula_pwfs_set_slots(ctx, pu, pw, a, b)
        det = torch.full((nb, d, d), float("nan"), device="cuda")
        sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
        parts.append(((a, b), det))
    torch.cuda.synchronize()
    a64 = amp.cpu().numpy().astype(np.float64)
    full_np = full.cpu().numpy().astype(np.float64)
    for k in (0, nb - 1):
        p64 = ph[k].cpu().numpy().astype(np.float64)
        ref_full = pyramid.bin_image(pyramid.pwfs_intensity(a64, p64, 2, n_mod, 3.0, n), n // nsub)
        peak = ref_full.max()
        for (a, b), det in parts:
            pts = [m for c in range(a, b) for m in slot_points(n_mod, c)]
            ref = pyramid.bin_image(pyramid.pwfs_intensity(a64, p64, 2, n_mod, 3.0, n, points=pts),
                                    n // nsub)
            assert np.max(np.abs(det[k].cpu().numpy() - ref)) <= 1e-5 * peak
        tot = sum(det[k].cpu().numpy().astype(np.float64) for _, det in parts)
        assert np.max(np.abs(tot - full_np[k])) <= 2e-6 * peak
    # the full range again: bit-identical to the first full image
    sp.specula_pwfs_set_slots(ctx, pu, pw, 0, n_mod // 2 + 1)
    again = torch.empty_like(full)
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph, again)
    torch.cuda.synchronize()
    assert torch.equal(again, full)


def test_refused_forms_and_ranges(env):
    torch, sp, ctx = env
    n, nsub, n_mod = 64, 16, 8
    pu = sp.PupilDesc(n, 0.1, 0.1)
    pw = sp.PwfsDesc(2, n_mod, nsub, n, 2.0)
    sp.specula_pwfs_plan(ctx, pu, pw)
    for a, b in ((0, 0), (-1, 2), (3, 2), (0, n_mod // 2 + 2)):
        with pytest.raises(sp.SpeculaError) as e:
            sp.specula_pwfs_set_slots(ctx, pu, pw, a, b)
        assert e.value.status == sp.EINVAL
    amp = torch.ones(n, n, device="cuda")
    ph = torch.zeros(n, n, device="cuda")
    det = torch.empty(2 * nsub, 2 * nsub, device="cuda")
    sp.specula_pwfs_set_slots(ctx, pu, pw, 1, 3)
    sp.specula_pwfs_set_tiles(ctx, pu, pw, 4, 1, 3)
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
    assert e.value.status == sp.EUNSUPPORTED
    sp.specula_pwfs_set_tiles(ctx, pu, pw, 4, 1, 2)
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
    sp.specula_pwfs_set_slots(ctx, pu, pw, 0, n_mod // 2 + 1)
    torch.cuda.synchronize()
