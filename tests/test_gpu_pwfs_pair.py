"""GPU parity of the packed-pair two-pass pyramid form (passes = 4: two
transforms per thread in float32 pairs) against the FP64 oracle.

Tolerance: the FP32 path's normalised-intensity max relative error <= 1e-5
on the unbinned N x N intensity and on the binned detector, as for the other
forms (the packed instructions round each float32 operation as the scalar
ones do; only the order of a few additions differs).  Against the scalar
two-pass form: 1e-6 (both are float32 evaluations of the same transforms).
The pair units cover the points m and n_mod - m of a slot, the two unpaired
points 0 and n_mod / 2 together, and a last unpaired point with itself (odd
n_mod); each has a case here."""
import numpy as np
import pytest

from gpu_common import (close_checked, kolmogorov_phase, load_pkg, need_gpu,
                        norm_intensity_error, pupil_amp)
from oracle import pyramid

pytestmark = pytest.mark.gpu

EPS = 1e-5


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


def _image(torch, sp, ctx, n_pix, n_mod, r, obsc, n_sub, phases, passes, chunk=64):
    pu = sp.PupilDesc(n_pix, 0.1, obsc)
    pw = sp.PwfsDesc(2, n_mod, n_sub, n_pix, r)
    sp.specula_pwfs_plan(ctx, pu, pw)
    sp.specula_pwfs_set_tiles(ctx, pu, pw, chunk, 1, passes)
    amp = torch.empty(n_pix, n_pix, device="cuda", dtype=torch.float32)
    sp.specula_pupil_mask(ctx, pu, amp)
    ph = torch.tensor(np.stack(phases).astype(np.float32), device="cuda")
    det = torch.full((len(phases), 2 * n_sub, 2 * n_sub), float("nan"), device="cuda")
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
    torch.cuda.synchronize()
    return det.cpu().numpy().astype(np.float64)


# (n_pix, n_mod, mod_amp, obsc, n_sub, n_batch)
CASES = [
    (160, 24, 3.0, 0.11, 40, 2),   # N = 320, the 8 m system, two batch elements
    (160, 15, 3.0, 0.11, 40, 1),   # odd n_mod: point 0 paired with itself
    (160, 1, 0.0, 0.11, 40, 1),    # one point, no modulation: the static pyramid
    (480, 48, 4.0, 0.28, 96, 1),   # N = 960, the ELT pyramid
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{2 * c[0]}_m{c[1]}")
def test_pair_form_against_the_oracle(env, case):
    torch, sp, ctx = env
    n_pix, n_mod, r, obsc, n_sub, nb = case
    amp = pupil_amp(n_pix, obsc)
    side = 1024 if n_pix > 256 else None
    phases = [kolmogorov_phase(n_pix, 8.0 / n_pix, 0.15, seed=31 + k, side=side)
              .astype(np.float32) for k in range(nb)]
    I_gpu = _image(torch, sp, ctx, n_pix, n_mod, r, obsc, n_pix, phases, 4)
    det_gpu = _image(torch, sp, ctx, n_pix, n_mod, r, obsc, n_sub, phases, 4)
    det_two = _image(torch, sp, ctx, n_pix, n_mod, r, obsc, n_sub, phases, 2)
    for k in range(nb):
        I_ref = pyramid.pwfs_intensity(amp, phases[k].astype(np.float64), 2, n_mod, r, n_pix)
        assert norm_intensity_error(I_gpu[k], I_ref) <= EPS
        assert abs(I_gpu[k].sum() - amp.sum()) <= 1e-5 * amp.sum()
        det_ref = pyramid.bin_image(I_ref, n_pix // n_sub)
        assert norm_intensity_error(det_gpu[k], det_ref) <= EPS
        assert norm_intensity_error(det_gpu[k], det_two[k]) <= 1e-6


def test_pair_tiling_is_bit_identical_and_the_autotuner_offers_it(env):
    """Whole batch elements per launch: 1, 2 and 3 elements per chunk give the
    same detector bit for bit; the autotuner's choice reproduces its form."""
    torch, sp, ctx = env
    n_pix, n_mod, n_sub = 160, 24, 40
    phases = [kolmogorov_phase(n_pix, 0.05, 0.15, seed=s).astype(np.float32) for s in (4, 5, 6)]
    nc = n_mod // 2 + 1
    outs = [_image(torch, sp, ctx, n_pix, n_mod, 3.0, 0.11, n_sub, phases, 4, chunk=c * nc)
            for c in (1, 2, 3)]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    pu = sp.PupilDesc(n_pix, 0.1, 0.11)
    pw = sp.PwfsDesc(2, n_mod, n_sub, n_pix, 3.0)
    assert sp.specula_pwfs_get_tiles(ctx, pu, pw) == (3 * nc, 1, 4)
    amp = torch.empty(n_pix, n_pix, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    ph = torch.tensor(np.stack(phases), device="cuda")
    det = torch.empty(3, 2 * n_sub, 2 * n_sub, device="cuda")
    ch, ka, ps = sp.specula_pwfs_autotune(ctx, pu, pw, amp, ph, det, reps=2)
    assert ps in (2, 3, 4)
    if ps == 4:
        assert ch % nc == 0 and ka == 1
        sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
        torch.cuda.synchronize()
        assert np.array_equal(det.cpu().numpy().astype(np.float64), outs[0])


@pytest.mark.parametrize("ranges", [[(0, 5), (5, 13)], [(0, 1), (1, 12), (12, 13)]])
def test_pair_form_on_slot_ranges(env, ranges):
    """Partial images over modulation-slot ranges (the point partition of a
    frame) in the paired form: each against the oracle on its points; the
    ranges split the unpaired points 0 and n_mod / 2 differently."""
    torch, sp, ctx = env
    from paper_2602_06688_gb300.sharding import slot_points
    n, nsub, n_mod = 160, 40, 24
    pu = sp.PupilDesc(n, 8.0 / n, 0.11)
    pw = sp.PwfsDesc(2, n_mod, nsub, n, 3.0)
    sp.specula_pwfs_plan(ctx, pu, pw)
    sp.specula_pwfs_set_tiles(ctx, pu, pw, 64, 1, 4)
    amp = torch.empty(n, n, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    phi = kolmogorov_phase(n, 8.0 / n, 0.15, seed=77)
    ph = torch.tensor(phi[None].astype(np.float32), device="cuda")
    a64 = amp.cpu().numpy().astype(np.float64)
    p64 = ph[0].cpu().numpy().astype(np.float64)
    peak = pyramid.bin_image(pyramid.pwfs_intensity(a64, p64, 2, n_mod, 3.0, n), n // nsub).max()
    tot = 0.0
    for a, b in ranges:
        sp.specula_pwfs_set_slots(ctx, pu, pw, a, b)
        det = torch.full((1, 2 * nsub, 2 * nsub), float("nan"), device="cuda")
        sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
        torch.cuda.synchronize()
        pts = [m for c in range(a, b) for m in slot_points(n_mod, c)]
        ref = pyramid.bin_image(pyramid.pwfs_intensity(a64, p64, 2, n_mod, 3.0, n, points=pts),
                                n // nsub)
        got = det[0].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - ref)) <= 1e-5 * peak
        tot = tot + got
    sp.specula_pwfs_set_slots(ctx, pu, pw, 0, n_mod // 2 + 1)
    full = torch.empty(1, 2 * nsub, 2 * nsub, device="cuda")
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph, full)
    torch.cuda.synchronize()
    assert np.max(np.abs(tot - full[0].cpu().numpy())) <= 2e-6 * peak


def test_pair_form_refused_where_unsupported(env):
    torch, sp, ctx = env
    for n_pix, n_sub, pad, dist in [(120, 40, 2, 120), (64, 16, 2, 64), (80, 40, 3, 96)]:
        pu = sp.PupilDesc(n_pix, 0.1, 0.0)
        pw = sp.PwfsDesc(pad, 8, n_sub, dist, 3.0)
        sp.specula_pwfs_plan(ctx, pu, pw)
        with pytest.raises(sp.SpeculaError) as e:
            sp.specula_pwfs_set_tiles(ctx, pu, pw, 16, 1, 4)
        assert e.value.status == sp.EUNSUPPORTED
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_pwfs_set_tiles(ctx, sp.PupilDesc(160, 0.1, 0.0),
                                  sp.PwfsDesc(2, 8, 40, 160, 3.0), 16, 1, 5)
    assert e.value.status == sp.EINVAL
