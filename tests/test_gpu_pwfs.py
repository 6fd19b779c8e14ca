"""GPU parity: modulated pyramid image and slopes vs the FP64 oracle.

Tolerance (FP32 path): normalised-intensity max relative error <= 1e-5, on
the unbinned N x N intensity and on the binned detector.  Slopes are ratios
of detector sums: with |d det| <= eps max(det) per pixel, each slope moves by
at most (4 eps max(det) + |S| |dT|) / T <= 5 eps max(det) / T + eps |S|; the
tests use eps = 1e-5.
"""
import math

import numpy as np
import pytest

from gpu_common import (close_checked, kolmogorov_phase, load_pkg,
                        need_gpu, norm_intensity_error, pupil_amp)
from oracle import geometry, pyramid, slopes

pytestmark = pytest.mark.gpu

EPS = 1e-5

# (n_pix, n_mod, mod_amp, obsc, n_sub, n_batch, chunk, ka)
CASES = [
    (32, 8, 3.0, 0.2, 8, 3, 5, 2),       # N = 64, ragged chunks across batch elements
    (64, 12, 3.0, 0.0, 16, 2, 64, 2),    # N = 128: the 8 m tiny system
    (120, 16, 3.0, 0.28, 40, 1, 7, 3),   # N = 240: the 39 m NGS pyramid
    (160, 24, 3.0, 0.11, 40, 1, 24, 2),  # N = 320: the 8 m system
]


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


def _run(torch, sp, ctx, n_pix, n_mod, r, obsc, n_sub, phases, chunk=None, ka=None,
         passes=None):
    pu = sp.PupilDesc(n_pix, 0.1, obsc)
    pw = sp.PwfsDesc(2, n_mod, n_sub, n_pix, r)
    sp.specula_pwfs_plan(ctx, pu, pw)
    if chunk or passes:
        ch0, ka0, ps0 = sp.specula_pwfs_get_tiles(ctx, pu, pw)
        sp.specula_pwfs_set_tiles(ctx, pu, pw, chunk or ch0, ka or ka0, passes or ps0)
    amp = torch.empty(n_pix, n_pix, device="cuda", dtype=torch.float32)
    sp.specula_pupil_mask(ctx, pu, amp)
    ph = torch.tensor(np.stack(phases).astype(np.float32), device="cuda")
    det = torch.full((len(phases), 2 * n_sub, 2 * n_sub), float("nan"), device="cuda")
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
    torch.cuda.synchronize()
    return det.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("passes", [2, 3])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{2 * c[0]}")
def test_pwfs_intensity_and_detector_parity(env, case, passes):
    """Both forms of the 2D filter (separable two-pass, three-pass) against
    the oracle."""
    torch, sp, ctx = env
    n_pix, n_mod, r, obsc, n_sub, nb, chunk, ka = case
    amp = pupil_amp(n_pix, obsc)
    phases = [kolmogorov_phase(n_pix, 8.0 / n_pix, 0.15, seed=11 + k).astype(np.float32)
              for k in range(nb)]
    # unbinned: n_sub = n_pix gives the N x N intensity
    I_gpu = _run(torch, sp, ctx, n_pix, n_mod, r, obsc, n_pix, phases, chunk, ka, passes)
    det_gpu = _run(torch, sp, ctx, n_pix, n_mod, r, obsc, n_sub, phases, chunk, ka, passes)
    for k in range(nb):
        I_ref = pyramid.pwfs_intensity(amp, phases[k].astype(np.float64), 2, n_mod, r, n_pix)
        e1 = norm_intensity_error(I_gpu[k], I_ref)
        assert e1 <= EPS, (k, e1)
        # flux: sum of the detector = number of pupil pixels (FP32 accumulation)
        assert abs(I_gpu[k].sum() - amp.sum()) <= 1e-5 * amp.sum()
        det_ref = pyramid.bin_image(I_ref, n_pix // n_sub)
        e2 = norm_intensity_error(det_gpu[k], det_ref)
        assert e2 <= EPS, (k, e2)


def test_pwfs_deterministic_and_flat_symmetric(env):
    torch, sp, ctx = env
    n_pix, n_mod, n_sub = 64, 12, 16
    flat = [np.zeros((n_pix, n_pix), np.float32)]
    a = _run(torch, sp, ctx, n_pix, n_mod, 3.0, 0.0, n_sub, flat)
    b = _run(torch, sp, ctx, n_pix, n_mod, 3.0, 0.0, n_sub, flat)
    assert np.array_equal(a, b)
    d = a[0]
    q = [d[16:, 16:].sum(), d[16:, :16].sum(), d[:16, :16].sum(), d[:16, 16:].sum()]
    assert np.allclose(q, d.sum() / 4, rtol=1e-5)
    assert np.allclose(d, d[:, ::-1], atol=1e-5 * d.max())


def test_pwfs_slopes_parity(env):
    torch, sp, ctx = env
    n_pix, n_mod, r, obsc, n_sub = 160, 24, 3.0, 0.11, 40
    amp = pupil_amp(n_pix, obsc)
    valid = geometry.valid_subaps(amp.astype(np.uint8), n_sub)
    phi = kolmogorov_phase(n_pix, 8.4 / n_pix, 0.12, seed=21).astype(np.float32)
    det_gpu_t = None
    pu = sp.PupilDesc(n_pix, 8.4 / n_pix, obsc)
    pw = sp.PwfsDesc(2, n_mod, n_sub, n_pix, r)
    sp.specula_pwfs_plan(ctx, pu, pw)
    amp_t = torch.tensor(amp.astype(np.float32), device="cuda")
    idx = torch.tensor(valid, device="cuda")
    dets = torch.empty(2, 2 * n_sub, 2 * n_sub, device="cuda")
    ph = torch.tensor(np.stack([np.zeros_like(phi), phi]), device="cuda")
    sp.specula_pwfs_image(ctx, pu, pw, amp_t, ph, dets)
    sc = sp.slopec_desc(sp.SLOPES_PYR, n_sub, idx)
    ref_t = torch.empty(2 * len(valid), device="cuda")
    sp.specula_slopes(ctx, sc, dets[0], None, ref_t)
    s_t = torch.empty(2 * len(valid), device="cuda")
    sp.specula_slopes(ctx, sc, dets[1], ref_t, s_t)
    torch.cuda.synchronize()
    det_gpu_t = dets.cpu().numpy().astype(np.float64)
    # (1) slope kernel alone on identical input: float32 rounding only
    s_same = slopes.pyr_slopes(det_gpu_t[1], n_sub, valid,
                               ref=slopes.pyr_slopes(det_gpu_t[0], n_sub, valid))
    T = np.mean(det_gpu_t[1].sum()) / len(valid)
    assert np.max(np.abs(s_t.cpu().numpy() - s_same)) <= 1e-6 * (1 + np.abs(s_same).max())
    # (2) end to end against the oracle's own detector
    det0 = pyramid.pwfs_image(amp, np.zeros((n_pix, n_pix)), 2, n_mod, r, n_sub, n_pix)
    det1 = pyramid.pwfs_image(amp, phi.astype(np.float64), 2, n_mod, r, n_sub, n_pix)
    s_ref = slopes.pyr_slopes(det1, n_sub, valid, ref=slopes.pyr_slopes(det0, n_sub, valid))
    T = det1.sum() / len(valid)
    tol = 5 * EPS * det1.max() / T + EPS * np.abs(s_ref).max()
    err = np.max(np.abs(s_t.cpu().numpy() - s_ref))
    assert err <= 2 * tol, (err, tol)   # factor 2: reference slopes carry the same bound


def test_pwfs_full_size_elt(env):
    """The 39 m ELT-scale geometry at full size (480 px pupil, 960^2 FFT, 48
    modulation points, 96 x 96 subapertures), one frame, compared in full,
    in both forms of the 2D filter."""
    torch, sp, ctx = env
    n_pix, n_mod, r, obsc, n_sub = 480, 48, 4.0, 0.28, 96
    amp = pupil_amp(n_pix, obsc)
    phi = kolmogorov_phase(n_pix, 39.0 / n_pix, 0.157, seed=5, side=1024).astype(np.float32)
    I_ref = pyramid.pwfs_intensity(amp, phi.astype(np.float64), 2, n_mod, r, n_pix)
    det_ref = pyramid.bin_image(I_ref, n_pix // n_sub)
    for passes in (2, 3):
        det_gpu = _run(torch, sp, ctx, n_pix, n_mod, r, obsc, n_sub, [phi], passes=passes)[0]
        assert norm_intensity_error(det_gpu, det_ref) <= EPS, passes
        I_gpu = _run(torch, sp, ctx, n_pix, n_mod, r, obsc, n_pix, [phi], passes=passes)[0]
        assert norm_intensity_error(I_gpu, I_ref) <= EPS, passes


def test_plan_required_and_bad_args(env):
    torch, sp, ctx = env
    pu = sp.PupilDesc(64, 0.1, 0.0)
    pw = sp.PwfsDesc(2, 7, 16, 64, 3.0)    # never planned
    amp = torch.zeros(64 * 64, device="cuda")
    det = torch.zeros(32 * 32, device="cuda")
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_pwfs_image(ctx, pu, pw, amp, amp, det)
    assert e.value.status == sp.ENOPLAN
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_pwfs_plan(ctx, sp.PupilDesc(50, 0.1, 0.0), sp.PwfsDesc(2, 4, 10, 50, 3.0))
    assert e.value.status == sp.EUNSUPPORTED
    with pytest.raises(sp.SpeculaError) as e:                 # images beyond the grid
        sp.specula_pwfs_plan(ctx, pu, sp.PwfsDesc(2, 4, 16, 70, 3.0))
    assert e.value.status == sp.EUNSUPPORTED
    with pytest.raises(sp.SpeculaError) as e:                 # padding 5
        sp.specula_pwfs_plan(ctx, pu, sp.PwfsDesc(5, 4, 16, 64, 3.0))
    assert e.value.status == sp.EUNSUPPORTED


def test_tiling_invariance_and_autotune(env):
    """For each form of the 2D filter, every (chunk, ka) tiling gives a
    bit-identical detector (item bins are reduced in modulation order
    whatever the chunking); the two forms agree to float rounding; the
    autotuner returns one of the candidates."""
    torch, sp, ctx = env
    n_pix, n_mod, n_sub = 32, 8, 8
    pu = sp.PupilDesc(n_pix, 0.25, 0.2)
    pw = sp.PwfsDesc(2, n_mod, n_sub, n_pix, 3.0)
    sp.specula_pwfs_plan(ctx, pu, pw)
    amp = torch.empty(n_pix, n_pix, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    ph = torch.tensor(np.stack([kolmogorov_phase(n_pix, 0.25, 0.15, seed=s) for s in (1, 2, 3)])
                      .astype(np.float32), device="cuda")
    first = {}
    for passes in (2, 3):
        outs = []
        for chunk, ka in [(1, 1), (3, 2), (5, 1), (8, 2), (24, 1)]:
            sp.specula_pwfs_set_tiles(ctx, pu, pw, chunk, ka, passes)
            det = torch.empty(3, 2 * n_sub, 2 * n_sub, device="cuda")
            sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
            torch.cuda.synchronize()
            outs.append(det.cpu())
        for o in outs[1:]:
            assert torch.equal(o, outs[0])
        first[passes] = outs[0]
    for k in range(3):
        assert norm_intensity_error(first[2][k].numpy(), first[3][k].numpy()) <= 1e-6
    det = torch.empty(3, 2 * n_sub, 2 * n_sub, device="cuda")
    ch, ka, ps = sp.specula_pwfs_autotune(ctx, pu, pw, amp, ph, det, reps=2)
    assert ch in (1, 2, 3, 4, 6, 8, 12, 16, 24) and ka in (1, 2) and ps in (2, 3)
    assert sp.specula_pwfs_get_tiles(ctx, pu, pw) == (ch, ka, ps)
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
    torch.cuda.synchronize()
    assert torch.equal(det.cpu(), first[ps])
