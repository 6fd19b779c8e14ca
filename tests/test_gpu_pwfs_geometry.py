"""GPU parity of the pyramid with other paddings and image separations (the
SOUL example's geometry) and of the slope computer driven by image index
maps, against the FP64 oracle; the whole SOUL-geometry frame against the
oracle chain.  Tolerances as for the pad-2 pyramid: normalised-intensity
error <= 1e-5; slopes within 2 (5e-5 max(det) / T + 1e-5 max|S|)."""
import numpy as np
import pytest

import synth
from gpu_common import close_checked, kolmogorov_phase, load_pkg, need_gpu, norm_intensity_error
from oracle import atmo, geometry, pyramid, recon, slopes

pytestmark = pytest.mark.gpu

# (n_pix, pad, pup_dist_px, n_sub, n_mod): SOUL (N 240), pad 4 (N 128, 64),
# the 960^2 grid at pad 3, and pad 2 with images closer than their width;
# fractional detector pixels (area-weighted rebinning in the column pass):
# the paper's SOUL as stated (220 px pupil, 660^2 grid, 24 points, 5.5 grid
# pixels per detector pixel), a 240 grid with 2.5 px detector pixels
# (16-lane transforms), pad 2 on a 320 grid with 2.5 px detector pixels, and
# an odd pupil side (165 px at pad 4 on the 660 grid: the row pass writes
# its transposed rows one complex at a time)
CASES = [(80, 3, 96, 40, 16), (32, 4, 48, 8, 8), (16, 4, 24, 4, 8), (320, 3, 384, 80, 16),
         (64, 2, 48, 16, 12), (220, 3, 264, 40, 24), (80, 3, 100, 32, 16), (160, 2, 160, 64, 12),
         (165, 4, 195, 33, 8)]


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"np{c[0]}_pad{c[1]}_pd{c[2]}")
def test_image_and_map_slopes_parity(env, case):
    torch, sp, ctx = env
    n, pad, pd, nsub, nmod = case
    pu = sp.PupilDesc(n, 8.0 / n, 0.11)
    pw = sp.PwfsDesc(pad, nmod, nsub, pd, 3.0)
    sp.specula_pwfs_plan(ctx, pu, pw)
    amp = torch.empty(n, n, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    a64 = amp.cpu().numpy().astype(np.float64)
    phs = [kolmogorov_phase(n, 8.0 / n, 0.15, seed=7 + k).astype(np.float32) for k in range(3)]
    ph = phs[0]
    side = pad * nsub
    det = torch.full((3, side, side), float("nan"), device="cuda")
    ph_t = torch.tensor(np.stack(phs), device="cuda")
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph_t, det)
    torch.cuda.synchronize()
    # the inputs are untouched (a canary for writes outside the plan's buffers)
    assert np.array_equal(amp.cpu().numpy().astype(np.float64), a64)
    assert np.array_equal(ph_t.cpu().numpy(), np.stack(phs))
    for k in range(3):
        ref = pyramid.pwfs_image(a64, phs[k].astype(np.float64), pad, nmod, 3.0, nsub, pd)
        assert norm_intensity_error(det[k].cpu().numpy(), ref) <= 1e-5, k
    # slopes from image maps (host maps = oracle maps), against the oracle on
    # the GPU's own detector
    maps = sp.specula_pyr_image_index_host(pu, pad, pd, nsub)
    valid = geometry.valid_subaps(a64.astype(np.uint8), nsub)
    assert np.array_equal(maps, geometry.pyr_image_index(valid, nsub, pad, pd, n))
    mt = torch.tensor(maps.ravel(), device="cuda")
    sc = sp.slopec_desc(sp.SLOPES_PYR_MAPS, side, mt)
    sl = torch.empty(2 * maps.shape[1], device="cuda")
    sp.specula_slopes(ctx, sc, det[0], None, sl)
    torch.cuda.synchronize()
    s_ref = slopes.pyr_slopes_maps(det[0].cpu().numpy().astype(np.float64), maps)
    assert np.max(np.abs(sl.cpu().numpy() - s_ref)) <= 1e-5 * (1 + np.abs(s_ref).max())
    del ph


@pytest.mark.parametrize("nsub,nmod,nb", [(100, 24, 1), (400, 4, 2)], ids=["andes", "unbinned"])
def test_andes_grid_parity(env, nsub, nmod, nb):
    """The ANDES grid of Sect. 6, Tab. 2 (400 px pupil at pad 4: 1600^2 =
    32 x 50, the 50-point stage in two lane strides): the 100 x 100
    subaperture detector with 24 points, and the unbinned 1600^2 intensity
    (batch 2), against the FP64 oracle; map slopes of the binned image."""
    torch, sp, ctx = env
    n, pad, pd = 400, 4, 480
    pu = sp.PupilDesc(n, 39.0 / n, 0.28)
    pw = sp.PwfsDesc(pad, nmod, nsub, pd, 3.0)
    sp.specula_pwfs_plan(ctx, pu, pw)
    amp = torch.empty(n, n, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    a64 = amp.cpu().numpy().astype(np.float64)
    phs = [kolmogorov_phase(n, 39.0 / n, 0.16, seed=21 + k).astype(np.float32) for k in range(nb)]
    side = pad * nsub
    det = torch.full((nb, side, side), float("nan"), device="cuda")
    ph_t = torch.tensor(np.stack(phs), device="cuda")
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph_t, det)
    torch.cuda.synchronize()
    assert np.array_equal(ph_t.cpu().numpy(), np.stack(phs))
    for k in range(nb):
        ref = pyramid.pwfs_image(a64, phs[k].astype(np.float64), pad, nmod, 3.0, nsub, pd)
        assert norm_intensity_error(det[k].cpu().numpy(), ref) <= 1e-5, k
    if nsub == n:
        return
    maps = sp.specula_pyr_image_index_host(pu, pad, pd, nsub)
    valid = geometry.valid_subaps(a64.astype(np.uint8), nsub)
    assert np.array_equal(maps, geometry.pyr_image_index(valid, nsub, pad, pd, n))
    mt = torch.tensor(maps.ravel(), device="cuda")
    sl = torch.empty(2 * maps.shape[1], device="cuda")
    sp.specula_slopes(ctx, sp.slopec_desc(sp.SLOPES_PYR_MAPS, side, mt), det[0], None, sl)
    torch.cuda.synchronize()
    s_ref = slopes.pyr_slopes_maps(det[0].cpu().numpy().astype(np.float64), maps)
    assert np.max(np.abs(sl.cpu().numpy() - s_ref)) <= 1e-5 * (1 + np.abs(s_ref).max())


def test_andes_grid_forms(env):
    """At N = 1600 only the two-pass form exists: the three-pass and paired
    tilings and the shifted-mask and DFT-as-GEMM forms are refused with
    SPECULA_EUNSUPPORTED, and the autotuner keeps the two-pass form."""
    torch, sp, ctx = env
    n = 400
    pu = sp.PupilDesc(n, 39.0 / n, 0.28)
    pw = sp.PwfsDesc(4, 8, 100, 480, 3.0)
    sp.specula_pwfs_plan(ctx, pu, pw)
    for passes in (3, 4):
        with pytest.raises(sp.SpeculaError) as e:
            sp.specula_pwfs_set_tiles(ctx, pu, pw, 4, 1, passes)
        assert e.value.status == sp.EUNSUPPORTED
    for form in (sp.PWFS_FORM_SHIFTED, sp.PWFS_FORM_DFTGEMM_BF16):
        with pytest.raises(sp.SpeculaError) as e:
            sp.specula_pwfs_set_form(ctx, pu, pw, form)
        assert e.value.status == sp.EUNSUPPORTED
    amp = torch.empty(n, n, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    ph = torch.tensor(kolmogorov_phase(n, 39.0 / n, 0.16, seed=5).astype(np.float32)[None],
                      device="cuda")
    det = torch.empty(1, 400, 400, device="cuda")
    chunk, ka, passes = sp.specula_pwfs_autotune(ctx, pu, pw, amp, ph, det, reps=2)
    assert passes == 2
    ref = torch.empty_like(det)
    sp.specula_pwfs_set_tiles(ctx, pu, pw, 1, 1, 2)
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph, ref)
    sp.specula_pwfs_set_tiles(ctx, pu, pw, chunk, ka, 2)
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
    torch.cuda.synchronize()
    assert torch.equal(det, ref)   # the tiling does not change the arithmetic


def test_maps_equal_quadrants_bit_exact(env):
    """At pad 2 with touching images the map-driven kernel reproduces the
    quadrant kernel bit for bit (same indices, same summation order)."""
    torch, sp, ctx = env
    n, nsub = 64, 16
    pu = sp.PupilDesc(n, 0.125, 0.1)
    pw = sp.PwfsDesc(2, 12, nsub, n, 3.0)
    sp.specula_pwfs_plan(ctx, pu, pw)
    amp = torch.empty(n, n, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    ph = torch.tensor(kolmogorov_phase(n, 0.125, 0.15, seed=9).astype(np.float32)[None],
                      device="cuda")
    det = torch.empty(1, 2 * nsub, 2 * nsub, device="cuda")
    sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
    valid = torch.tensor(sp.specula_valid_subaps_host(pu, nsub), device="cuda")
    maps = torch.tensor(sp.specula_pyr_image_index_host(pu, 2, n, nsub).ravel(), device="cuda")
    a, b = torch.empty(2 * valid.numel(), device="cuda"), torch.empty(2 * valid.numel(), device="cuda")
    sp.specula_slopes(ctx, sp.slopec_desc(sp.SLOPES_PYR, nsub, valid), det, None, a)
    sp.specula_slopes(ctx, sp.slopec_desc(sp.SLOPES_PYR_MAPS, 2 * nsub, maps), det, None, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("name", ["soul8m", "soul220", "andes400"])
def test_soul_frame_vs_oracle_chain(env, name):
    """The SOUL-geometry frame (40 x 40 subapertures, images 48 detector px
    apart on 120 px; soul8m: 80 px pupil with 2 x 2 bins, soul220: the
    paper's 220 px pupil on a 660^2 grid with 5.5 px detector pixels) and
    the ANDES frame (400 px pupil on a 1600^2 grid, 100 x 100 subapertures,
    35 layers, 4000 modes): extraction, image, map slopes, MVM against the
    oracle chain."""
    torch, sp, ctx = env
    from paper_2602_06688_gb300.frame import PwfsFrame
    wl = synth.workload(name)
    fr = PwfsFrame(ctx, wl)
    s = wl.sensors[0]
    n, g = s.pupil.n_pix, s.pwfs
    t = 0.071
    fr.frame(t)
    torch.cuda.synchronize()
    assert fr.det.shape[-1] == g.pad * g.n_sub and not fr.quadrants
    scr = [x.cpu().numpy().astype(np.float64) for x in fr.screens]
    phi = atmo.atmo_extract(scr, wl.layers, s.source, n, s.pupil.pitch_m, t)
    amp = geometry.pupil_mask(n, s.pupil.obsc_frac).astype(np.float64)
    valid = geometry.valid_subaps(amp.astype(np.uint8), g.n_sub)
    maps = geometry.pyr_image_index(valid, g.n_sub, g.pad, g.pup_dist_px, n)
    det_ref = pyramid.pwfs_image(amp, phi, g.pad, g.n_mod, g.mod_amp, g.n_sub, g.pup_dist_px)
    flat = pyramid.pwfs_image(amp, np.zeros_like(phi), g.pad, g.n_mod, g.mod_amp, g.n_sub,
                              g.pup_dist_px)
    assert norm_intensity_error(fr.det.cpu().numpy().astype(np.float64), det_ref) <= 1e-5
    s_ref = slopes.pyr_slopes_maps(det_ref, maps, ref=slopes.pyr_slopes_maps(flat, maps))
    T = det_ref.ravel()[maps].sum() / len(valid)
    tol = 2 * (5e-5 * det_ref.max() / T + 1e-5 * np.abs(s_ref).max())
    sl = fr.slopes.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(sl - s_ref)) <= tol
    R = fr.R.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(fr.modes.cpu().numpy() - recon.mvm(R, sl)) <= 1e-5 * (np.abs(R) @ np.abs(sl)))
