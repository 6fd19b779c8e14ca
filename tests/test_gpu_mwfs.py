"""GPU parity of the multi-sensor system in one persistent launch (every
sensor's phase, image and slopes, and the reconstructor product) against the
oracle chains; agreement with the per-sensor calls; invariance under the
number of CTAs; graph replay; the full 39 m system on sampled outputs."""
import numpy as np
import pytest

import synth
from gpu_common import close_checked, load_pkg, need_gpu, norm_intensity_error
from oracle import atmo, geometry, pyramid, recon, sh, slopes, system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


@pytest.fixture(scope="module")
def small(env):
    torch, sp, ctx = env
    from paper_2602_06688_gb300.system import System
    return System(ctx, synth.workload("mwfs8m_small"))


def _read(torch, sp, S, k, what, shape):
    out = torch.empty(*shape, device="cuda")
    S.m.read(k, what, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _sh_bound(spots, fft_n):
    # CoG error from a spot error <= 1e-5 of its peak (see test_gpu_sh_recon)
    b = 1e-5 * fft_n ** 3 * (spots.max(axis=(1, 2)) / spots.sum(axis=(1, 2)))
    return np.concatenate([b, b]) + 1e-6


def _covered(sen, amp):
    """Pixels whose phase the launch computes: the whole grid for a pyramid,
    the valid subapertures' pixels for a Shack-Hartmann sensor."""
    n = amp.shape[0]
    if sen.kind == "pwfs":
        return np.ones((n, n), dtype=bool)
    g = sen.sh
    cov = np.zeros((n, n), dtype=bool)
    for idx in geometry.valid_subaps(amp.astype(np.uint8), g.n_sub):
        a, b = divmod(int(idx), g.n_sub)
        cov[a * g.sub_pix:(a + 1) * g.sub_pix, b * g.sub_pix:(b + 1) * g.sub_pix] = True
    return cov


def _check_system(torch, sp, S, t, idx_sample=None):
    """Every sensor against the oracle: phase against the oracle extraction;
    image and slopes against the oracle run on the GPU's own phase (so each
    stage is held to its own tolerance); modes against the oracle MVM of the
    GPU's slopes."""
    scr = [x.cpu().numpy().astype(np.float64) for x in S.screens]
    got = S.slopes.cpu().numpy().astype(np.float64)
    gref = S.ref.cpu().numpy().astype(np.float64)
    for k, sen in enumerate(S.wl.sensors):
        n = sen.pupil.n_pix
        o, nv = S.offsets[k], S.n_valid[k]
        ph = _read(torch, sp, S, k, sp.MWFS_PHASE, (n, n))
        phi = atmo.atmo_extract(scr, S.wl.layers, sen.source, n, sen.pupil.pitch_m, t)
        amp = geometry.pupil_mask(n, sen.pupil.obsc_frac).astype(np.float64)
        cover = _covered(sen, amp)
        assert np.max(np.abs(ph - phi)[cover]) <= 1e-5 * (1 + np.abs(phi).max()), k
        assert np.all(ph[~cover] == 0.0), k
        blk, rblk = got[o:o + 2 * nv], gref[o:o + 2 * nv]
        if sen.kind == "sh":
            g = sen.sh
            valid = geometry.valid_subaps(amp.astype(np.uint8), g.n_sub)
            sel = np.arange(nv) if idx_sample is None else idx_sample
            spots = sh.sh_spots(amp, ph, g.n_sub, g.sub_pix, g.fft_n, valid[sel])
            flat = sh.sh_spots(amp, np.zeros((n, n)), g.n_sub, g.sub_pix, g.fft_n, valid[sel])
            r_ref = slopes.sh_slopes(flat)
            s_raw = slopes.sh_slopes(spots)
            both = np.concatenate([sel, sel + nv])
            assert np.all(np.abs(rblk[both] - r_ref) <= _sh_bound(flat, g.fft_n)), k
            bound = _sh_bound(spots, g.fft_n) + _sh_bound(flat, g.fft_n)
            assert np.all(np.abs(blk[both] - (s_raw - r_ref)) <= bound), k
        else:
            g = sen.pwfs
            valid = geometry.valid_subaps(amp.astype(np.uint8), g.n_sub)
            nd = 2 * g.n_sub
            det = _read(torch, sp, S, k, sp.MWFS_DETECTOR, (nd, nd))
            det_ref = pyramid.pwfs_image(amp, ph, g.pad, g.n_mod, g.mod_amp, g.n_sub,
                                         g.pup_dist_px)
            assert norm_intensity_error(det, det_ref) <= 1e-5, k
            flat = pyramid.pwfs_image(amp, np.zeros((n, n)), g.pad, g.n_mod, g.mod_amp,
                                      g.n_sub, g.pup_dist_px)
            r_ref = slopes.pyr_slopes(flat, g.n_sub, valid)
            s_ref = slopes.pyr_slopes(det_ref, g.n_sub, valid, ref=r_ref)
            T = det_ref.sum() / nv
            tol = 2 * (5e-5 * det_ref.max() / T + 1e-5 * np.abs(s_ref).max())
            assert np.max(np.abs(blk - s_ref)) <= tol, k
    return got


def test_small_system_vs_oracle(env, small):
    torch, sp, ctx = env
    t = 0.0371
    small.frame(t)
    torch.cuda.synchronize()
    got = _check_system(torch, sp, small, t)
    R = small.R.cpu().numpy().astype(np.float64)
    m_ref = recon.mvm(R, got)
    mag = np.abs(R) @ np.abs(got)
    assert np.all(np.abs(small.modes.cpu().numpy() - m_ref) <= 1e-5 * mag)


def test_oracle_system_slope_layout(env, small):
    offs, tot = system.slope_offsets(small.wl.sensors)
    assert offs == [int(o) for o in small.offsets] and tot == small.n_slopes


def test_persistent_matches_per_sensor_calls(env, small):
    torch, sp, ctx = env
    for t in (0.0, 0.013):
        s1, m1 = small.frame(t)
        s2, m2 = small.frame_separate(t)
        torch.cuda.synchronize()
        a, b = s1.cpu().numpy().astype(np.float64), s2.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(a - b)) <= 1e-5 * (1 + np.abs(b).max())
        for k, e in enumerate(small.sep):
            n = e["phase"].shape[0]
            ph = _read(torch, sp, small, k, sp.MWFS_PHASE, (n, n))
            pe = e["phase"].cpu().numpy().astype(np.float64)
            sen = small.wl.sensors[k]
            cover = _covered(sen, geometry.pupil_mask(n, sen.pupil.obsc_frac))
            assert np.max(np.abs(ph - pe)[cover]) <= 2e-6 * (1 + np.abs(pe).max())
            if e["kind"] == "pwfs":
                nd = e["img"].shape[0]
                det = _read(torch, sp, small, k, sp.MWFS_DETECTOR, (nd, nd))
                assert norm_intensity_error(det, e["img"].cpu().numpy()) <= 1e-6
        R = small.R.cpu().numpy().astype(np.float64)
        mag = np.abs(R) @ np.abs(b)
        assert np.all(np.abs(m1.cpu().numpy() - m2.cpu().numpy()) <= 2e-5 * mag)


def test_grid_size_does_not_change_the_frame(env, small):
    torch, sp, ctx = env
    sched = small.m.schedule()
    assert sched["n_tasks"] > 0 and sched["max_grid"] >= 1
    outs = []
    for g in (0, 1, 7, 64, sched["max_grid"]):
        small.m.set_grid(g)
        small.frame(0.02)
        torch.cuda.synchronize()
        outs.append((small.slopes.clone(), small.modes.clone()))
    small.m.set_grid(0)
    for s, m in outs[1:]:
        assert torch.equal(s, outs[0][0]) and torch.equal(m, outs[0][1])
    assert sp.specula_ctx_status(ctx) == sp.OK


def test_graph_replay_is_one_kernel_and_matches_eager(env, small):
    torch, sp, ctx = env
    st = torch.cuda.Stream()
    g = small.capture(st)
    assert g.kernel_count() == 1
    for t in (0.0, 0.05):
        small.frame(t)
        torch.cuda.synchronize()
        eager = (small.slopes.clone(), small.modes.clone())
        small.slopes.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            small.t_dev.fill_(t)
        g.launch(st)
        torch.cuda.synchronize()
        assert torch.equal(small.slopes, eager[0]) and torch.equal(small.modes, eager[1])
    g.close()
    gs = small.capture(st, separate=True)
    assert gs.kernel_count() > 1
    gs.close()


def test_create_rejects_unsupported_systems(env):
    torch, sp, ctx = env
    wl = synth.workload("mwfs8m_small")
    scr = [torch.zeros(l.side, l.side, device="cuda") for l in wl.layers]
    lay = [sp.layer_desc(l) for l in wl.layers]
    big = synth.workload("pwfs8m").sensors[0]          # FFT side 320: no variant
    with pytest.raises(sp.SpeculaError) as e:
        sp.Mwfs(ctx, [sp.wfs_desc(big)], lay, scr)
    assert e.value.status == sp.EUNSUPPORTED
    d = sp.wfs_desc(wl.sensors[0])
    d.sh.n_sub = 7                                      # 7 x 12 != 96 pixels
    with pytest.raises(sp.SpeculaError) as e:
        sp.Mwfs(ctx, [d], lay, scr)
    assert e.value.status == sp.EINVAL


def test_mwfs39m_full(env):
    """The full 39 m system (6 laser-star SH 68 x 68, 3 pyramids 240^2 x 16
    modulation points, 10 layers, 4000 x 47376 MVM) in one launch against
    the oracle in full: every phase, every SH subaperture's slopes, the
    pyramid detectors and slopes, and every mode."""
    torch, sp, ctx = env
    from paper_2602_06688_gb300.system import System
    S = System(ctx, synth.workload("mwfs39m"), with_separate=False)
    t = 0.0123
    S.frame(t)
    torch.cuda.synchronize()
    assert sp.specula_ctx_status(ctx) == sp.OK
    got = _check_system(torch, sp, S, t)
    R = S.R.cpu().numpy().astype(np.float64)
    m_ref = recon.mvm(R, got)
    mag = np.abs(R) @ np.abs(got)
    assert np.all(np.abs(S.modes.cpu().numpy() - m_ref) <= 1e-5 * mag)
    S.m.close()
