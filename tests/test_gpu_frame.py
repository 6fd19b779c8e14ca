"""GPU parity of a whole frame (extraction -> pyramid -> slopes -> MVM) against
the oracle chain, and graph replay against eager launches."""
import numpy as np
import pytest

import synth
from gpu_common import close_checked, load_pkg, need_gpu, norm_intensity_error
from oracle import atmo, geometry, pyramid, recon, slopes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


@pytest.mark.parametrize("name", ["pwfs8m_tiny", "pwfs8m"])
def test_frame_vs_oracle_chain(env, name):
    torch, sp, ctx = env
    from paper_2602_06688_gb300.frame import PwfsFrame
    wl = synth.workload(name)
    fr = PwfsFrame(ctx, wl)
    s = wl.sensors[0]
    n, nsub = s.pupil.n_pix, s.pwfs.n_sub
    t = 0.123
    fr.frame(t)
    torch.cuda.synchronize()
    # oracle on the GPU's screens (float32 values; generator parity is tested
    # separately) and the same stand-in reconstructor
    scr = [x.cpu().numpy().astype(np.float64) for x in fr.screens]
    phi = atmo.atmo_extract(scr, wl.layers, s.source, n, s.pupil.pitch_m, t)
    ph_gpu = fr.phase.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(ph_gpu - phi)) <= 1e-5 * (1 + np.abs(phi).max())
    amp = geometry.pupil_mask(n, s.pupil.obsc_frac).astype(np.float64)
    valid = geometry.valid_subaps(amp.astype(np.uint8), nsub)
    g = s.pwfs
    det_ref = pyramid.pwfs_image(amp, phi, g.pad, g.n_mod, g.mod_amp, nsub, n)
    flat = pyramid.pwfs_image(amp, np.zeros_like(phi), g.pad, g.n_mod, g.mod_amp, nsub, n)
    det = fr.det.cpu().numpy().astype(np.float64)
    assert norm_intensity_error(det, det_ref) <= 1e-5
    s_ref = slopes.pyr_slopes(det_ref, nsub, valid, ref=slopes.pyr_slopes(flat, nsub, valid))
    T = det_ref.sum() / len(valid)
    tol = 2 * (5e-5 * det_ref.max() / T + 1e-5 * np.abs(s_ref).max())
    sl = fr.slopes.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(sl - s_ref)) <= tol
    R = fr.R.cpu().numpy().astype(np.float64)
    m_ref = recon.mvm(R, sl)
    mag = np.abs(R) @ np.abs(sl)
    assert np.all(np.abs(fr.modes.cpu().numpy() - m_ref) <= 1e-5 * mag)


def test_graph_replay_matches_eager(env):
    torch, sp, ctx = env
    from paper_2602_06688_gb300.frame import PwfsFrame
    fr = PwfsFrame(ctx, synth.workload("pwfs8m_tiny"))
    st = torch.cuda.Stream()
    g = fr.capture(st)
    assert g.kernel_count() >= 6
    for t in (0.0, 0.017, 0.5):
        fr.frame(t)
        torch.cuda.synchronize()
        eager = fr.modes.clone()
        fr.modes.zero_()
        torch.cuda.synchronize()
        fr.replay(t, st)
        torch.cuda.synchronize()
        assert torch.equal(fr.modes, eager)
    g.close()


def test_batched_frames_match_single_frames(env):
    """A batch of B consecutive frames (one pyramid, slope and MVM call over
    the batch) gives the same modes as B single frames at those times."""
    torch, sp, ctx = env
    from paper_2602_06688_gb300.frame import PwfsFrame
    wl = synth.workload("pwfs8m_tiny")
    one = PwfsFrame(ctx, wl)
    four = PwfsFrame(ctx, wl, batch=4)
    four.frame(0.2)
    torch.cuda.synchronize()
    got = four.modes.clone()
    for k in range(4):
        one.frame(0.2 + k * wl.dt_s)
        torch.cuda.synchronize()
        ref = one.modes.cpu().numpy().astype(np.float64)
        R = one.R.cpu().numpy().astype(np.float64)
        mag = np.abs(R) @ np.abs(one.slopes.cpu().numpy().astype(np.float64))
        assert np.all(np.abs(got[k].cpu().numpy() - ref) <= 2e-5 * mag + 1e-7), k
    st = torch.cuda.Stream()
    g = four.capture(st)
    four.replay(0.2, st)
    torch.cuda.synchronize()
    assert torch.equal(four.modes, got)
    g.close()


def test_elt_frame_in_the_bench_configuration(env):
    """The full-size ELT frame (pwfs39m: 35 layers, 960^2 FFT, 48 points,
    4000 x 13344 MVM) as the bench times it: autotuned tiles, replayed from a
    CUDA graph on a side stream, against the oracle chain on the same screens
    (every detector pixel, every slope and mode)."""
    torch, sp, ctx = env
    from paper_2602_06688_gb300.frame import PwfsFrame
    wl = synth.workload("pwfs39m")
    fr = PwfsFrame(ctx, wl, autotune=True)
    st = torch.cuda.Stream()
    fr.capture(st)
    t = 0.0371
    fr.replay(t, st)
    torch.cuda.synchronize()
    s = wl.sensors[0]
    n, nsub, g = s.pupil.n_pix, s.pwfs.n_sub, s.pwfs
    scr = [x.cpu().numpy().astype(np.float64) for x in fr.screens]
    phi = atmo.atmo_extract(scr, wl.layers, s.source, n, s.pupil.pitch_m, t)
    assert np.max(np.abs(fr.phase.cpu().numpy() - phi)) <= 1e-5 * (1 + np.abs(phi).max())
    amp = geometry.pupil_mask(n, s.pupil.obsc_frac).astype(np.float64)
    valid = geometry.valid_subaps(amp.astype(np.uint8), nsub)
    det_ref = pyramid.pwfs_image(amp, phi, g.pad, g.n_mod, g.mod_amp, nsub, n)
    det = fr.det.cpu().numpy().astype(np.float64)
    assert norm_intensity_error(det, det_ref) <= 1e-5
    flat = pyramid.pwfs_image(amp, np.zeros_like(phi), g.pad, g.n_mod, g.mod_amp, nsub, n)
    s_ref = slopes.pyr_slopes(det_ref, nsub, valid, ref=slopes.pyr_slopes(flat, nsub, valid))
    T = det_ref.sum() / len(valid)
    tol = 2 * (5e-5 * det_ref.max() / T + 1e-5 * np.abs(s_ref).max())
    sl = fr.slopes.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(sl - s_ref)) <= tol
    R = fr.R.cpu().numpy().astype(np.float64)
    mag = np.abs(R) @ np.abs(sl)
    assert np.all(np.abs(fr.modes.cpu().numpy() - recon.mvm(R, sl)) <= 1e-5 * mag)
    fr.graph.close()


@pytest.mark.parametrize("correction", [False, True])
def test_learned_reconstructor_in_the_frame(env, correction):
    """The frame with a network in place of the MVM, or as a correction on
    top of it (m = R s + f(s)): its modes equal the network (plus the MVM)
    applied to the frame's own slopes by separate library calls, bit for bit,
    eager and replayed from the frame's graph."""
    torch, sp, ctx = env
    from paper_2602_06688_gb300.frame import PwfsFrame
    fr = PwfsFrame(ctx, synth.workload("pwfs8m_tiny"))
    sizes = (fr.n_slopes, 128, 128, fr.n_modes)
    mlp = sp.MLP(ctx, sizes, 8)
    for l in range(3):
        bnd = 1.0 / np.sqrt(sizes[l])
        mlp.set_layer(l, synth.uniform_draws(40 + 2 * l, (sizes[l + 1], sizes[l]), -bnd, bnd),
                      synth.uniform_draws(41 + 2 * l, (sizes[l + 1],), -bnd, bnd))
    fr.use_learned(mlp, correction=correction)
    st = torch.cuda.Stream()
    fr.capture(st)
    for t in (0.0, 0.023):
        fr.frame(t)
        torch.cuda.synchronize()
        eager = fr.modes.clone()
        f = torch.empty(1, fr.n_modes, device="cuda")
        mlp.infer(fr.slopes.view(1, -1), f)
        ref = f.view(-1).clone()
        if correction:
            lin = torch.empty(fr.n_modes, device="cuda")
            sp.specula_recon(ctx, fr.rec, fr.slopes, lin)
            torch.cuda.synchronize()
            ref = lin + f.view(-1)
        torch.cuda.synchronize()
        assert torch.equal(eager.view(-1), ref)
        fr.modes.zero_()
        fr.replay(t, st)
        torch.cuda.synchronize()
        assert torch.equal(fr.modes, eager)
    fr.use_learned(None)
    mlp.close()
