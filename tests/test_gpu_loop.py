"""GPU parity of the closed loop (modal mirror, residual statistics,
integrator) against the FP64 oracle loop, on the 8 m single-layer pyramid
system with a calibrated 60-mode reconstructor.

Tolerances: the mirror shape is a float32 sum of n_modes products
(|error| <= n_modes eps_32 sum_j |c_j B_j|); per step the pyramid image
carries ~1e-5 of normalised-intensity error, so the slopes and modes carry
~1e-5 relative error, which the integrator (gain g, leak) keeps bounded
at the same order over the run; the checks use 2e-4 of the largest command
and of the open-loop residual RMS, and 2e-4 absolute on the Strehl ratio."""
import numpy as np
import pytest

import synth
from gpu_common import close_checked, load_pkg, need_gpu
from oracle import loop as oloop

pytestmark = pytest.mark.gpu

STEPS = 12


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


@pytest.fixture(scope="module")
def cl(env):
    torch, sp, ctx = env
    from paper_2602_06688_gb300.loop import ClosedLoop
    lp = ClosedLoop(ctx, synth.workload("pwfs8m_tiny"), n_modes=60, gain=0.4)
    yield lp
    lp.close()


def _np(t):
    return t.cpu().numpy().astype(np.float64)


def test_mirror_residual_and_update_parity(env, cl):
    torch, sp, ctx = env
    rng = np.random.default_rng(4)
    cmd = torch.tensor(rng.standard_normal(cl.n_modes).astype(np.float32), device="cuda")
    dm = torch.empty_like(cl.dm)
    sp.specula_dm_shape(ctx, cl.basis, cmd, dm)
    torch.cuda.synchronize()
    B, c = _np(cl.basis), _np(cmd)
    ref = oloop.dm_shape(B, c)
    bound = cl.n_modes * 2.0 ** -23 * np.tensordot(np.abs(c), np.abs(B), axes=1) + 1e-12
    assert np.all(np.abs(_np(dm) - ref) <= bound)
    atm = torch.tensor((rng.standard_normal(dm.shape) * 2).astype(np.float32), device="cuda")
    resid = torch.empty_like(dm)
    stats = torch.empty(2, dtype=torch.float64, device="cuda")
    sp.specula_loop_residual(ctx, cl.fr.amp, atm, dm, 0.45, resid, stats)
    torch.cuda.synchronize()
    r32 = atm.cpu().numpy() - dm.cpu().numpy()                 # the same float32 subtraction
    assert np.array_equal(resid.cpu().numpy(), r32)
    rms, sr = oloop.residual_stats(_np(cl.fr.amp), r32.astype(np.float64), 0.45)
    got = stats.cpu().numpy()
    assert abs(got[0] - rms) <= 1e-6 * rms and abs(got[1] - sr) <= 1e-6
    m = torch.tensor(rng.standard_normal(cl.n_modes).astype(np.float32), device="cuda")
    c0 = cmd.clone()
    sp.specula_loop_integrate(ctx, 0.3, 0.1, m, cmd)
    torch.cuda.synchronize()
    ref = 0.9 * _np(c0) + 0.3 * _np(m)
    assert np.max(np.abs(_np(cmd) - ref)) <= 4 * 2.0 ** -24 * (np.abs(ref).max() + 1)
    with pytest.raises(sp.SpeculaError):
        sp.specula_loop_integrate(ctx, 0.3, 1.5, m, cmd)


def test_closed_loop_matches_the_oracle(env, cl):
    torch, sp, ctx = env
    fr, wl = cl.fr, synth.workload("pwfs8m_tiny")
    times = [k * fr.dt for k in range(STEPS)]
    cl.reset()
    st_g, cm_g = [], []
    for t in times:
        cl.step(t)
        torch.cuda.synchronize()
        st_g.append(cl.stats.cpu().numpy().copy())
        cm_g.append(_np(cl.cmd))
    st_g, cm_g = np.array(st_g), np.array(cm_g)
    s = wl.sensors[0]
    amp = _np(fr.amp)
    phases = oloop.atmosphere([_np(x) for x in fr.screens], wl.layers, s.source, s.pupil.n_pix,
                              s.pupil.pitch_m, times)
    sensor = oloop.pyramid_sensor(amp, s.pwfs.pad, s.pwfs.n_mod, s.pwfs.mod_amp, s.pwfs.n_sub,
                                  s.pwfs.pup_dist_px, fr.valid.cpu().numpy(), _np(cl.R))
    st_o, cm_o, _ = oloop.run_loop(phases, amp, _np(cl.basis), sensor, cl.gain, cl.leak,
                                   cl.wfs_over_sci)
    cmax = np.abs(cm_o).max()
    assert np.max(np.abs(cm_g - cm_o)) <= 2e-4 * cmax
    assert np.max(np.abs(st_g[:, 0] - st_o[:, 0])) <= 2e-4 * st_o[0, 0]
    assert np.max(np.abs(st_g[:, 1] - st_o[:, 1])) <= 2e-4
    # the loop corrects: the residual falls well below the open-loop phase
    assert st_o[-1, 0] < 0.5 * st_o[0, 0] and st_g[-1, 0] < 0.5 * st_g[0, 0]
    assert st_g[-1, 1] > st_g[0, 1]


def test_loop_graph_replay_is_bit_identical(env, cl):
    torch, sp, ctx = env
    st = torch.cuda.Stream()
    g = cl.capture(st)
    assert g.kernel_count() > 5
    cl.reset()
    for k in range(6):
        cl.step(k * cl.fr.dt)
    torch.cuda.synchronize()
    eager = (cl.cmd.clone(), cl.stats.clone())
    cl.reset()
    torch.cuda.synchronize()
    for k in range(6):
        cl.replay(k * cl.fr.dt, st)
    torch.cuda.synchronize()
    assert torch.equal(cl.cmd, eager[0]) and torch.equal(cl.stats, eager[1])
    cl.close()


def test_closed_loop_on_the_soul_geometry(env):
    """The loop on the SOUL example's geometry (pad 3, separated images, map
    slopes, calibrated with map slopes): the residual falls and the Strehl
    ratio rises over 40 steps."""
    torch, sp, ctx = env
    from paper_2602_06688_gb300.loop import ClosedLoop
    lp = ClosedLoop(ctx, synth.workload("soul8m"), n_modes=150, gain=0.4)
    assert lp.rank == 150
    sr = []
    for k in range(40):
        lp.step(k * lp.fr.dt)
        torch.cuda.synchronize()
        sr.append(lp.stats.cpu().numpy().copy())
    sr = np.array(sr)
    assert sr[-1, 1] > 5 * sr[0, 1] and sr[-5:, 0].mean() < 0.5 * sr[0, 0]
    lp.close()


@pytest.mark.parametrize("residual", [True, False])
def test_learned_reconstructor_in_the_loop(env, residual):
    """The network in the loop (R s + f(s), or f(s) alone), trained on the
    loop's own residual spectrum, runs from the captured graph: the graph
    replay equals eager steps bit for bit, the commands stay bounded, and the
    correction keeps the linear loop's Strehl ratio (within 5%)."""
    torch, sp, ctx = env
    from paper_2602_06688_gb300.loop import ClosedLoop, LoopNetwork
    lp = ClosedLoop(ctx, synth.workload("pwfs8m_tiny"), n_modes=60, gain=0.4)
    steps, settle = 120, 60

    def run(graph):
        lp.reset()
        s = []
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            for k in range(steps):
                if graph:
                    lp.replay(k * lp.fr.dt, st)
                else:
                    lp.step(k * lp.fr.dt, stream=st)
                s.append(lp.stats.clone())
        torch.cuda.synchronize()
        return torch.stack(s).cpu().numpy(), lp.cmd.clone()

    lin, _ = run(False)
    net = LoopNetwork(lp, hidden=(256, 256), residual=residual)
    info = net.train(n_pairs=8192, epochs=10)
    assert np.isfinite(info["final_loss"])
    lp.net = net
    eager, c_eager = run(False)
    lp.capture(torch.cuda.Stream())
    graph, c_graph = run(True)
    lp.net = None
    lp.close()
    assert np.array_equal(eager, graph) and torch.equal(c_eager, c_graph)
    assert float(c_eager.abs().max()) < 50.0
    s_lin, s_net = lin[settle:, 1].mean(), eager[settle:, 1].mean()
    if residual:
        assert s_net >= 0.95 * s_lin, (s_net, s_lin)
    else:
        assert s_net > 0.5 * s_lin, (s_net, s_lin)
