"""Failure detection on the GPU without a fault: a dependency wait of the
persistent multi-sensor launch that runs out (a task made to wait for an
arrival count that never comes, under a short limit) ends the launch with
SPECULA_ETIMEOUT and leaves the context usable; the non-finite guard of the
slope computers reports a NaN injected into the phase on the host."""
import time

import numpy as np
import pytest

import synth
from gpu_common import close_checked, load_pkg, need_gpu
from oracle import geometry

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
    return System(ctx, synth.workload("mwfs8m_small"), with_separate=False)


def test_stalled_task_times_out_and_the_next_frame_is_clean(env, small):
    torch, sp, ctx = env
    small.frame(0.02)
    torch.cuda.synchronize()
    assert sp.specula_ctx_status(ctx) == sp.OK
    want = (small.slopes.clone(), small.modes.clone())
    n = small.m.schedule()["n_tasks"]
    for task in (0, n // 2, n - 1):
        small.m.set_wait(2_000_000, task)            # 2 ms
        t0 = time.perf_counter()
        small.frame(0.02)
        st = sp.specula_ctx_status(ctx)              # synchronises
        assert st == sp.ETIMEOUT, (task, st)
        assert time.perf_counter() - t0 < 1.0
        small.m.set_wait(0, -1)
        small.frame(0.02)
        torch.cuda.synchronize()
        assert sp.specula_ctx_status(ctx) == sp.OK
        assert torch.equal(small.slopes, want[0]) and torch.equal(small.modes, want[1])


def test_set_wait_rejects_bad_arguments(env, small):
    torch, sp, ctx = env
    n = small.m.schedule()["n_tasks"]
    for args in ((-1, -1), (10_000_000_001, -1), (0, n), (0, -2)):
        with pytest.raises(sp.SpeculaError) as e:
            small.m.set_wait(*args)
        assert e.value.status == sp.EINVAL


def test_guard_reports_nan_in_a_screen(env, small):
    torch, sp, ctx = env
    scr = small.screens[0]
    keep = scr.clone()
    scr.fill_(float("nan"))                     # every sensor sees it
    small.frame(0.01)
    assert sp.specula_ctx_status(ctx) == sp.ENONFINITE
    sp.specula_ctx_set_guard(ctx, 0)
    small.frame(0.01)
    assert sp.specula_ctx_status(ctx) == sp.OK
    assert torch.isnan(small.slopes).any()
    sp.specula_ctx_set_guard(ctx, 1)
    scr.copy_(keep)
    small.frame(0.01)
    assert sp.specula_ctx_status(ctx) == sp.OK
    assert torch.isfinite(small.slopes).all()


def _pyr(torch, sp, ctx, phase):
    n_pix, n_sub = 32, 8
    pu = sp.PupilDesc(n_pix, 0.1, 0.2)
    pw = sp.PwfsDesc(2, 8, n_sub, n_pix, 3.0)
    sp.specula_pwfs_plan(ctx, pu, pw)
    amp = torch.empty(n_pix, n_pix, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    det = torch.empty(1, 2 * n_sub, 2 * n_sub, device="cuda")
    sp.specula_pwfs_image(ctx, pu, pw, amp, torch.tensor(phase[None], device="cuda"), det)
    valid = geometry.valid_subaps(amp.cpu().numpy().astype(np.uint8), n_sub)
    idx = torch.tensor(valid, device="cuda")
    s = torch.empty(1, 2 * len(valid), device="cuda")
    sp.specula_slopes(ctx, sp.slopec_desc(sp.SLOPES_PYR, n_sub, idx), det, None, s)
    return s


def _sh(torch, sp, ctx, phase):
    n_sub, sub_pix, fft_n = 8, 8, 16
    n_pix = n_sub * sub_pix
    pu = sp.PupilDesc(n_pix, 0.1, 0.2)
    shd = sp.ShDesc(n_sub, sub_pix, fft_n)
    nv = sp.specula_sh_plan(ctx, pu, shd)
    amp = torch.empty(n_pix, n_pix, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    spots = torch.empty(1, nv, fft_n, fft_n, device="cuda")
    sp.specula_sh_image(ctx, pu, shd, amp, torch.tensor(phase[None], device="cuda"), spots, nv)
    valid = geometry.valid_subaps(amp.cpu().numpy().astype(np.uint8), n_sub)
    s = torch.empty(1, 2 * nv, device="cuda")
    sp.specula_slopes(ctx, sp.slopec_desc(sp.SLOPES_SH, n_sub, torch.tensor(valid, device="cuda"),
                                          fft_n), spots, None, s)
    return s


@pytest.mark.parametrize("kind", ["pyr", "sh"])
def test_guard_reports_nan_in_the_phase(env, kind):
    torch, sp, ctx = env
    run = _pyr if kind == "pyr" else _sh
    n_pix = 32 if kind == "pyr" else 64
    rng = np.random.default_rng(3)
    phase = rng.standard_normal((n_pix, n_pix)).astype(np.float32)
    s = run(torch, sp, ctx, phase)
    assert sp.specula_ctx_status(ctx) == sp.OK and torch.isfinite(s).all()
    phase[n_pix // 4, n_pix // 2] = np.nan        # one pixel inside the pupil
    s = run(torch, sp, ctx, phase)
    assert sp.specula_ctx_status(ctx) == sp.ENONFINITE
    assert not torch.isfinite(s).all()
    sp.specula_ctx_set_guard(ctx, 0)
    run(torch, sp, ctx, phase)
    assert sp.specula_ctx_status(ctx) == sp.OK
    sp.specula_ctx_set_guard(ctx, 1)
    with pytest.raises(sp.SpeculaError):
        sp.specula_ctx_set_guard(ctx, 2)
