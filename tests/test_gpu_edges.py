"""Edge and degenerate cases on the GPU against the oracle: empty batches,
a static (unmodulated) pyramid, all modulation points at the same place,
the unbinned intensity, an MVM whose slope count is not a multiple of four,
the maximum layer count of the extraction and the sizes just beyond it."""
import ctypes as C
import math
from types import SimpleNamespace as NS

import numpy as np
import pytest

from gpu_common import close_checked, kolmogorov_phase, load_pkg, need_gpu, norm_intensity_error
from oracle import atmo, pyramid, recon

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_empty_batches_are_no_ops(env):
    torch, sp, ctx = env
    lib = sp.lib()
    pu = sp.PupilDesc(32, 0.1, 0.2)
    pw = sp.PwfsDesc(2, 8, 8, 32, 3.0)
    sp.specula_pwfs_plan(ctx, pu, pw)
    amp = torch.ones(32, 32, device="cuda")
    det = torch.full((16, 16), 7.0, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.specula_pwfs_image(ctx.handle, C.byref(pu), C.byref(pw), _ptr(amp), _ptr(amp), 0,
                                  _ptr(det), st) == sp.OK
    idx = torch.arange(4, dtype=torch.int32, device="cuda")
    sc = sp.slopec_desc(sp.SLOPES_PYR, 8, idx)
    out = torch.full((8,), 7.0, device="cuda")
    assert lib.specula_slopes(ctx.handle, C.byref(sc), _ptr(det), None, 0, _ptr(out), st) == sp.OK
    R = torch.zeros(3, 8, device="cuda")
    m = torch.full((3,), 7.0, device="cuda")
    rec = sp.recon_desc(3, 8, sp.PREC_FP32, R)
    assert lib.specula_recon(ctx.handle, C.byref(rec), _ptr(out), 0, _ptr(m), st) == sp.OK
    torch.cuda.synchronize()
    assert bool((det == 7.0).all()) and bool((out == 7.0).all()) and bool((m == 7.0).all())
    assert sp.specula_ctx_status(ctx) == sp.OK


@pytest.mark.parametrize("n_mod,r", [(1, 0.0), (4, 0.0), (2, 1.5)])
def test_degenerate_modulation(env, n_mod, r):
    """One point without modulation (the static pyramid), several points all
    at the centre, and two points (the pair that shares its row filter)."""
    torch, sp, ctx = env
    n, nsub = 64, 16
    pu = sp.PupilDesc(n, 0.1, 0.1)
    pw = sp.PwfsDesc(2, n_mod, nsub, n, r)
    sp.specula_pwfs_plan(ctx, pu, pw)
    amp = torch.empty(n, n, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    ph = kolmogorov_phase(n, 8.0 / n, 0.15, seed=3).astype(np.float32)
    det = torch.empty(2 * nsub, 2 * nsub, device="cuda")
    sp.specula_pwfs_image(ctx, pu, pw, amp, torch.tensor(ph, device="cuda"), det)
    torch.cuda.synchronize()
    ref = pyramid.pwfs_image(amp.cpu().numpy().astype(np.float64), ph.astype(np.float64), 2,
                             n_mod, r, nsub, n)
    assert norm_intensity_error(det.cpu().numpy(), ref) <= 1e-5


def test_unbinned_intensity(env):
    """n_sub = n_pix: the detector is the N x N intensity itself."""
    torch, sp, ctx = env
    n = 32
    pu = sp.PupilDesc(n, 0.1, 0.0)
    pw = sp.PwfsDesc(2, 6, n, n, 2.0)
    sp.specula_pwfs_plan(ctx, pu, pw)
    amp = torch.empty(n, n, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    ph = kolmogorov_phase(n, 0.25, 0.15, seed=4).astype(np.float32)
    det = torch.empty(2 * n, 2 * n, device="cuda")
    sp.specula_pwfs_image(ctx, pu, pw, amp, torch.tensor(ph, device="cuda"), det)
    torch.cuda.synchronize()
    ref = pyramid.pwfs_intensity(amp.cpu().numpy().astype(np.float64), ph.astype(np.float64), 2, 6,
                                 2.0, n)
    assert norm_intensity_error(det.cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("nm,ns,nb", [(33, 101, 2), (1, 3, 1), (7, 4099, 3)])
def test_mvm_ragged_sizes(env, nm, ns, nb):
    torch, sp, ctx = env
    rng = np.random.default_rng(ns)
    R = rng.standard_normal((nm, ns)).astype(np.float32)
    s = rng.standard_normal((nb, ns)).astype(np.float32)
    out = torch.empty(nb, nm, device="cuda")
    sp.specula_recon(ctx, sp.recon_desc(nm, ns, sp.PREC_FP32, torch.tensor(R, device="cuda")),
                     torch.tensor(s, device="cuda"), out)
    torch.cuda.synchronize()
    ref = recon.mvm(R.astype(np.float64), s.astype(np.float64))
    mag = np.abs(s.astype(np.float64)) @ np.abs(R.astype(np.float64)).T
    assert np.all(np.abs(out.cpu().numpy() - ref) <= 1e-5 * mag + 1e-12)


def test_extraction_at_the_layer_limit(env):
    """64 layers (the most the coordinate tables hold) against the oracle;
    65 layers and a pupil of 8193 px are refused."""
    torch, sp, ctx = env
    rng = np.random.default_rng(11)
    Ls = [NS(side=64, pitch_m=0.1, height_m=float(h), vx_mps=float(rng.uniform(-9, 9)),
             vy_mps=float(rng.uniform(-9, 9))) for h in np.linspace(0, 15e3, 64)]
    src = NS(theta_x_rad=1e-5, theta_y_rad=0.0, height_m=math.inf, wavelength_nm=600.0)
    scr = [rng.standard_normal((64, 64)).astype(np.float32) for _ in Ls]
    scr_t = [torch.tensor(x, device="cuda") for x in scr]
    n = 40
    out = torch.empty(n, n, device="cuda")
    lay = [sp.layer_desc(L) for L in Ls]
    sp.specula_atmo_extract(ctx, lay, scr_t, sp.source_desc(src), sp.PupilDesc(n, 0.07, 0.0), 0.3,
                            out)
    torch.cuda.synchronize()
    ref = atmo.atmo_extract([x.astype(np.float64) for x in scr], Ls, src, n, 0.07, 0.3)
    tol = (500.0 / 600.0) * sum(np.abs(x).max() for x in scr) * 4 * 2.0 ** -24
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= tol
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_atmo_extract(ctx, lay + lay[:1], scr_t + scr_t[:1], sp.source_desc(src),
                                sp.PupilDesc(n, 0.07, 0.0), 0.3, out)
    assert e.value.status == sp.EUNSUPPORTED
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_atmo_extract(ctx, lay[:1], scr_t[:1], sp.source_desc(src),
                                sp.PupilDesc(8193, 0.07, 0.0), 0.3,
                                torch.empty(8193 * 8193, device="cuda"))
    assert e.value.status == sp.EUNSUPPORTED


def test_guard_bands_cover_the_workspaces(env):
    """Plans at padding 3 and 4 (the sizes an undersized per-point buffer
    once overran) leave every workspace guard band intact."""
    torch, sp, ctx = env
    for pad, n, nsub, dist in ((3, 80, 16, 40), (4, 32, 8, 16)):
        pu = sp.PupilDesc(n, 0.1, 0.1)
        pw = sp.PwfsDesc(pad, 6, nsub, dist, 2.0)
        sp.specula_pwfs_plan(ctx, pu, pw)
        amp = torch.empty(n, n, device="cuda")
        sp.specula_pupil_mask(ctx, pu, amp)
        det = torch.empty(pad * nsub, pad * nsub, device="cuda")
        sp.specula_pwfs_image(ctx, pu, pw, amp, torch.zeros(n, n, device="cuda"), det)
    n_checked, n_bad = sp.specula_check_guards(ctx)
    assert n_checked >= 8 and n_bad == 0


@pytest.mark.parametrize("bits,rtol", [(32, 1e-6), (64, 1e-14)])
def test_fma_probe_computes_its_chains(env, bits, rtol):
    """The peak probe's output is the sum of its 8 chains a = a x + y started
    at (thread + i): the work it claims is done, not optimised away."""
    torch, sp, ctx = env
    dt = torch.float32 if bits == 32 else torch.float64
    sink = torch.full((3 * 256,), float("nan"), dtype=dt, device="cuda")
    sp.specula_fma_probe(ctx, bits, 3, 7, sink)
    torch.cuda.synchronize()
    x = float(np.float32(1.0000001)) if bits == 32 else 1.0000001
    y = float(np.float32(-1e-7)) if bits == 32 else -1e-7
    ref = np.zeros(256)
    for i in range(8):
        a = np.arange(256, dtype=np.float64) + i
        for _ in range(7):
            a = a * x + y
        ref += a
    got = sink.cpu().numpy().astype(np.float64).reshape(3, 256)
    assert np.allclose(got, ref[None, :], rtol=rtol, atol=0)
