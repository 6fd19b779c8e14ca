"""GPU parity: integer geometry (bit-exact), phase screens and layer extraction."""
import math
from types import SimpleNamespace as NS

import numpy as np
import pytest

import synth
from gpu_common import close_checked, load_pkg, need_gpu
from oracle import atmo, geometry, screens

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


@pytest.mark.parametrize("n,eps,nsub", [(64, 0.0, 16), (160, 0.11, 40), (480, 0.28, 96),
                                        (816, 0.28, 68), (120, 0.28, 40), (8, 0.5, 4)])
def test_device_geometry_bit_exact(env, n, eps, nsub):
    torch, sp, ctx = env
    pu = sp.PupilDesc(n, 0.1, eps)
    amp = torch.empty(n, n, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    idx = torch.full((nsub * nsub,), -1, dtype=torch.int32, device="cuda")
    nv = torch.zeros(1, dtype=torch.int32, device="cuda")
    sp.specula_valid_subaps(ctx, pu, nsub, idx, nv)
    torch.cuda.synchronize()
    ref = geometry.pupil_mask(n, eps)
    assert np.array_equal(amp.cpu().numpy(), ref.astype(np.float32))
    rv = geometry.valid_subaps(ref, nsub)
    assert int(nv.item()) == len(rv)
    assert np.array_equal(idx.cpu().numpy()[:len(rv)], rv)


@pytest.mark.parametrize("M,delta,r0,L0,seed", [(256, 0.125, 0.15, math.inf, 1000),
                                                (1024, 0.0525, 0.163, 40.0, 2000),
                                                (64, 0.5, 0.1, 25.0, 7)])
def test_screen_generate_parity(env, M, delta, r0, L0, seed):
    torch, sp, ctx = env
    cn = synth.screen_noise(seed, M)
    cs = synth.subharmonic_noise(seed)
    ref = screens.fft_screen(M, delta, r0, L0, cn, cs)
    out = torch.empty(M, M, device="cuda")
    sp.specula_screen_generate(ctx, M, delta, r0, L0, torch.tensor(cn, device="cuda"), cs, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    # both sides float64; the GPU rounds once to float32
    assert np.max(np.abs(got - ref)) <= 2.0 ** -23 * np.max(np.abs(ref))


def _layers_case(kind):
    rng = np.random.default_rng(3)
    if kind == "tiny":
        Ls = [NS(side=256, pitch_m=0.125, height_m=0.0, vx_mps=10.0, vy_mps=0.0)]
        src = NS(theta_x_rad=0.0, theta_y_rad=0.0, height_m=math.inf, wavelength_nm=750.0)
        return Ls, src, 64, 0.125
    if kind == "ngs3":
        Ls = [NS(side=512, pitch_m=0.0525, height_m=h, vx_mps=float(v * math.cos(a)),
                 vy_mps=float(v * math.sin(a)))
              for h, v, a in zip([0.0, 5e3, 10e3], [5.0, 12.5, 20.0], rng.uniform(0, 6.28, 3))]
        src = NS(theta_x_rad=2e-5, theta_y_rad=-1e-5, height_m=math.inf, wavelength_nm=750.0)
        return Ls, src, 160, 0.0525
    if kind == "mixed":
        # screens coarser than the pupil (window path) and finer than it (window too
        # large: gathered from global memory) in one call; 100 px: ragged tiles
        Ls = [NS(side=s_, pitch_m=p_, height_m=h, vx_mps=float(rng.uniform(-20, 20)),
                 vy_mps=float(rng.uniform(-20, 20)))
              for s_, p_, h in [(256, 0.1, 0.0), (1024, 0.02, 2e3), (512, 0.05, 4e3),
                                (1024, 0.0125, 8e3)]]
        src = NS(theta_x_rad=1e-5, theta_y_rad=2e-5, height_m=math.inf, wavelength_nm=750.0)
        return Ls, src, 100, 0.05
    # laser star, cone effect, off axis, ten layers, screens coarser than the pupil
    Ls = [NS(side=256, pitch_m=0.1, height_m=float(h), vx_mps=float(rng.uniform(-20, 20)),
             vy_mps=float(rng.uniform(-20, 20))) for h in np.linspace(0, 20e3, 10)]
    src = NS(theta_x_rad=45 * synth.ARCSEC * 0.5, theta_y_rad=45 * synth.ARCSEC * 0.866,
             height_m=90e3, wavelength_nm=589.0)
    return Ls, src, 200, 0.0478


@pytest.mark.parametrize("kind", ["tiny", "ngs3", "lgs10", "mixed"])
def test_atmo_extract_parity(env, kind):
    torch, sp, ctx = env
    Ls, src, n, pitch = _layers_case(kind)
    rng = np.random.default_rng(9)
    scr = [rng.standard_normal((L.side, L.side)).astype(np.float32) * 3.0 for L in Ls]
    scr_t = [torch.tensor(s, device="cuda") for s in scr]
    out = torch.empty(n, n, device="cuda")
    for t in [0.0, 0.037, 0.999, 7.3]:
        sp.specula_atmo_extract(ctx, [sp.layer_desc(L) for L in Ls], scr_t, sp.source_desc(src),
                                sp.PupilDesc(n, pitch, 0.0), t, out)
        torch.cuda.synchronize()
        ref = atmo.atmo_extract([s.astype(np.float64) for s in scr], Ls, src, n, pitch, t)
        # float32 interpolation: a few ulp of the largest screen value per layer
        tol = (500.0 / src.wavelength_nm) * sum(np.abs(s).max() for s in scr) * 4 * 2.0 ** -24
        assert np.max(np.abs(out.cpu().numpy() - ref)) <= tol


def test_atmo_integer_positions_are_exact_samples(env):
    """With the sample positions on screen pixels the extraction returns the
    screen values bit for bit: pins the float64 floor decisions."""
    torch, sp, ctx = env
    M, n, pitch = 64, 16, 0.5
    S = np.random.default_rng(4).standard_normal((M, M)).astype(np.float32)
    for k in range(3):
        L = NS(side=M, pitch_m=pitch, height_m=0.0, vx_mps=-(0.5 + k) * pitch,
               vy_mps=-(0.5 + 40) * pitch)
        src = NS(theta_x_rad=0.0, theta_y_rad=0.0, height_m=math.inf, wavelength_nm=500.0)
        out = torch.empty(n, n, device="cuda")
        sp.specula_atmo_extract(ctx, [sp.layer_desc(L)], [torch.tensor(S, device="cuda")],
                                sp.source_desc(src), sp.PupilDesc(n, pitch, 0.0), 1.0, out)
        torch.cuda.synchronize()
        rows = (np.arange(n) + 25 + 40) % M
        cols = np.arange(n) + 25 + k
        assert np.array_equal(out.cpu().numpy(), S[rows][:, cols])


def test_atmo_device_time(env):
    torch, sp, ctx = env
    Ls, src, n, pitch = _layers_case("tiny")
    scr = [torch.randn(256, 256, device="cuda")]
    a = torch.empty(n, n, device="cuda")
    b = torch.empty(n, n, device="cuda")
    td = torch.tensor([0.0123], dtype=torch.float64, device="cuda")
    sp.specula_atmo_extract(ctx, [sp.layer_desc(L) for L in Ls], scr, sp.source_desc(src),
                            sp.PupilDesc(n, pitch, 0.0), 0.0123, a)
    sp.specula_atmo_extract(ctx, [sp.layer_desc(L) for L in Ls], scr, sp.source_desc(src),
                            sp.PupilDesc(n, pitch, 0.0), -1.0, b, t_dev=td)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
