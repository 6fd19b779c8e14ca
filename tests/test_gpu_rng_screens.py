"""GPU parity: Philox normals, batched device-noise screens, random phases."""
import math

import numpy as np
import pytest

from gpu_common import close_checked, load_pkg, need_gpu
from oracle import philox, screens

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


def test_rng_matches_oracle(env):
    torch, sp, ctx = env
    seed, s0, ns, n = (1 << 40) + 12345, 7, 3, 1001
    out = torch.empty(ns, n, dtype=torch.complex128, device="cuda")
    sp.specula_rng_complex(ctx, seed, s0, ns, 1, n, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for b in range(ns):
        ref = philox.complex_noise(seed, s0 + b, 1, n)
        # identical uniforms; log/cos/sin of two libraries differ in the last bits
        assert np.max(np.abs(got[b] - ref)) <= 1e-13


@pytest.mark.parametrize("M,delta,r0,L0", [(64, 0.25, 0.2, 30.0), (256, 0.0525, 1.0, 40.0)])
def test_screen_batch_matches_oracle(env, M, delta, r0, L0):
    torch, sp, ctx = env
    seed, s0, ns = 99, 11, 3
    out = torch.empty(ns, M, M, device="cuda")
    sp.specula_screen_generate_batch(ctx, ns, M, delta, r0, L0, seed, s0, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    for b in range(ns):
        cn = philox.complex_noise(seed, s0 + b, 0, M * M).reshape(M, M)
        cs = philox.complex_noise(seed, s0 + b, 1, 27).reshape(3, 3, 3)
        ref = screens.fft_screen(M, delta, r0, L0, cn, cs)
        assert np.max(np.abs(got[b] - ref)) <= 2.0 ** -23 * np.max(np.abs(ref)) * 1.01


def test_random_phase_crop_and_scale(env):
    torch, sp, ctx = env
    ns, side, n = 4, 64, 40
    scr = torch.randn(ns, side, side, device="cuda")
    scale = torch.tensor([1.0, 0.5, 2.0, -3.0], device="cuda")
    ph = torch.empty(ns, n, n, device="cuda")
    sp.specula_random_phase(ctx, scr, ns, side, n, scale, ph)
    torch.cuda.synchronize()
    o = (side - n) // 2
    ref = scr[:, o:o + n, o:o + n] * scale[:, None, None]
    assert torch.equal(ph, ref)
    assert math.isfinite(float(ph.abs().max()))
