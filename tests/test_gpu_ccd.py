"""GPU parity of the detector noise against the FP64 oracle: photon counts
bit-exact (both sides decide them in float64 from the same Philox words),
the readout-noise sum within one float32 rounding."""
import numpy as np
import pytest

from gpu_common import load_pkg, need_gpu
from oracle import ccd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    ctx.close()


def _det(torch, n):
    """A detector-like image: smooth, positive, spanning both samplers."""
    y, x = np.mgrid[:n, :n]
    d = (1.0 + np.cos(0.3 * x) * np.sin(0.21 * y)) ** 2 * 0.5 + 0.01
    d[n // 3, :] = 0.0                                       # dark pixels
    return torch.tensor(d.astype(np.float32), device="cuda")


@pytest.mark.parametrize("scale", [3.0, 60.0, 400.0])
def test_photon_counts_bit_exact(env, scale):
    torch, sp, ctx = env
    det = _det(torch, 33)                                    # 1089 px: ragged last block
    out = torch.empty_like(det)
    sp.specula_ccd(ctx, det, scale, 0.0, 0x1234_5678_9ABC, 17, out)
    torch.cuda.synchronize()
    ref = ccd.ccd_read(det.cpu().numpy(), scale, 0.0, 0x1234_5678_9ABC, 17)
    got = out.cpu().numpy()
    assert np.array_equal(got, ref)
    lam = det.cpu().numpy().astype(np.float64) * scale
    if scale == 60.0:                                        # both samplers in one image
        assert (lam <= ccd.LAMBDA_SWITCH).any() and (lam > ccd.LAMBDA_SWITCH).any()


def test_readout_noise_and_frames(env):
    torch, sp, ctx = env
    det = _det(torch, 33)
    a, b, c = (torch.empty_like(det) for _ in range(3))
    sp.specula_ccd(ctx, det, 20.0, 3.0, 99, 4, a)
    sp.specula_ccd(ctx, det, 20.0, 3.0, 99, 4, b)
    sp.specula_ccd(ctx, det, 20.0, 3.0, 99, 5, c)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and not torch.equal(a, c)
    ref = ccd.ccd_read(det.cpu().numpy(), 20.0, 3.0, 99, 4).astype(np.float64)
    got = a.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 2.0 ** -23 * np.abs(ref) + 1e-30)
    with pytest.raises(sp.SpeculaError):
        sp.specula_ccd(ctx, det, -1.0, 0.0, 1, 0, a)


def test_noise_statistics_on_the_gpu(env):
    """Many pixels of one flux: Poisson mean and variance (both samplers)."""
    torch, sp, ctx = env
    n = 200_000
    for lam in (4.0, 120.0):
        det = torch.full((n,), 1.0, device="cuda")
        out = torch.empty_like(det)
        sp.specula_ccd(ctx, det, lam, 0.0, 7, 0, out)
        torch.cuda.synchronize()
        k = out.cpu().numpy().astype(np.float64)
        assert abs(k.mean() - lam) < 5 * np.sqrt(lam / n)
        assert abs(k.var() - lam) < 5 * np.sqrt((lam + 2 * lam * lam) / n)
