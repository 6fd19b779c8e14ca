"""GPU parity of the detector noise against the oracle: photon counts
bit-exact (both sides decide them with the same IEEE operations on the same
Philox words), the readout-noise sum within one float32 rounding plus the
float32 readout normal's last-bit differences."""
import numpy as np
import pytest

from gpu_common import close_checked, load_pkg, need_gpu
from oracle import ccd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


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
    # the readout normal is float32 on both sides (library log/sin may differ
    # in the last bit): one float32 rounding of the sum plus ron x 1e-6
    assert np.all(np.abs(got - ref) <= 2.0 ** -23 * np.abs(ref) + 3.0 * 1e-6)
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


def test_device_frame_index(env):
    torch, sp, ctx = env
    det = _det(torch, 33)
    a, b = torch.empty_like(det), torch.empty_like(det)
    fd = torch.tensor([3], dtype=torch.int32, device="cuda")
    sp.specula_ccd(ctx, det, 20.0, 1.0, 5, 2, a, frame_dev=fd)
    sp.specula_ccd(ctx, det, 20.0, 1.0, 5, 5, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_noisy_frame_replay_matches_eager(env):
    """The pyramid frame with detector noise: a graph replay at t = k dt draws
    the noise of frame k, as the eager frame at that time does."""
    torch, sp, ctx = env
    import synth
    from paper_2602_06688_gb300.frame import PwfsFrame
    fr = PwfsFrame(ctx, synth.workload("pwfs8m_tiny"),
                   noise={"photons": 1e5, "qe": 0.9, "ron": 1.0, "seed": 3})
    st = torch.cuda.Stream()
    fr.capture(st)
    seen = []
    for k in (1, 4):
        fr.frame(k * fr.dt)
        torch.cuda.synchronize()
        eager = fr.slopes.clone()
        fr.slopes.zero_()
        torch.cuda.synchronize()
        fr.replay(k * fr.dt, st)
        torch.cuda.synchronize()
        assert torch.equal(fr.slopes, eager)
        seen.append(eager)
    assert not torch.equal(seen[0], seen[1])
    fr.graph.close()
