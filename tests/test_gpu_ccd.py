"""GPU detector noise against the FP64 oracle.  The kernel evaluates the
oracle's model on the same Philox words in float32 (the multiplicative
method's uniforms, product and exp(-lambda) threshold; the Box-Muller pair),
the oracle in float64, so per pixel:

* photon counts agree on all but a small fraction of pixels and every
  disagreement is one count: the float32 product can end on the other side
  of the threshold when it lands within a few roundings of it, and the
  rounded normal can cross a half-integer by the float32 normal's error;
* reads agree within one float32 rounding plus ron times the float32
  Box-Muller error (at most 5e-4 absolute: sqrt of the error of r^2, reached
  only where u0 rounds to 1);

and over many pixels of one flux the GPU's counts follow Poisson(lambda)
below the switch and the rounded normal above it (moments and chi-squared),
and its readout normal passes a Kolmogorov-Smirnov test."""
import math

import numpy as np
import pytest

from gpu_common import close_checked, load_pkg, need_gpu
from oracle import ccd

pytestmark = pytest.mark.gpu

G_ABS = 5e-4          # float32 Box-Muller normal against float64, absolute


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


def _agree(got, ref, ron):
    """Per-pixel agreement: the count difference (0 or 1 in magnitude) and the
    read within the float32 bound; returns the number of count differences."""
    got, ref = got.astype(np.float64).ravel(), ref.astype(np.float64).ravel()
    dk = np.round(got - ref)
    assert np.all(np.abs(dk) <= 1.0)
    tol = 2.0 ** -22 * np.abs(ref) + ron * G_ABS + 2.0 ** -22 * np.abs(got)
    assert np.all(np.abs(got - ref - dk) <= tol)
    return int(np.count_nonzero(dk))


@pytest.mark.parametrize("scale", [3.0, 60.0, 400.0])
def test_photon_counts_agree(env, scale):
    torch, sp, ctx = env
    det = _det(torch, 33)                                    # 1089 px: ragged last block
    out = torch.empty_like(det)
    sp.specula_ccd(ctx, det, scale, 0.0, 0x1234_5678_9ABC, 17, out)
    torch.cuda.synchronize()
    ref = ccd.ccd_read(det.cpu().numpy(), scale, 0.0, 0x1234_5678_9ABC, 17)
    got = out.cpu().numpy()
    assert np.all(got == np.round(got))
    n_diff = _agree(got, ref, 0.0)
    assert n_diff <= 2 + got.size // 500, n_diff
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
    ref = ccd.ccd_read(det.cpu().numpy(), 20.0, 3.0, 99, 4)
    n_diff = _agree(a.cpu().numpy(), ref, 3.0)
    assert n_diff <= 2 + ref.size // 500, n_diff
    with pytest.raises(sp.SpeculaError):
        sp.specula_ccd(ctx, det, -1.0, 0.0, 1, 0, a)


def _chi2_pvalue(k, pmf, kmax):
    from scipy import stats
    n = k.size
    probs = np.array([pmf(j) for j in range(kmax + 1)])
    probs = np.append(probs, max(0.0, 1.0 - probs.sum()))
    obs = np.bincount(np.minimum(k, kmax + 1), minlength=kmax + 2).astype(np.float64)
    exp_, ob, acc_e, acc_o = [], [], 0.0, 0.0
    for e, o in zip(probs * n, obs):
        acc_e += e
        acc_o += o
        if acc_e >= 5.0:
            exp_.append(acc_e)
            ob.append(acc_o)
            acc_e = acc_o = 0.0
    exp_[-1] += acc_e
    ob[-1] += acc_o
    exp_, ob = np.array(exp_), np.array(ob)
    return float(stats.chi2.sf(float(((ob - exp_) ** 2 / exp_).sum()), len(exp_) - 1))


def test_noise_statistics_on_the_gpu(env):
    """200k pixels of one flux: Poisson(lambda) in moments and by chi-squared
    below the switch, the rounded normal of mean and variance lambda above
    it; the readout normal of dark pixels by Kolmogorov-Smirnov."""
    from scipy import stats
    torch, sp, ctx = env
    n = 200_000
    for lam in (4.0, 120.0):
        det = torch.full((n,), 1.0, device="cuda")
        out = torch.empty_like(det)
        sp.specula_ccd(ctx, det, lam, 0.0, 7, 0, out)
        torch.cuda.synchronize()
        k = out.cpu().numpy().astype(np.int64)
        assert abs(k.mean() - lam) < 5 * np.sqrt(lam / n)
        assert abs(k.var() - lam) < 5 * np.sqrt((lam + 2 * lam * lam) / n)
        if lam <= ccd.LAMBDA_SWITCH:
            pmf = lambda j: math.exp(-lam + j * math.log(lam) - math.lgamma(j + 1))
        else:
            s = math.sqrt(lam)
            cdf = lambda x: 0.5 * math.erfc(-x / math.sqrt(2.0))
            pmf = lambda j: cdf((j + 0.5 - lam) / s) - (cdf((j - 0.5 - lam) / s) if j else 0.0)
        assert _chi2_pvalue(k, pmf, int(lam + 8 * math.sqrt(lam) + 8)) > 1e-3
    dark = torch.zeros(n, device="cuda")
    out = torch.empty_like(dark)
    sp.specula_ccd(ctx, dark, 1.0, 2.0, 11, 3, out)
    torch.cuda.synchronize()
    g = out.cpu().numpy().astype(np.float64) / 2.0
    assert stats.kstest(g, "norm").pvalue > 1e-3


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
