"""GPU parity: Shack-Hartmann spots and slopes; reconstructor MVM precisions."""
import numpy as np
import pytest

from gpu_common import close_checked, kolmogorov_phase, load_pkg, need_gpu, pupil_amp
from oracle import geometry, recon, sh, slopes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


# the last two: Sect. 6 Tab. 2's SCAO SH (20 x 20 lenslets of 8 px, 56^2
# spots) and ERIS (40 x 40 of 4 px, 68^2 spots), transforms wider than a warp
@pytest.mark.parametrize("n_sub,sub_pix,fft_n,obsc,nb", [(10, 8, 16, 0.2, 2), (68, 12, 24, 0.28, 1),
                                                         (20, 8, 56, 0.14, 2), (40, 4, 68, 0.14, 1)])
def test_sh_spots_and_slopes(env, n_sub, sub_pix, fft_n, obsc, nb):
    torch, sp, ctx = env
    n_pix = n_sub * sub_pix
    amp = pupil_amp(n_pix, obsc)
    valid = geometry.valid_subaps(amp.astype(np.uint8), n_sub)
    phis = [kolmogorov_phase(n_pix, 39.0 / n_pix, 0.157, seed=40 + k, wavelength_nm=589.0)
            .astype(np.float32) for k in range(nb)]
    pu = sp.PupilDesc(n_pix, 39.0 / n_pix, obsc)
    shd = sp.ShDesc(n_sub, sub_pix, fft_n)
    nv = sp.specula_sh_plan(ctx, pu, shd)
    assert nv == len(valid)
    amp_t = torch.tensor(amp.astype(np.float32), device="cuda")
    ph = torch.tensor(np.stack(phis), device="cuda")
    spots = torch.empty(nb, nv, fft_n, fft_n, device="cuda")
    sp.specula_sh_image(ctx, pu, shd, amp_t, ph, spots, nv)
    idx = torch.tensor(valid, device="cuda")
    sc = sp.slopec_desc(sp.SLOPES_SH, n_sub, idx, fft_n)
    s_t = torch.empty(nb, 2 * nv, device="cuda")
    sp.specula_slopes(ctx, sc, spots, None, s_t)
    torch.cuda.synchronize()
    got = spots.cpu().numpy().astype(np.float64)
    for k in range(nb):
        ref = sh.sh_spots(amp, phis[k].astype(np.float64), n_sub, sub_pix, fft_n, valid)
        # per spot, relative to its brightest pixel
        err = np.max(np.abs(got[k] - ref), axis=(1, 2)) / np.max(ref, axis=(1, 2))
        assert err.max() <= 1e-5, err.max()
        s_ref = slopes.sh_slopes(ref)
        # CoG in pixels; from the spot error: |dS| <= (n/2 + |S|) n^2 eps max / sum
        bound = 1e-5 * fft_n ** 3 * (ref.max(axis=(1, 2)) / ref.sum(axis=(1, 2)))
        bound = np.concatenate([bound, bound]) + 1e-6
        assert np.all(np.abs(s_t[k].cpu().numpy() - s_ref) <= bound)
        # slope kernel alone on identical input
        s_same = slopes.sh_slopes(got[k])
        assert np.max(np.abs(s_t[k].cpu().numpy() - s_same)) <= 2e-6 * fft_n


# batches of 32 and more run the bf16 forms on the tensor cores (one
# multi-term GEMM over the slopes' bf16 halves)
@pytest.mark.parametrize("nm,ns,nb", [(200, 416, 1), (500, 2512, 3), (4000, 13344, 1), (37, 104, 5),
                                      (37, 104, 64), (500, 2512, 40), (4000, 13344, 128)])
def test_recon_precisions(env, nm, ns, nb):
    torch, sp, ctx = env
    rng = np.random.default_rng(nm)
    R = (rng.standard_normal((nm, ns)) / np.sqrt(ns)).astype(np.float32)
    s = rng.standard_normal((nb, ns)).astype(np.float32)
    ref = recon.mvm(R.astype(np.float64), s.astype(np.float64))
    mag = np.abs(s.astype(np.float64)) @ np.abs(R.astype(np.float64)).T   # sum_j |R_ij s_j|
    R_t = torch.tensor(R, device="cuda")
    s_t = torch.tensor(s, device="cuda")
    out = torch.empty(nb, nm, device="cuda")
    sp.specula_recon(ctx, sp.recon_desc(nm, ns, sp.PREC_FP32, R_t), s_t, out)
    torch.cuda.synchronize()
    assert np.all(np.abs(out.cpu().numpy() - ref) <= 1e-5 * mag)
    hi = torch.empty(nm, ns, dtype=torch.int16, device="cuda")
    lo = torch.empty(nm, ns, dtype=torch.int16, device="cuda")
    sp.specula_recon_convert(ctx, R_t, sp.PREC_BF16X2, hi, lo)
    torch.cuda.synchronize()
    # the split is exact where bf16 holds R: hi is the nearest bf16 of R
    hb = hi.view(torch.bfloat16).float().cpu().numpy()
    assert np.all(np.abs(hb - R) <= 2.0 ** -8 * np.abs(R))
    if ns % 8 == 0:
        sp.specula_recon(ctx, sp.recon_desc(nm, ns, sp.PREC_BF16, hi), s_t, out)
        torch.cuda.synchronize()
        assert np.all(np.abs(out.cpu().numpy() - ref) <= 2.0 ** -8 * mag + 1e-5 * mag)
        sp.specula_recon(ctx, sp.recon_desc(nm, ns, sp.PREC_BF16X2, hi, lo), s_t, out)
        torch.cuda.synchronize()
        assert np.all(np.abs(out.cpu().numpy() - ref) <= 2.0 ** -16 * mag + 1e-5 * mag)
    # deterministic
    a = torch.empty_like(out)
    sp.specula_recon(ctx, sp.recon_desc(nm, ns, sp.PREC_FP32, R_t), s_t, a)
    b = torch.empty_like(out)
    sp.specula_recon(ctx, sp.recon_desc(nm, ns, sp.PREC_FP32, R_t), s_t, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
