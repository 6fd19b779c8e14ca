"""GPU parity of the Shack-Hartmann subaperture partition (the DistributedSH
analogue) and of the mode-row reconstructor split, on one GPU: every block of
subapertures gives exactly the spots and slopes of the full sensor at those
subapertures (the same kernel on a subset), the blocks against the oracle at
the SH tolerance, the host helpers at world size 1, and the refused ranges."""
import numpy as np
import pytest

from gpu_common import close_checked, kolmogorov_phase, load_pkg, need_gpu
from oracle import geometry, sh, slopes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


def _setup(torch, sp, ctx, n, n_sub, sub_pix, fft_n, obsc=0.28):
    pu = sp.PupilDesc(n, 39.0 / n, obsc)
    shd = sp.ShDesc(n_sub, sub_pix, fft_n)
    nv = sp.specula_sh_plan(ctx, pu, shd)
    amp = torch.empty(n, n, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    return pu, shd, nv, amp


@pytest.mark.parametrize("n,n_sub,sub_pix,fft_n,blocks", [(816, 68, 12, 24, 3), (128, 16, 8, 16, 4)])
def test_blocks_equal_the_full_sensor(env, n, n_sub, sub_pix, fft_n, blocks):
    torch, sp, ctx = env
    from paper_2602_06688_gb300.sharding import block_ranges, join_xy
    pu, shd, nv, amp = _setup(torch, sp, ctx, n, n_sub, sub_pix, fft_n)
    phi = kolmogorov_phase(n, 39.0 / n, 0.5, seed=9, side=1024 if n > 512 else None)
    ph = torch.tensor(phi[None].astype(np.float32), device="cuda")
    idx = torch.zeros(nv, dtype=torch.int32, device="cuda")
    full = torch.empty(1, nv, fft_n, fft_n, device="cuda")
    sp.specula_sh_image(ctx, pu, shd, amp, ph, full, nv)
    sc = sp.slopec_desc(sp.SLOPES_SH, n_sub, idx, fft_n)
    s_full = torch.empty(1, 2 * nv, device="cuda")
    sp.specula_slopes(ctx, sc, full, None, s_full)
    pieces = []
    for b, e in block_ranges(nv, blocks):
        sp.specula_sh_set_range(ctx, pu, shd, b, e)
        part = torch.full((1, e - b, fft_n, fft_n), float("nan"), device="cuda")
        sp.specula_sh_image(ctx, pu, shd, amp, ph, part, e - b)
        scb = sp.slopec_desc(sp.SLOPES_SH, n_sub, idx[b:e], fft_n)
        s_b = torch.empty(1, 2 * (e - b), device="cuda")
        sp.specula_slopes(ctx, scb, part, None, s_b)
        torch.cuda.synchronize()
        assert torch.equal(part[0], full[0, b:e])
        pieces.append(s_b[0])
    assert torch.equal(join_xy(pieces), s_full[0])
    sp.specula_sh_set_range(ctx, pu, shd, 0, nv)      # the whole sensor again
    again = torch.empty_like(full)
    sp.specula_sh_image(ctx, pu, shd, amp, ph, again, nv)
    torch.cuda.synchronize()
    assert torch.equal(again, full)
    # one block against the oracle (relative to each spot's brightest pixel)
    amp64 = geometry.pupil_mask(n, 0.28).astype(np.float64)
    valid = geometry.valid_subaps(amp64.astype(np.uint8), n_sub)
    b, e = block_ranges(nv, blocks)[1]
    ref = sh.sh_spots(amp64, ph[0].cpu().numpy().astype(np.float64), n_sub, sub_pix, fft_n,
                      valid[b:e])
    got = full[0, b:e].cpu().numpy().astype(np.float64)
    err = np.max(np.abs(got - ref), axis=(1, 2)) / np.max(ref, axis=(1, 2))
    assert err.max() <= 1e-5


def test_host_helpers_at_world_one(env):
    torch, sp, ctx = env
    from paper_2602_06688_gb300.sharding import ModeRowRecon, SubapShardedSH
    n, n_sub, sub_pix, fft_n = 128, 16, 8, 16
    pu, shd, nv, amp = _setup(torch, sp, ctx, n, n_sub, sub_pix, fft_n)
    ph = torch.tensor(kolmogorov_phase(n, 39.0 / n, 0.5, seed=4)[None].astype(np.float32),
                      device="cuda")
    sh_s = SubapShardedSH(ctx, pu, shd, nv)
    got = sh_s.slopes(amp, ph)
    full = torch.empty(1, nv, fft_n, fft_n, device="cuda")
    sp.specula_sh_image(ctx, pu, shd, amp, ph, full, nv)
    ref = torch.empty(1, 2 * nv, device="cuda")
    sp.specula_slopes(ctx, sp.slopec_desc(sp.SLOPES_SH, n_sub,
                                          torch.zeros(nv, dtype=torch.int32, device="cuda"),
                                          fft_n), full, None, ref)
    torch.cuda.synchronize()
    assert torch.equal(got, ref[0])
    R = torch.randn(301, 2 * nv, device="cuda")
    mr = ModeRowRecon(ctx, R)
    m = mr.modes(ref[0])
    m_ref = torch.empty(301, device="cuda")
    sp.specula_recon(ctx, sp.recon_desc(301, 2 * nv, sp.PREC_FP32, R), ref[0], m_ref)
    torch.cuda.synchronize()
    assert torch.equal(m, m_ref)


def test_refused_ranges(env):
    torch, sp, ctx = env
    n, n_sub, sub_pix, fft_n = 128, 16, 8, 16
    pu, shd, nv, amp = _setup(torch, sp, ctx, n, n_sub, sub_pix, fft_n)
    for b, e in [(-1, 4), (5, 4), (0, nv + 1)]:
        with pytest.raises(sp.SpeculaError) as ex:
            sp.specula_sh_set_range(ctx, pu, shd, b, e)
        assert ex.value.status == sp.EINVAL
    with pytest.raises(sp.SpeculaError) as ex:
        sp.specula_sh_set_range(ctx, sp.PupilDesc(64, 0.3, 0.28), sp.ShDesc(8, 8, 16), 0, 1)
    assert ex.value.status == sp.ENOPLAN
    sp.specula_sh_set_range(ctx, pu, shd, 3, 3)      # an empty block images nothing
    sentinel = torch.full((1,), 7.0, device="cuda")
    sp.specula_sh_image(ctx, pu, shd, amp, torch.zeros(1, n, n, device="cuda"), sentinel, 0)
    torch.cuda.synchronize()
    assert float(sentinel[0]) == 7.0
    sp.specula_sh_set_range(ctx, pu, shd, 0, nv)
