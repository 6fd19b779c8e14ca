"""GPU parity of the polychromatic Shack-Hartmann spots against the oracle
(three wavelengths, batch 2, both supported spot sizes), the single
reference band against the monochromatic call bit for bit, and the refused
arguments.  Tolerance as for the monochromatic spots: 1e-5 of each spot's
brightest pixel, plus the float32 rounding of the weights and sums."""
import numpy as np
import pytest

from gpu_common import close_checked, kolmogorov_phase, load_pkg, need_gpu
from oracle import geometry, sh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


def _setup(torch, sp, ctx, n, n_sub, sub_pix, fft_n, obsc=0.2):
    pu = sp.PupilDesc(n, 8.0 / n, obsc)
    shd = sp.ShDesc(n_sub, sub_pix, fft_n)
    nv = sp.specula_sh_plan(ctx, pu, shd)
    amp = torch.empty(n, n, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    return pu, shd, nv, amp


@pytest.mark.parametrize("n,n_sub,sub_pix,fft_n", [(128, 16, 8, 16), (240, 20, 12, 24)])
def test_poly_spots_match_the_oracle(env, n, n_sub, sub_pix, fft_n):
    torch, sp, ctx = env
    pu, shd, nv, amp = _setup(torch, sp, ctx, n, n_sub, sub_pix, fft_n)
    phs = np.stack([kolmogorov_phase(n, 8.0 / n, 0.4, seed=s) for s in (5, 6)]).astype(np.float32)
    ph = torch.tensor(phs, device="cuda")
    ratios, weights = [1.25, 1.0, 0.8], [0.3, 0.45, 0.25]
    out = torch.full((2, nv, fft_n, fft_n), float("nan"), device="cuda")
    sp.specula_sh_image_poly(ctx, pu, shd, ratios, weights, amp, ph, out, nv)
    torch.cuda.synchronize()
    assert sp.specula_ctx_status(ctx) == 0
    a64 = geometry.pupil_mask(n, 0.2).astype(np.float64)
    valid = geometry.valid_subaps(a64.astype(np.uint8), n_sub)
    for b in range(2):
        ref = sh.sh_spots_poly(a64, phs[b].astype(np.float64), n_sub, sub_pix, fft_n, valid,
                               ratios, weights)
        got = out[b].cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        err = np.max(np.abs(got - ref), axis=(1, 2)) / np.max(ref, axis=(1, 2))
        assert err.max() <= 2e-5, err.max()


def test_reference_band_alone_is_the_mono_call(env):
    torch, sp, ctx = env
    n, n_sub, sub_pix, fft_n = 128, 16, 8, 16
    pu, shd, nv, amp = _setup(torch, sp, ctx, n, n_sub, sub_pix, fft_n)
    ph = torch.tensor(kolmogorov_phase(n, 8.0 / n, 0.4, seed=8)[None].astype(np.float32),
                      device="cuda")
    mono = torch.empty(1, nv, fft_n, fft_n, device="cuda")
    sp.specula_sh_image(ctx, pu, shd, amp, ph, mono, nv)
    poly = torch.empty_like(mono)
    sp.specula_sh_image_poly(ctx, pu, shd, [1.0], [1.0], amp, ph, poly, nv)
    torch.cuda.synchronize()
    assert torch.equal(mono, poly)


def test_poly_arguments(env):
    torch, sp, ctx = env
    n, n_sub, sub_pix, fft_n = 128, 16, 8, 16
    pu, shd, nv, amp = _setup(torch, sp, ctx, n, n_sub, sub_pix, fft_n)
    ph = torch.zeros(1, n, n, device="cuda")
    out = torch.empty(1, nv, fft_n, fft_n, device="cuda")
    for r in ([0.0], [-1.0], [float("nan")]):
        with pytest.raises(sp.SpeculaError) as e:
            sp.specula_sh_image_poly(ctx, pu, shd, r, [1.0], amp, ph, out, nv)
        assert e.value.status == sp.EINVAL
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_sh_image_poly(ctx, sp.PupilDesc(64, 0.3, 0.28), sp.ShDesc(8, 8, 16), [1.0],
                                 [1.0], amp, torch.zeros(1, 64, 64, device="cuda"), out, nv)
    assert e.value.status == sp.ENOPLAN


def test_reserved_workspaces_make_the_calls_capturable(env):
    """After the set-up reserve calls, the batched bf16 reconstructor and the
    polychromatic SH enqueue without allocating: both capture into a graph
    whose replay equals the eager calls bit for bit."""
    torch, sp, _ = env
    ctx = sp.Context(0)
    try:
        n, n_sub, sub_pix, fft_n = 128, 16, 8, 16
        pu, shd, nv, amp = _setup(torch, sp, ctx, n, n_sub, sub_pix, fft_n)
        ph = torch.tensor(np.stack([kolmogorov_phase(n, 8.0 / n, 0.4, seed=s) for s in (1, 2)])
                          .astype(np.float32), device="cuda")
        nm, ns, nb = 300, 2 * nv, 64
        g = torch.Generator(device="cuda").manual_seed(5)
        R = torch.randn(nm, ns, device="cuda", generator=g) / ns ** 0.5
        hi = torch.empty(nm, ns, dtype=torch.int16, device="cuda")
        lo = torch.empty_like(hi)
        sp.specula_recon_convert(ctx, R, sp.PREC_BF16X2, hi, lo)
        rec = sp.recon_desc(nm, ns, sp.PREC_BF16X2, hi, lo)
        X = torch.randn(nb, ns, device="cuda", generator=g)
        sp.specula_recon_reserve(ctx, rec, nb)
        sp.specula_sh_poly_reserve(ctx, pu, shd, 2)
        ratios, weights = [1.2, 0.9], [0.5, 0.5]
        st = torch.cuda.Stream()
        m_g = torch.empty(nb, nm, device="cuda")
        s_g = torch.empty(2, nv, fft_n, fft_n, device="cuda")
        torch.cuda.synchronize()
        sp.specula_graph_begin(ctx, st)
        try:
            sp.specula_recon(ctx, rec, X, m_g, stream=st)
            sp.specula_sh_image_poly(ctx, pu, shd, ratios, weights, amp, ph, s_g, nv, stream=st)
        finally:
            graph = sp.specula_graph_end(ctx, st)
        graph.launch(st)
        torch.cuda.synchronize()
        m_e = torch.empty_like(m_g)
        s_e = torch.empty_like(s_g)
        sp.specula_recon(ctx, rec, X, m_e)
        sp.specula_sh_image_poly(ctx, pu, shd, ratios, weights, amp, ph, s_e, nv)
        torch.cuda.synchronize()
        assert torch.equal(m_g, m_e) and torch.equal(s_g, s_e)
        graph.close()
    finally:
        close_checked(sp, ctx)
