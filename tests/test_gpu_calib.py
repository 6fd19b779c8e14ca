"""GPU parity: push-pull interaction matrix and the float64 pseudo-inverse."""
import numpy as np
import pytest

from gpu_common import close_checked, load_pkg, need_gpu
from oracle import calib, geometry, modal

pytestmark = pytest.mark.gpu

EPS = 1e-5


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


def _gpu_im(torch, sp, ctx, n, obsc, nsub, nmod, r, nm, a):
    pu = sp.PupilDesc(n, 8.0 / n, obsc)
    pw = sp.PwfsDesc(2, nmod, nsub, n, r)
    sp.specula_pwfs_plan(ctx, pu, pw)
    amp = torch.empty(n, n, device="cuda")
    sp.specula_pupil_mask(ctx, pu, amp)
    valid = sp.specula_valid_subaps_host(pu, nsub)
    idx = torch.tensor(valid, device="cuda")
    basis = torch.empty(nm, n, n, device="cuda")
    sp.specula_modal_basis(ctx, pu, nm, basis)
    im = torch.full((2 * len(valid), nm), float("nan"), dtype=torch.float64, device="cuda")
    sp.specula_calib_intmat(ctx, pu, pw, amp, basis, nm, a, sp.slopec_desc(sp.SLOPES_PYR, nsub, idx),
                            im)
    torch.cuda.synchronize()
    return im, valid, basis, amp


@pytest.mark.parametrize("n,obsc,nsub,nmod,r,nm", [(32, 0.2, 8, 8, 3.0, 20),
                                                   (64, 0.0, 16, 12, 3.0, 40)])
def test_intmat_parity(env, n, obsc, nsub, nmod, r, nm):
    torch, sp, ctx = env
    a = 0.1
    im, valid, _, _ = _gpu_im(torch, sp, ctx, n, obsc, nsub, nmod, r, nm, a)
    amp = geometry.pupil_mask(n, obsc).astype(np.float64)
    B = modal.modal_basis(n, obsc, nm)
    ref = calib.push_pull_im(amp, B, a, 2, nmod, r, nsub, n, valid)
    got = im.cpu().numpy()
    # per image |dS| <= 5 eps max(det)/T + eps |S| (detector bound); the push-
    # pull difference divides two such errors by 2a.  max(det)/T <= 1 here.
    bound = 2 * (5 * EPS + EPS * 1.0) / (2 * a)
    err = np.max(np.abs(got - ref))
    assert err <= bound, (err, bound)
    assert np.max(np.abs(ref)) > 0.1


def test_pinv_parity_and_penrose(env):
    torch, sp, ctx = env
    im, valid, basis, amp = _gpu_im(torch, sp, ctx, 64, 0.0, 16, 12, 3.0, 60, 0.1)
    A = im.cpu().numpy()
    s = calib.singular_values(A)
    rcond = 1e-3
    # the truncation must not sit on a singular value (both sides would be
    # right but could keep different ranks)
    assert np.min(np.abs(s / s[0] - rcond)) > 1e-6
    R = torch.empty(A.shape[1], A.shape[0], dtype=torch.float64, device="cuda")
    R32 = torch.empty(A.shape[1], A.shape[0], dtype=torch.float32, device="cuda")
    rank = sp.specula_pinv_fp64(ctx, im, rcond, R, R32)
    torch.cuda.synchronize()
    Rref, kref = calib.pinv_truncated(A, rcond)
    assert rank == kref
    Rg = R.cpu().numpy()
    assert np.max(np.abs(Rg - Rref)) <= 1e-8 * np.abs(Rref).max()
    assert np.array_equal(R32.cpu().numpy(), Rg.astype(np.float32))
    if rank == A.shape[1]:
        assert np.allclose(Rg @ A, np.eye(rank), atol=1e-8)


def test_pinv_rank_deficient_and_odd(env):
    torch, sp, ctx = env
    rng = np.random.default_rng(5)
    A = rng.standard_normal((90, 31)) @ np.diag(np.logspace(0, -8, 31)) @ rng.standard_normal((31, 31))
    A_t = torch.tensor(A, device="cuda")
    R = torch.empty(31, 90, dtype=torch.float64, device="cuda")
    rank = sp.specula_pinv_fp64(ctx, A_t, 1e-4, R)
    torch.cuda.synchronize()
    Rref, kref = calib.pinv_truncated(A, 1e-4)
    assert rank == kref < 31
    assert np.max(np.abs(R.cpu().numpy() - Rref)) <= 1e-7 * np.abs(Rref).max()


def test_calibrated_reconstructor_recovers_modes(env):
    """A pure mode of small amplitude through the GPU frame (image -> slopes ->
    calibrated R) comes back as that mode."""
    torch, sp, ctx = env
    n, nsub, nmod, nm = 64, 16, 12, 40
    im, valid, basis, amp = _gpu_im(torch, sp, ctx, n, 0.0, nsub, nmod, 3.0, nm, 0.1)
    R = torch.empty(nm, im.shape[0], dtype=torch.float64, device="cuda")
    R32 = torch.empty(nm, im.shape[0], device="cuda")
    sp.specula_pinv_fp64(ctx, im, 1e-3, R, R32)
    pu = sp.PupilDesc(n, 8.0 / n, 0.0)
    pw = sp.PwfsDesc(2, nmod, nsub, n, 3.0)
    idx = torch.tensor(valid, device="cuda")
    sc = sp.slopec_desc(sp.SLOPES_PYR, nsub, idx)
    det = torch.empty(2 * nsub, 2 * nsub, device="cuda")
    ref = torch.empty(2 * len(valid), device="cuda")
    sp.specula_pwfs_image(ctx, pu, pw, amp, torch.zeros(n, n, device="cuda"), det)
    sp.specula_slopes(ctx, sc, det, None, ref)
    rec = sp.recon_desc(nm, 2 * len(valid), sp.PREC_FP32, R32)
    for j in (0, 1, 2, 5, 20):
        amp_j = 0.02
        ph = (amp_j * basis[j]).contiguous()
        sp.specula_pwfs_image(ctx, pu, pw, amp, ph, det)
        sl = torch.empty(2 * len(valid), device="cuda")
        sp.specula_slopes(ctx, sc, det, ref, sl)
        m = torch.empty(nm, device="cuda")
        sp.specula_recon(ctx, rec, sl, m)
        torch.cuda.synchronize()
        mv = m.cpu().numpy()
        assert abs(mv[j] - amp_j) < 0.05 * amp_j, (j, mv[j])
        others = np.delete(mv, j)
        assert np.max(np.abs(others)) < 0.05 * amp_j


def test_modal_basis_to_high_radial_order(env):
    """The device basis (Kintner's recurrence in float64, stored as float32)
    against the oracle: all of the first 40 modes against the float64
    definition, and 400 sampled (mode, pixel) values of a 4000-mode basis
    (radial order 88) against the 60-digit evaluation of the same definition;
    the host variant gives the same values."""
    torch, sp, ctx = env
    n, obsc, nm = 160, 0.28, 4000
    pu = sp.PupilDesc(n, 8.0 / n, obsc)
    basis = torch.empty(nm, n, n, device="cuda")
    sp.specula_modal_basis(ctx, pu, nm, basis)
    torch.cuda.synchronize()
    low = modal.modal_basis(n, obsc, 40)
    got = basis[:40].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - low) <= 2.0 ** -23 * np.abs(low) + 1e-12)
    mask = geometry.pupil_mask(n, obsc).astype(bool)
    rho, theta = modal.pupil_polar(n)
    rng = np.random.default_rng(17)
    inside = np.flatnonzero(mask.ravel())
    qs = np.concatenate([rng.integers(0, nm, 300), np.arange(nm - 100, nm)])
    ps = rng.choice(inside, qs.size)
    vals = basis.reshape(nm, -1)[torch.tensor(qs, device="cuda"),
                                 torch.tensor(ps, device="cuda")].cpu().numpy().astype(np.float64)
    for q, p, v in zip(qs, ps, vals):
        ref = modal.zernike_mp(int(q) + 2, float(rho.ravel()[p]), float(theta.ravel()[p]))
        assert abs(v - ref) <= 2.0 ** -22 * abs(ref) + 1e-9, (q, p, v, ref)
    out = basis.reshape(nm, -1)[:, ~mask.ravel()]
    assert float(out.abs().max()) == 0.0
    host = sp.specula_modal_basis_host(pu, 60).reshape(60, n, n)
    assert np.all(np.abs(basis[:60].cpu().numpy() - host.astype(np.float32)) <=
                  2.0 ** -23 * np.abs(host) + 1e-12)
