"""Oracle pins: Zernike basis, modal projection, push-pull IM and pinv."""
import math

import numpy as np
import pytest

from oracle import calib, geometry, modal


def test_noll_table():
    ref = [(0, 0), (1, 1), (1, -1), (2, 0), (2, -2), (2, 2), (3, -1), (3, 1), (3, -3),
           (3, 3), (4, 0), (4, 2), (4, -2), (4, 4), (4, -4), (5, 1), (5, -1)]
    assert [modal.noll_to_nm(j) for j in range(1, 18)] == ref


def test_closed_forms():
    rng = np.random.default_rng(0)
    rho, th = rng.uniform(0, 1, 50), rng.uniform(0, 2 * np.pi, 50)
    assert np.allclose(modal.zernike(2, rho, th), 2 * rho * np.cos(th), atol=1e-14)
    assert np.allclose(modal.zernike(3, rho, th), 2 * rho * np.sin(th), atol=1e-14)
    assert np.allclose(modal.zernike(4, rho, th), math.sqrt(3) * (2 * rho ** 2 - 1), atol=1e-14)
    assert np.allclose(modal.zernike(7, rho, th),
                       math.sqrt(8) * (3 * rho ** 3 - 2 * rho) * np.sin(th), atol=1e-14)
    assert np.allclose(modal.zernike(11, rho, th),
                       math.sqrt(5) * (6 * rho ** 4 - 6 * rho ** 2 + 1), atol=1e-13)


def test_continuous_orthonormality():
    """(1/pi) integral over the unit disk of Z_i Z_j = delta_ij (Gauss-Legendre
    in rho, uniform in theta: exact for these polynomials)."""
    x, w = np.polynomial.legendre.leggauss(40)
    rho = 0.5 * (x + 1)
    wr = 0.5 * w * rho
    th = np.linspace(0, 2 * np.pi, 96, endpoint=False)
    R, T = np.meshgrid(rho, th, indexing="ij")
    W = wr[:, None] * (2 * np.pi / len(th)) / np.pi
    J = 45
    Z = np.stack([modal.zernike(j, R, T) for j in range(1, J + 1)])
    G = np.einsum("iab,jab,ab->ij", Z, Z, W)
    assert np.max(np.abs(G - np.eye(J))) < 1e-12


def test_projection_recovers_coefficients():
    n, obsc, nm = 32, 0.2, 20
    B = modal.modal_basis(n, obsc, nm)
    mask = geometry.pupil_mask(n, obsc)
    c = np.random.default_rng(1).standard_normal(nm)
    phi = np.tensordot(c, B, axes=1)
    assert np.allclose(modal.project(B, phi, mask), c, atol=1e-10)
    cc = np.random.default_rng(2).standard_normal((3, nm))
    phis = np.tensordot(cc, B, axes=1)
    assert np.allclose(modal.project(B, phis, mask), cc, atol=1e-10)


def test_pinv_truncated_penrose():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((60, 20)) @ np.diag(np.logspace(0, -6, 20)) @ rng.standard_normal((20, 20))
    for rc in (1e-3, 1e-9):
        R, k = calib.pinv_truncated(A, rc)
        s = calib.singular_values(A)
        assert k == int((s > rc * s[0]).sum())
        # Penrose conditions hold for the rank-k truncation A_k of A
        U, sv, Vt = np.linalg.svd(A, full_matrices=False)
        Ak = (U[:, :k] * sv[:k]) @ Vt[:k]
        assert np.allclose(Ak @ R @ Ak, Ak, atol=1e-9 * np.abs(Ak).max())
        assert np.allclose(R @ Ak @ R, R, atol=1e-9 * np.abs(R).max())
        assert np.allclose((Ak @ R).T, Ak @ R, atol=1e-9)
        assert np.allclose((R @ Ak).T, R @ Ak, atol=1e-9)


@pytest.fixture(scope="module")
def small_im():
    n, nsub, obsc, nmod, r, nm = 32, 8, 0.0, 8, 3.0, 12
    amp = geometry.pupil_mask(n, obsc).astype(np.float64)
    valid = geometry.valid_subaps(amp.astype(np.uint8), nsub)
    B = modal.modal_basis(n, obsc, nm)
    IM = calib.push_pull_im(amp, B, 0.05, 2, nmod, r, nsub, n, valid)
    return IM, valid, nsub, amp, B


def test_im_tip_tilt_transpose_and_sign(small_im):
    IM, valid, nsub, _, _ = small_im
    nv = len(valid)

    def grid(v):
        g = np.zeros(nsub * nsub)
        g[valid] = v
        return g.reshape(nsub, nsub)

    tip, tilt = IM[:, 0], IM[:, 1]
    assert tip[:nv].mean() > 0 and tilt[nv:].mean() > 0        # +x tip -> +Sx
    assert abs(tip[nv:].mean()) < 1e-12 and abs(tilt[:nv].mean()) < 1e-12
    # Z3(x, y) = Z2(y, x): the tilt's y slopes are the transposed tip x slopes
    assert np.allclose(grid(tilt[nv:]), grid(tip[:nv]).T, atol=1e-12)


def test_reconstructor_closure(small_im):
    IM, *_ = small_im
    R, k = calib.pinv_truncated(IM, 1e-3)
    assert k == IM.shape[1]
    assert np.allclose(R @ IM, np.eye(k), atol=1e-10)


def test_radial_mp_matches_float64_at_low_order_and_closed_forms():
    """At low radial order the float64 sum is exact to rounding: the two agree;
    R_n^m(1) = 1 for every order (the sum of the coefficients); R_n^n = rho^n."""
    rho = np.linspace(0.0, 1.0, 17)
    for n in range(0, 16):
        for m in range(n % 2, n + 1, 2):
            ref = modal.radial(n, m, rho)
            got = np.array([modal.radial_mp(n, m, r) for r in rho])
            # float64 rounding bound of the alternating sum: eps sum_s |c_s| (times the terms)
            csum = sum(math.factorial(n - s) // (math.factorial(s) * math.factorial((n + m) // 2 - s)
                                                 * math.factorial((n - m) // 2 - s))
                       for s in range((n - m) // 2 + 1))
            assert np.max(np.abs(got - ref)) <= 4 * (n + 1) * 2.0 ** -52 * csum, (n, m)
    for n, m in [(40, 0), (61, 3), (88, 2), (89, 89), (90, 44)]:
        assert abs(modal.radial_mp(n, m, 1.0) - 1.0) <= 1e-14
    assert abs(modal.radial_mp(37, 37, 0.9) - 0.9 ** 37) <= 1e-15


def test_radial_mp_orthogonality_at_high_order():
    """int_0^1 R_n^m R_n'^m rho d rho = delta_nn' / (2 (n + 1)), by Gauss-Legendre
    quadrature (exact for these degrees) on radial_mp, at the orders a
    4000-mode basis reaches (radial order 88)."""
    x, w = np.polynomial.legendre.leggauss(120)
    rho, wt = 0.5 * (x + 1.0), 0.5 * w
    for (n1, n2, m) in [(84, 84, 0), (84, 86, 0), (87, 87, 5), (85, 87, 5), (88, 88, 20)]:
        f1 = np.array([modal.radial_mp(n1, m, r) for r in rho])
        f2 = np.array([modal.radial_mp(n2, m, r) for r in rho])
        v = float(np.sum(wt * f1 * f2 * rho))
        ref = 1.0 / (2 * (n1 + 1)) if n1 == n2 else 0.0
        assert abs(v - ref) <= 1e-10, (n1, n2, m, v)
