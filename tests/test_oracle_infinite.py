"""Oracle pins: infinite phase screens (conditional line-by-line growth).

The covariance is pinned to the spectrum it comes from: a numerical Hankel
transform of the FFT screens' von Karman spectrum, the elementary integral of
its variance, and the small-separation expansion of the Bessel function.  The
conditional operators are pinned to the joint covariance they must reproduce
and to the precision-matrix form of the Gaussian conditional.  The growth
conventions are pinned by exact mirror and transpose identities and by the
structure function of a long grown strip."""
import math

import numpy as np
from scipy import integrate, special

from oracle import infinite as inf
from oracle import screens

R0, L0 = 0.15, 25.0


def _hankel(r, r0=R0, L0_=L0):
    """2 pi int f Phi(f) J0(2 pi f r) df, split at the zeros of J0; the
    alternating tail is closed by averaging the last two partial sums."""
    def f(x):
        return 2 * math.pi * x * screens.vk_psd(np.array([x]), np.array([0.0]), r0, L0_)[0] \
            * special.j0(2 * math.pi * x * r)
    if r == 0:
        return integrate.quad(f, 0, np.inf, limit=500)[0]
    z = special.jn_zeros(0, 1500) / (2 * math.pi * r)
    edges = np.concatenate([[0.0], z])
    s = np.cumsum([integrate.quad(f, a, b, limit=200)[0] for a, b in zip(edges[:-1], edges[1:])])
    return 0.5 * (s[-1] + s[-2])


def test_covariance_is_the_hankel_transform_of_the_spectrum():
    for r in (0.0, 0.02, 0.2, 1.0, 5.0, 20.0):
        c = inf.vk_covariance(np.array([r]), R0, L0)[0]
        assert abs(_hankel(r) - c) <= 1e-9 * c


def test_variance_closed_form():
    """int 2 pi f 0.023 r0^-5/3 (f^2 + L0^-2)^-11/6 df = 0.023 pi (6/5) (L0/r0)^5/3."""
    for r0, L0_ in ((0.1, 10.0), (0.15, 25.0), (0.3, 100.0)):
        c0 = inf.vk_covariance(np.array([0.0]), r0, L0_)[0]
        assert abs(c0 - 0.023 * math.pi * 1.2 * (L0_ / r0) ** (5 / 3)) <= 1e-13 * c0


def test_small_separation_expansion():
    """x^nu K_nu(x) = 2^(nu-1) Gamma(nu) (1 + x^2 / (4 (1 - nu)))
    - Gamma(1 - nu) 2^(-nu-1) x^(2 nu) / nu + O(x^(2 + 2 nu)), and the leading
    term gives the Kolmogorov law D(r) = 2 (C(0) - C(r)) = k (r/r0)^(5/3) with
    k = 6.8839 x 0.023 / (the exact spectrum constant)."""
    nu = 5.0 / 6.0
    for x in (1e-3, 3e-3):
        r = x * L0 / (2 * math.pi)
        c0, cr = inf.vk_covariance(np.array([0.0, r]), R0, L0)
        scale = c0 / (2 ** (nu - 1) * math.gamma(nu))
        series = 2 ** (nu - 1) * math.gamma(nu) * (1 + x * x / (4 * (1 - nu))) \
            - math.gamma(1 - nu) * 2 ** (-nu - 1) * x ** (2 * nu) / nu
        assert abs(cr / scale - series) <= 10 * x ** (2 + 2 * nu)
    r = 1e-6 * L0
    c0, cr = inf.vk_covariance(np.array([0.0, r]), R0, L0)
    k_exact = 2 * (24 / 5 * math.gamma(6 / 5)) ** (5 / 6)
    c_exact = math.gamma(11 / 6) ** 2 / (2 * math.pi ** (11 / 3)) * (24 / 5 * math.gamma(6 / 5)) ** (5 / 6)
    k_here = k_exact * 0.023 / c_exact
    assert abs(k_exact - 6.8839) < 1e-4
    D = 2 * (c0 - cr)
    assert abs(D / (r / R0) ** (5 / 3) / k_here - 1) < 2e-2   # O((r/L0)^(1/3)) = 1e-2 here


def _joint(side, n_st, pitch, r0, L0_):
    Cxx, Czx, Czz = inf.stencil_covariances(side, n_st, pitch, r0, L0_)
    return Cxx, Czx, Czz, np.block([[Cxx, Czx.T], [Czx, Czz]])


def test_operators_reproduce_the_joint_covariance():
    side, n_st, pitch = 16, 2, 0.1
    A, B = inf.line_operators(side, n_st, pitch, R0, L0)
    Cxx, Czx, Czz, _ = _joint(side, n_st, pitch, R0, L0)
    scale = Czz.max()
    assert np.max(np.abs(A @ Cxx - Czx)) <= 1e-8 * scale
    assert np.max(np.abs(A @ Cxx @ A.T + B @ B - Czz)) <= 1e-8 * scale
    assert np.array_equal(B, B.T) or np.max(np.abs(B - B.T)) <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(B).min() >= -1e-10 * np.abs(B).max()


def test_operators_from_the_precision_matrix():
    """Gaussian conditional through Q = Sigma^-1: E[Z|X] = -Q_ZZ^-1 Q_ZX X and
    Cov[Z|X] = Q_ZZ^-1 (side 6, two stencil lines: a well-conditioned case)."""
    side, n_st, pitch = 6, 2, 0.5
    A, B = inf.line_operators(side, n_st, pitch, 0.3, 10.0)
    _, _, _, S = _joint(side, n_st, pitch, 0.3, 10.0)
    Q = np.linalg.inv(S)
    m = side * n_st
    Qzz, Qzx = Q[m:, m:], Q[m:, :m]
    A2 = -np.linalg.solve(Qzz, Qzx)
    C2 = np.linalg.inv(Qzz)
    assert np.max(np.abs(A - A2)) <= 1e-7 * np.abs(A2).max()
    assert np.max(np.abs(B @ B - C2)) <= 1e-7 * np.abs(C2).max()


def test_stencil_index_order_tiny():
    """side 2, one stencil line: X = (line -1 pixel 0, pixel 1), Z = (pixel 0,
    pixel 1); the distances are 1, 1, sqrt 2 pitch as drawn by hand."""
    pitch = 0.3
    Cxx, Czx, Czz = inf.stencil_covariances(2, 1, pitch, R0, L0)
    c = inf.vk_covariance(np.array([0.0, pitch, math.sqrt(2) * pitch]), R0, L0)
    assert np.allclose(Cxx, [[c[0], c[1]], [c[1], c[0]]], rtol=1e-15, atol=0)
    assert np.allclose(Czz, Cxx, rtol=1e-15, atol=0)
    assert np.allclose(Czx, [[c[1], c[2]], [c[2], c[1]]], rtol=1e-15, atol=0)


def test_directions_and_axes_are_mirror_images():
    side, n_st = 12, 2
    A, B = inf.line_operators(side, n_st, 0.1, R0, L0)
    rng = np.random.default_rng(3)
    S = rng.standard_normal((side, side)) * 5
    noise = rng.standard_normal(side)
    h = 7
    down = S.copy()
    inf.add_line(down, A, B, 0, -1, h, noise)
    up = S[::-1].copy()
    inf.add_line(up, A, B, 0, +1, -1 - h, noise)
    assert np.array_equal(up[::-1], down)
    cols = S.copy()
    inf.add_line(cols, A, B, 1, +1, h, noise)
    rows = S.T.copy()
    inf.add_line(rows, A, B, 0, +1, h, noise)
    assert np.array_equal(rows.T, cols)
    # the line written is the one at slot head mod side; nothing else changes
    changed = np.any(down != S, axis=1)
    assert changed.tolist() == [i == h % side for i in range(side)]


def test_r0_scaling_of_the_operators():
    """A does not depend on r0; B scales as r0^(-5/6)."""
    A1, B1 = inf.line_operators(10, 2, 0.1, 0.1, L0)
    A2, B2 = inf.line_operators(10, 2, 0.1, 0.4, L0)
    assert np.max(np.abs(A1 - A2)) <= 1e-9
    assert np.max(np.abs(B2 - (0.1 / 0.4) ** (5 / 6) * B1)) <= 1e-10 * np.abs(B1).max()


def test_line_noise_is_standard_normal_and_keyed_by_line():
    side = 64
    a = np.stack([inf.line_noise(9, 0, L, side) for L in range(-200, 200)])
    assert abs(a.mean()) < 0.02 and abs(a.var() - 1) < 0.03
    assert not np.allclose(inf.line_noise(9, 0, 5, side), inf.line_noise(9, 0, -5, side))
    assert not np.allclose(inf.line_noise(9, 0, 5, side), inf.line_noise(9, 1, 5, side))
    assert np.array_equal(inf.line_noise(9, 2, -7, side), inf.line_noise(9, 2, -7, side))
    # a line's first elements do not depend on its length
    assert np.array_equal(inf.line_noise(9, 2, 3, 10), inf.line_noise(9, 2, 3, 16)[:10])


def test_grown_strip_has_the_von_karman_structure_function():
    """Start from an exact joint draw of a 20 x 20 screen, grow 2500 rows,
    and compare the structure function of the new rows along and across the
    growth direction with 2 (C(0) - C(r)) (statistical tolerance)."""
    side, n_st, pitch, r0, L0_ = 20, 2, 0.1, 0.1, 8.0
    A, B = inf.line_operators(side, n_st, pitch, r0, L0_)
    yy, xx = np.mgrid[0:side, 0:side].astype(np.float64)
    pts = np.stack([xx.ravel(), yy.ravel()], axis=1)
    dist = pitch * np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(axis=2))
    C = inf.vk_covariance(dist, r0, L0_)
    Lc = np.linalg.cholesky(C + 1e-9 * np.eye(side * side) * C[0, 0])
    S = (Lc @ np.random.default_rng(1).standard_normal(side * side)).reshape(side, side)
    n_new = 2500
    strip = np.empty((n_new, side))
    head = side
    for k in range(n_new):
        head = inf.extend(S, A, B, 0, +1, head, 1, seed=77, stream=0)
        strip[k] = inf.get_line(S, 0, head - 1)
    for lag in (1, 2, 4):
        theory = 2 * (C[0, 0] - inf.vk_covariance(np.array([lag * pitch]), r0, L0_)[0])
        along = inf.structure_function(strip, lag)
        across = float(np.mean((strip[:, lag:] - strip[:, :-lag]) ** 2))
        assert abs(along / theory - 1) < 0.08, (lag, along / theory)
        assert abs(across / theory - 1) < 0.08, (lag, across / theory)
