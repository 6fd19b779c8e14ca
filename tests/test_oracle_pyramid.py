"""Oracle pins: modulated pyramid WFS and its slopes (physics invariants)."""
import numpy as np
import pytest

from oracle import dft, geometry, pyramid, slopes

NP, NSUB = 32, 8
B = NP // NSUB


@pytest.fixture(scope="module")
def pupil():
    amp = geometry.pupil_mask(NP, 0.2).astype(np.float64)
    valid = geometry.valid_subaps(amp.astype(np.uint8), NSUB)
    return amp, valid


def _rand_phase(seed, n=NP, scale=1.0):
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((n, n))


def test_brute_force_tiny_pyramid():
    """Steps 1-6 evaluated with the defining DFT sums on a 4 px pupil."""
    n, pad, nmod, r = 4, 2, 3, 1.5
    N = pad * n
    amp = np.ones((n, n))
    phi = _rand_phase(1, n)
    got = pyramid.pwfs_intensity(amp, phi, pad, nmod, r, n)
    x = dft.centred_coords(n)
    cs, sn = geometry.mod_angles(nmod)
    M = pyramid.pyramid_mask(N, n)
    ref = np.zeros((N, N))
    for m in range(nmod):
        P = np.zeros((N, N), complex)
        P[2:6, 2:6] = amp * np.exp(1j * phi) * np.exp(
            2j * np.pi * r * (x[None, :] * cs[m] + x[:, None] * sn[m]) / n)
        F = dft.brute_centred_dft2(P) * M
        ref += np.abs(dft.brute_centred_dft2(F, inverse=True)) ** 2
    assert np.max(np.abs(got - ref / nmod)) < 1e-12 * ref.max()


def test_parseval_flux(pupil):
    amp, _ = pupil
    I = pyramid.pwfs_intensity(amp, _rand_phase(2, scale=2.0), 2, 8, 3.0, NP)
    assert abs(I.sum() - amp.sum()) < 1e-12 * amp.sum()
    det = pyramid.bin_image(I, B)
    assert abs(det.sum() - amp.sum()) < 1e-12 * amp.sum()


def test_flat_wavefront_four_equal_mirrored_images(pupil):
    amp, valid = pupil
    I = pyramid.pwfs_intensity(amp, np.zeros((NP, NP)), 2, 8, 3.0, NP)
    h = NP
    q = [I[h:, h:].sum(), I[h:, :h].sum(), I[:h, :h].sum(), I[:h, h:].sum()]
    assert np.allclose(q, amp.sum() / 4, rtol=1e-12)
    # Q2 = mirror_x(Q1), Q4 = mirror_y(Q1), Q3 = mirror_xy(Q1), pixel-wise
    assert np.allclose(I, I[:, ::-1], atol=1e-13)
    assert np.allclose(I, I[::-1, :], atol=1e-13)
    det = pyramid.bin_image(I, B)
    s = slopes.pyr_slopes(det, NSUB, valid)
    n = len(valid)
    assert abs(s[:n].sum()) < 1e-12 and abs(s[n:].sum()) < 1e-12
    # per-subaperture raw slopes are not zero (asymmetric pupil images) ...
    assert np.abs(s).max() > 1e-3
    # ... but vanish once the flat-wavefront reference is subtracted
    assert np.all(slopes.pyr_slopes(det, NSUB, valid, ref=s) == 0.0)


def test_single_face_is_exact_shift():
    """A mask equal to the (+,+) face's linear phase everywhere moves the
    padded field by (+c, +c) pixels, circularly: pins the mask sign and the
    face -> quadrant assignment."""
    n, N, nmod = 8, 16, 1
    c = n // 2
    u = dft.centred_coords(N)
    face = np.exp(-2j * np.pi * c * (u[None, :] + u[:, None]) / N)
    full = pyramid.pyramid_mask(N, n)
    sel = (u[:, None] > 0) & (u[None, :] > 0)
    assert np.allclose(full[sel], face[sel], atol=1e-15)
    amp = np.ones((n, n))
    phi = _rand_phase(3, n)
    I = pyramid.pwfs_intensity(amp, phi, 2, nmod, 0.0, n, mask=face)
    P = np.zeros((N, N))
    P[4:12, 4:12] = 1.0
    assert np.allclose(I, np.roll(P, (c, c), axis=(0, 1)), atol=1e-12)


def test_unit_mask_is_identity(pupil):
    amp, _ = pupil
    N = 2 * NP
    I = pyramid.pwfs_intensity(amp, _rand_phase(4), 2, 6, 2.0, NP,
                               mask=np.ones((N, N)))
    P = np.zeros((N, N))
    P[NP // 2:NP // 2 + NP, NP // 2:NP // 2 + NP] = amp ** 2
    assert np.allclose(I, P, atol=1e-13)


def test_tilt_antisymmetry_and_sign(pupil):
    amp, valid = pupil
    x = dft.centred_coords(NP)
    flat = pyramid.pwfs_image(amp, np.zeros((NP, NP)), 2, 8, 3.0, NSUB, NP)
    ref = slopes.pyr_slopes(flat, NSUB, valid)
    n = len(valid)
    a = 0.4
    tilt = 2 * np.pi * a * x[None, :] / NP * np.ones((NP, 1))
    sp = slopes.pyr_slopes(pyramid.pwfs_image(amp, tilt, 2, 8, 3.0, NSUB, NP),
                           NSUB, valid, ref)
    sm = slopes.pyr_slopes(pyramid.pwfs_image(amp, -tilt, 2, 8, 3.0, NSUB, NP),
                           NSUB, valid, ref)
    assert sp[:n].mean() > 0.01            # +x tilt gives positive mean Sx
    assert abs(sp[:n].mean() + sm[:n].mean()) < 1e-12
    # pointwise: dSx(-a) at (y, x_sub) = -dSx(+a) at (y, n_sub-1-x_sub)
    gp = np.full(NSUB * NSUB, np.nan)
    gm = np.full(NSUB * NSUB, np.nan)
    gp[valid] = sp[:n]
    gm[valid] = sm[:n]
    gp = gp.reshape(NSUB, NSUB)
    gm = gm.reshape(NSUB, NSUB)
    ok = ~np.isnan(gp)
    assert np.allclose(gm[ok], -gp[:, ::-1][ok], atol=1e-12)


def test_transpose_symmetry(pupil):
    amp, valid = pupil
    phi = _rand_phase(7, scale=0.5)
    n = len(valid)

    def grid(v):
        g = np.zeros(NSUB * NSUB)
        g[valid] = v
        return g.reshape(NSUB, NSUB)

    s1 = slopes.pyr_slopes(pyramid.pwfs_image(amp, phi, 2, 8, 3.0, NSUB, NP),
                           NSUB, valid)
    s2 = slopes.pyr_slopes(pyramid.pwfs_image(amp, phi.T, 2, 8, 3.0, NSUB, NP),
                           NSUB, valid)
    assert np.allclose(grid(s1[n:]), grid(s2[:n]).T, atol=1e-12)
    assert np.allclose(grid(s1[:n]), grid(s2[n:]).T, atol=1e-12)


def test_pyr_slopes_hand_example():
    det = np.array([[1.0, 2.0], [3.0, 6.0]])   # Q3=1, Q4=2, Q2=3, Q1=6
    s = slopes.pyr_slopes(det, 1, np.array([0]))
    assert np.allclose(s, [((6 + 2) - (3 + 1)) / 12, ((6 + 3) - (1 + 2)) / 12])
