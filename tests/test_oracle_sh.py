"""Oracle pins: Shack-Hartmann spots and centre-of-gravity slopes."""
import numpy as np

from oracle import dft, geometry, recon, sh, slopes

NSUB, S, N = 6, 6, 12
NP = NSUB * S


def _pupil():
    amp = geometry.pupil_mask(NP, 0.25).astype(np.float64)
    return amp, geometry.valid_subaps(amp.astype(np.uint8), NSUB)


def test_brute_force_spot():
    amp = np.ones((S, S))
    phi = np.random.default_rng(1).standard_normal((S, S))
    got = sh.sh_spots(amp, phi, 1, S, N, np.array([0]))[0]
    P = np.zeros((N, N), complex)
    P[3:9, 3:9] = np.exp(1j * phi)
    ref = np.abs(dft.brute_centred_dft2(P)) ** 2 / N ** 2
    assert np.max(np.abs(got - ref)) < 1e-12 * ref.max()


def test_flat_wavefront_zero_centroid_and_parseval():
    amp, valid = _pupil()
    sp = sh.sh_spots(amp, np.zeros((NP, NP)), NSUB, S, N, valid)
    s = slopes.sh_slopes(sp)
    assert np.max(np.abs(s)) < 1e-12
    for k, idx in enumerate(valid):
        a, b = divmod(int(idx), NSUB)
        flux = amp[a * S:(a + 1) * S, b * S:(b + 1) * S].sum()
        assert abs(sp[k].sum() - flux) < 1e-12 * flux


def test_integer_tilt_is_exact_roll():
    """A tilt of k lambda/d across a subaperture (k cycles over s px) moves the
    spot by exactly 2k px circularly on the n = 2s grid."""
    amp, valid = _pupil()
    x = dft.centred_coords(NP)
    rng = np.random.default_rng(2)
    phi = 0.3 * rng.standard_normal((NP, NP))
    base = sh.sh_spots(amp, phi, NSUB, S, N, valid)
    for kx, ky in [(1, 0), (0, -1), (2, 1)]:
        tilt = 2 * np.pi * (kx * x[None, :] + ky * x[:, None]) / S
        moved = sh.sh_spots(amp, phi + tilt, NSUB, S, N, valid)
        ref = np.roll(base, (2 * ky, 2 * kx), axis=(1, 2))
        assert np.max(np.abs(moved - ref)) < 1e-12 * base.max()


def test_cog_hand_example():
    spot = np.zeros((1, 4, 4))
    spot[0, 3, 1] = 2.0          # row 3 (y = +1.5), column 1 (x = -0.5)
    spot[0, 0, 0] = 2.0          # row 0 (y = -1.5), column 0 (x = -1.5)
    s = slopes.sh_slopes(spot)
    assert np.allclose(s, [(-0.5 - 1.5) / 2, (1.5 - 1.5) / 2])


def test_mvm_direct_sum():
    rng = np.random.default_rng(3)
    R = rng.standard_normal((5, 7))
    s = rng.standard_normal(7)
    ref = [sum(R[i, j] * s[j] for j in range(7)) for i in range(5)]
    assert np.allclose(recon.mvm(R, s), ref, atol=1e-13)
    sb = rng.standard_normal((3, 7))
    assert np.allclose(recon.mvm(R, sb)[1], recon.mvm(R, sb[1]), atol=1e-13)
