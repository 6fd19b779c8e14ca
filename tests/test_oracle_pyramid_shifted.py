"""Oracle pins: the shifted-mask form of the modulated pyramid.

Moving the pyramid mask by -s instead of tilting the field by +s gives the
same image wherever no frequency wraps (whole-bin shifts of a band-limited
field), reduces to the tilt form without modulation, and keeps the flux."""
import numpy as np

from oracle import dft, geometry, pyramid

NP = 32


def _pupil_field(seed, n=NP, obsc=0.2, scale=1.5):
    amp = geometry.pupil_mask(n, obsc).astype(np.float64)
    rng = np.random.default_rng(seed)
    return amp, scale * rng.standard_normal((n, n))


def _band_limited(N, margin, seed):
    """A padded field whose centred spectrum is zero within `margin` bins of
    the edge of the centred frequency range."""
    rng = np.random.default_rng(seed)
    u = dft.centred_coords(N)
    keep = np.abs(u) <= (N - 1) / 2.0 - margin
    F = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    F *= keep[:, None] & keep[None, :]
    return dft.centred_idft2(F)


def test_tilt_on_the_padded_grid_is_the_pupil_tilt():
    """s = r pad (cos, sin) bins on the N grid is the tilt of r cycles across
    the pupil: the padded-field form reproduces the pinned pupil form."""
    amp, phi = _pupil_field(1)
    pad, nmod, r = 2, 8, 2.7
    N = pad * NP
    P = np.zeros((N, N), complex)
    off = (N - NP) // 2
    P[off:off + NP, off:off + NP] = amp * np.exp(1j * phi)
    sx, sy = pyramid.shift_bins(nmod, r, pad)
    got = pyramid.tilted_intensity(P, sx, sy, NP)
    ref = pyramid.pwfs_intensity(amp, phi, pad, nmod, r, NP)
    assert np.max(np.abs(got - ref)) < 1e-12 * ref.max()


def test_whole_bin_shifts_of_a_band_limited_field_agree_exactly():
    """No wrapped frequency: moving the mask by -s equals tilting by +s (a
    sign error, a wrong |u + s| or a mask on the wrong axis fails this)."""
    N = 32
    P = _band_limited(N, margin=4, seed=2)
    sx = [2.0, -3.0, 0.0, 1.0, -1.0]
    sy = [-1.0, 2.0, 0.0, 3.0, -4.0]
    for pd in (N / 2, 10.0):
        a = pyramid.tilted_intensity(P, sx, sy, pd)
        b = pyramid.shifted_mask_intensity(P, sx, sy, pd)
        assert np.max(np.abs(a - b)) < 1e-12 * a.max()


def test_brute_force_shifted_mask_tiny():
    """One DFT, shifted masks, inverse DFTs, with the defining sums (N = 8)."""
    n, pad = 4, 2
    N = n * pad
    amp, phi = _pupil_field(3, n=n, obsc=0.0)
    P = np.zeros((N, N), complex)
    P[2:6, 2:6] = amp * np.exp(1j * phi)
    sx, sy = pyramid.shift_bins(3, 1.3, pad)
    F = dft.brute_centred_dft2(P)
    ref = np.zeros((N, N))
    u = dft.centred_coords(N)
    for a, b in zip(sx, sy):
        M = np.exp(-2j * np.pi * (n / 2.0) * (np.abs(u[:, None] + b) + np.abs(u[None, :] + a)) / N)
        ref += np.abs(dft.brute_centred_dft2(F * M, inverse=True)) ** 2
    got = pyramid.pwfs_intensity_shifted(amp, phi, pad, 3, 1.3, n)
    assert np.max(np.abs(got - ref / 3)) < 1e-12 * ref.max()


def test_no_modulation_reduces_to_the_tilt_form():
    amp, phi = _pupil_field(4)
    a = pyramid.pwfs_intensity(amp, phi, 2, 4, 0.0, NP)
    b = pyramid.pwfs_intensity_shifted(amp, phi, 2, 4, 0.0, NP)
    assert np.max(np.abs(a - b)) < 1e-12 * a.max()


def test_parseval_flux_shifted():
    amp, phi = _pupil_field(5, scale=2.0)
    I = pyramid.pwfs_intensity_shifted(amp, phi, 2, 8, 3.0, NP)
    assert abs(I.sum() - amp.sum()) < 1e-12 * amp.sum()


def test_flat_wavefront_mirror_symmetry_shifted():
    """A symmetric modulation set over a centro-symmetric pupil: four equal,
    mirrored pupil images, as in the tilt form."""
    amp, _ = _pupil_field(6)
    I = pyramid.pwfs_intensity_shifted(amp, np.zeros((NP, NP)), 2, 8, 3.0, NP)
    h = NP
    q = [I[h:, h:].sum(), I[h:, :h].sum(), I[:h, :h].sum(), I[:h, h:].sum()]
    assert np.allclose(q, amp.sum() / 4, rtol=1e-12)
    assert np.allclose(I, I[:, ::-1], atol=1e-13)
    assert np.allclose(I, I[::-1, :], atol=1e-13)


def test_polychromatic_image_pins():
    """One wavelength at the reference is the monochromatic image; the flux is
    the weighted pupil count; flat-wavefront images stay mirror-symmetric."""
    amp, phi = _pupil_field(8)
    mono = pyramid.pwfs_image(amp, phi, 2, 8, 2.5, 8, NP)
    one = pyramid.pwfs_image_poly(amp, phi, 2, 8, 2.5, 8, NP, [1.0], [1.0])
    assert np.array_equal(one, mono)
    r, w = [1.25, 1.0, 0.8], [0.2, 0.5, 0.3]
    det = pyramid.pwfs_image_poly(amp, phi, 2, 8, 2.5, 8, NP, r, w)
    assert abs(det.sum() - amp.sum() * sum(w)) < 1e-12 * amp.sum()
    flat = pyramid.pwfs_image_poly(amp, np.zeros_like(phi), 2, 8, 2.5, 8, NP, r, w)
    assert np.allclose(flat, flat[:, ::-1], atol=1e-13) and np.allclose(flat, flat[::-1], atol=1e-13)
    # a longer wavelength sees a smaller phase: ratio 0 would be a flat wavefront
    d0 = pyramid.pwfs_image_poly(amp, phi, 2, 8, 2.5, 8, NP, [1e-12], [1.0])
    ref = pyramid.pwfs_image(amp, np.zeros_like(phi), 2, 8, 2.5e-12, 8, NP)
    assert np.max(np.abs(d0 - ref)) < 1e-9
