"""Oracle pins: the pyramid with other paddings and image separations (the
SOUL example's geometry: 40-subaperture pupil images 48 detector pixels apart
on a 120 px detector) and the slope computer driven by image index maps."""
import numpy as np

from oracle import geometry, pyramid, slopes


def test_maps_reduce_to_quadrants_at_pad_2():
    n, nsub = 32, 8
    amp = geometry.pupil_mask(n, 0.2).astype(np.float64)
    valid = geometry.valid_subaps(amp.astype(np.uint8), nsub)
    assert np.array_equal(geometry.pyr_image_index(valid, nsub, 2, n, n),
                          geometry.pyr_quadrant_index(valid, nsub))
    rng = np.random.default_rng(1)
    det = pyramid.pwfs_image(amp, rng.standard_normal((n, n)), 2, 8, 3.0, nsub, n)
    maps = geometry.pyr_image_index(valid, nsub, 2, n, n)
    assert np.array_equal(slopes.pyr_slopes_maps(det, maps), slopes.pyr_slopes(det, nsub, valid))


def _soul_like(n=40, nsub=20, pad=3, pup_dist=48):
    """Half the SOUL example's sampling: 20 subapertures of 2 px, images 24
    detector pixels apart on a 60 px detector (pad 3)."""
    amp = geometry.pupil_mask(n, 0.12).astype(np.float64)
    valid = geometry.valid_subaps(amp.astype(np.uint8), nsub)
    return amp, valid, geometry.pyr_image_index(valid, nsub, pad, pup_dist, n)


def test_separated_images_flux_and_symmetry():
    """pad 3, images apart: all the light lands inside the four pupil
    footprints' neighbourhood, the flux is kept, a flat wavefront gives four
    mirrored images and zero mean slopes."""
    n, nsub, pad, pd = 40, 20, 3, 48
    amp, valid, maps = _soul_like(n, nsub, pad, pd)
    det = pyramid.pwfs_image(amp, np.zeros((n, n)), pad, 12, 3.0, nsub, pd)
    assert det.shape == (pad * nsub, pad * nsub)
    assert abs(det.sum() - amp.sum()) < 1e-12 * amp.sum()
    assert np.allclose(det, det[:, ::-1], atol=1e-13) and np.allclose(det, det[::-1], atol=1e-13)
    s = slopes.pyr_slopes_maps(det, maps)
    nv = len(valid)
    assert abs(s[:nv].sum()) < 1e-10 and abs(s[nv:].sum()) < 1e-10
    # the four images hold most of the flux (the rest is diffraction between them)
    assert det.ravel()[maps].sum() > 0.8 * det.sum()


def test_tilt_sign_on_separated_images():
    """+x tilt gives a positive mean x slope after the reference is removed."""
    n, nsub, pad, pd = 40, 20, 3, 48
    amp, valid, maps = _soul_like(n, nsub, pad, pd)
    x = np.arange(n) - (n - 1) / 2.0
    ref = slopes.pyr_slopes_maps(pyramid.pwfs_image(amp, np.zeros((n, n)), pad, 12, 3.0, nsub, pd),
                                 maps)
    tilt = np.broadcast_to(0.3 * 2 * np.pi * x[None, :] / n, (n, n))
    s = slopes.pyr_slopes_maps(pyramid.pwfs_image(amp, tilt, pad, 12, 3.0, nsub, pd), maps, ref)
    nv = len(valid)
    assert s[:nv].mean() > 0.01 and abs(s[nv:].mean()) < 1e-10


def _pins_for(n, nsub, pad, pd, obsc=0.28, mirror=True):
    amp = geometry.pupil_mask(n, obsc).astype(np.float64)
    valid = geometry.valid_subaps(amp.astype(np.uint8), nsub)
    maps = geometry.pyr_image_index(valid, nsub, pad, pd, n)
    flat = pyramid.pwfs_image(amp, np.zeros((n, n)), pad, 8, 3.0, nsub, pd)
    assert flat.shape == (pad * nsub, pad * nsub)
    assert abs(flat.sum() - amp.sum()) < 1e-12 * amp.sum()
    assert np.allclose(flat, flat.T, atol=1e-13)            # x and y play the same part
    nv = len(valid)
    s = slopes.pyr_slopes_maps(flat, maps)
    if mirror:
        assert np.allclose(flat, flat[:, ::-1], atol=1e-13) and np.allclose(flat, flat[::-1], atol=1e-13)
        assert abs(s[:nv].sum()) < 1e-10 and abs(s[nv:].sum()) < 1e-10
    x = np.arange(n) - (n - 1) / 2.0
    tilt = np.broadcast_to(0.3 * 2 * np.pi * x[None, :] / n, (n, n))
    st = slopes.pyr_slopes_maps(pyramid.pwfs_image(amp, tilt, pad, 8, 3.0, nsub, pd), maps, s)
    assert st[:nv].mean() > 0.01 and abs(st[nv:].mean()) < 1e-3 * st[:nv].mean()
    return flat


def test_andes_like_geometry():
    """The ANDES reading scaled down: pad 4 (oversampling 4), 4 px
    subapertures, images 1.2 pupil diameters apart: flux kept, four mirrored
    images and zero mean slopes for a flat wavefront, +x tilt -> +x slopes."""
    _pins_for(40, 10, 4, 48)


def test_odd_pupil_side():
    """An odd pupil side (33 px at pad 4) sits at offset floor((N - n)/2), so
    its centre is half a grid pixel off the grid's: the flat-wavefront
    images keep the flux and the x <-> y symmetry but are not mirror
    images (that offset shows as a constant slope, which the reference
    removes); the tilt sign holds."""
    flat = _pins_for(33, 11, 4, 51, mirror=False)
    assert np.abs(flat - flat[:, ::-1]).max() > 1e-3 * flat.max()


def _valid_supersampled(mask, n_sub):
    """Brute force: split every pupil pixel into n_sub x n_sub sub-pixels of
    side 1 / n_sub; sub-pixel k (in those units) belongs to subaperture
    k // n_pix along each axis.  Valid iff at least half the subaperture's
    sub-pixels (n_pix^2 of them) lie in the stop."""
    n = mask.shape[0]
    fine = np.kron(mask.astype(np.int64), np.ones((n_sub, n_sub), dtype=np.int64))
    counts = fine.reshape(n_sub, n, n_sub, n).sum(axis=(1, 3))
    return np.flatnonzero((2 * counts >= n * n).ravel()).astype(np.int32)


def test_valid_subaps_fractional_against_supersampling():
    for n, nsub, obsc in ((22, 4, 0.2), (33, 6, 0.3), (220, 40, 0.12), (32, 8, 0.2), (25, 10, 0.0)):
        m = geometry.pupil_mask(n, obsc)
        assert np.array_equal(geometry.valid_subaps(m, nsub), _valid_supersampled(m, nsub)), (n, nsub)


def test_fractional_detector_soul_scaled():
    """The SOUL example's ratios at a tenth of the size: a 22 px pupil of 4
    subapertures (5.5 px each, as 220 / 40), pad 3 (66 grid), images
    6 detector pixels apart on a 12 px detector (48 / 40 x 5), so each
    detector pixel integrates 5.5 x 5.5 grid pixels.  The flux is kept, a
    flat wavefront gives mirror-symmetric images that hold most of the light
    on their mapped pixels and zero mean slopes."""
    n, nsub, pad, pd = 22, 4, 3, 33
    amp = geometry.pupil_mask(n, 0.0).astype(np.float64)
    valid = geometry.valid_subaps(amp.astype(np.uint8), nsub)
    maps = geometry.pyr_image_index(valid, nsub, pad, pd, n)
    # corners: 12 / 2 +- 3 - 2 = 1 and 7
    assert set(np.unique(maps // 12)) <= set(range(1, 5)) | set(range(7, 11))
    det = pyramid.pwfs_image(amp, np.zeros((n, n)), pad, 8, 2.0, nsub, pd)
    assert det.shape == (12, 12)
    assert abs(det.sum() - amp.sum()) < 1e-12 * amp.sum()
    assert np.allclose(det, det[:, ::-1], atol=1e-12) and np.allclose(det, det[::-1], atol=1e-12)
    assert det.ravel()[maps].sum() > 0.7 * det.sum()
    s = slopes.pyr_slopes_maps(det, maps)
    nv = len(valid)
    assert abs(s[:nv].sum()) < 1e-10 and abs(s[nv:].sum()) < 1e-10
    # the detector is the area-weighted rebinning of the grid intensity
    I = pyramid.pwfs_intensity(amp, np.zeros((n, n)), pad, 8, 2.0, pd)
    assert np.allclose(det, pyramid.rebin_area(I, 12), rtol=0, atol=1e-12)
