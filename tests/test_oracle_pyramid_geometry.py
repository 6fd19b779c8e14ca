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
