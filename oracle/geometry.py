"""Integer geometry of the sensors: pupil stop, valid subapertures, index maps,
and the modulation-point angle table.

Follows the data objects PupilStop, PupData and SubapData (App. A, Tab. 3) and
the calibrators PyrPupdataCalibrator / ShSubapCalibrator (App. A, Tab. 4).  The
paper selects valid pupil pixels with a flux threshold on a calibration image
(App. B, Listing 2, the ``th0.30`` tag of ``pupdata_object``); the calibration
data are not public, so this oracle uses the geometric reading below, which is
exact in integers.
"""
import math

import numpy as np


def pupil_mask(n_pix: int, obsc_frac: float) -> np.ndarray:
    """Circular pupil stop with a central obscuration, (n_pix, n_pix) uint8.

    Pixel (j, i) (row j, column i) has doubled centred coordinates
    (2i - n + 1, 2j - n + 1); it is inside iff
        r4 = (2i - n + 1)^2 + (2j - n + 1)^2 <= n^2   and   r4 > (obsc * n)^2.
    r4 and n^2 are integers; the obscuration bound is the float64 product
    e * e with e = obsc * n.
    """
    n = int(n_pix)
    idx = 2 * np.arange(n, dtype=np.int64) - n + 1
    r4 = idx[None, :] ** 2 + idx[:, None] ** 2
    e = float(obsc_frac) * n
    thr = e * e
    inside = (r4 <= n * n) & (r4.astype(np.float64) > thr)
    return inside.astype(np.uint8)


def valid_subaps(mask: np.ndarray, n_sub: int) -> np.ndarray:
    """Valid subapertures of an n_sub x n_sub grid over the pupil stop.

    A subaperture covers b x b pupil pixels, b = n_pix / n_sub (whole or
    fractional: the subaperture lattice tiles the pupil grid).  It is valid
    iff at least half of its area is inside the stop.  With ov(i, A) the
    overlap of pixel i with subaperture A in units of 1 / n_sub (an integer),
    the condition is 2 sum ov(y, A) ov(x, C) mask[y, x] >= n_pix^2, exact in
    integers; for a whole b it is 2 * count >= b^2.  Returns int32 linear
    indices a * n_sub + b_col in row-major (row a first) order.
    """
    n = mask.shape[0]
    i = np.arange(n)[None, :]
    A = np.arange(n_sub)[:, None]
    ov = np.maximum(np.minimum((i + 1) * n_sub, (A + 1) * n)
                    - np.maximum(i * n_sub, A * n), 0).astype(np.int64)
    counts = ov @ mask.astype(np.int64) @ ov.T
    ok = 2 * counts >= n * n
    return np.flatnonzero(ok.ravel()).astype(np.int32)


def pyr_quadrant_index(valid: np.ndarray, n_sub: int) -> np.ndarray:
    """Detector linear indices of the four pupil images of each subaperture.

    The detector is 2 n_sub x 2 n_sub (row = y).  The pyramid face (+x, +y)
    images the pupil into the quadrant of larger row and column indices, and
    so on; subaperture (a, b) lands at the same (a, b) inside each quadrant:
        Q1 (+x,+y): (n_sub + a, n_sub + b)    Q2 (-x,+y): (n_sub + a, b)
        Q3 (-x,-y): (a, b)                     Q4 (+x,-y): (a, n_sub + b)
    Returns int32 (4, n_valid): rows Q1..Q4.
    """
    a = valid // n_sub
    bb = valid % n_sub
    w = 2 * n_sub
    q1 = (n_sub + a) * w + (n_sub + bb)
    q2 = (n_sub + a) * w + bb
    q3 = a * w + bb
    q4 = a * w + (n_sub + bb)
    return np.stack([q1, q2, q3, q4]).astype(np.int32)


def mod_angles(n_mod: int):
    """Modulation points: theta_m = (2 pi m) / n_mod, m = 0..n_mod-1, counter-
    clockwise from +x (ModulatedPyramid ``mod_amp``, App. B, Listing 2).

    Returns float64 arrays (cos theta_m, sin theta_m), each from the C
    library's cos/sin on the same float64 argument ((2 * pi) * m) / n_mod.
    """
    c = np.empty(n_mod)
    s = np.empty(n_mod)
    for m in range(n_mod):
        th = 2.0 * math.pi * m / n_mod
        c[m] = math.cos(th)
        s[m] = math.sin(th)
    return c, s


def pyr_image_index(valid: np.ndarray, n_sub: int, pad: int, pup_dist: int,
                    n_pix: int) -> np.ndarray:
    """Detector linear indices of the four pupil images of each subaperture
    for any padding and image separation (the SOUL example's ``pup_diam`` /
    ``pup_dist`` / ``output_resolution``, App. B, Listing 2).

    The padded grid (pad n_pix) is sampled onto an n_det = pad n_sub
    detector whose pixel is b = n_pix / n_sub grid pixels (whole: b x b
    binning; fractional: area-weighted rebinning).  The four images, n_sub
    detector pixels wide, are centred d = pup_dist / (2 b) detector pixels
    from the detector centre along +-x and +-y (face (+x, +y) to larger row
    and column); subaperture (a, c) of image Q sits at row r0_Q + a, column
    c0_Q + c with
        r0 = n_det / 2 + sy d - n_sub / 2,  c0 = n_det / 2 + sx d - n_sub / 2,
    (sx, sy) = (+,+) Q1, (-,+) Q2, (-,-) Q3, (+,-) Q4.  Needs integer image
    corners (2 d = pup_dist n_sub / n_pix an integer and 2 d - n_sub even),
    so each image's subapertures fall on whole detector pixels; returns a
    (4, n_valid) int64 array.  With pad 2 and pup_dist = n_pix it is
    ``pyr_quadrant_index``.
    """
    assert (pup_dist * n_sub) % n_pix == 0
    n_det = pad * n_sub
    two_d = pup_dist * n_sub // n_pix
    assert (two_d - n_sub) % 2 == 0 and n_det % 2 == 0
    a = valid // n_sub
    c = valid % n_sub
    out = []
    for sx, sy in ((1, 1), (-1, 1), (-1, -1), (1, -1)):
        r0 = (n_det + sy * two_d - n_sub) // 2
        c0 = (n_det + sx * two_d - n_sub) // 2
        assert 0 <= r0 and r0 + n_sub <= n_det and 0 <= c0 and c0 + n_sub <= n_det
        out.append((r0 + a).astype(np.int64) * n_det + (c0 + c))
    return np.stack(out)
