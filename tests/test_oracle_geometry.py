"""Oracle pins: centred DFT and the integer sensor geometry (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import dft, geometry

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "geometry_counts.json")


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 8])
def test_centred_dft_matches_brute_force(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    ref = dft.brute_centred_dft2(a)
    got = dft.centred_dft2(a)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    inv = dft.centred_idft2(a)
    ref_inv = dft.brute_centred_dft2(a, inverse=True)
    assert np.max(np.abs(inv - ref_inv)) <= 1e-12 * np.max(np.abs(ref_inv))


def test_centred_dft_of_real_symmetric_is_real():
    # centred grid: a real field symmetric under x -> -x has a real spectrum
    n = 10
    x = dft.centred_coords(n)
    a = np.exp(-(x[None, :] ** 2 + x[:, None] ** 2) / 7.0)
    f = dft.centred_dft2(a)
    assert np.max(np.abs(f.imag)) < 1e-12 * np.max(np.abs(f))
    assert np.allclose(dft.centred_idft2(f), a, atol=1e-13)


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"])
def test_pupil_and_subaps_hand_counts(case):
    m = geometry.pupil_mask(case["n_pix"], case["obsc"])
    assert int(m.sum()) == case["pixels"]
    v = geometry.valid_subaps(m, case["n_sub"])
    assert len(v) == case["valid"]


def test_pupil_corner_blocks_invalid_8px():
    m = geometry.pupil_mask(8, 0.0)
    v = geometry.valid_subaps(m, 4)
    assert set(v.tolist()) == set(range(16)) - {0, 3, 12, 15}


@pytest.mark.parametrize("n,eps,nsub", [(64, 0.0, 16), (160, 0.11, 40),
                                        (480, 0.28, 96), (816, 0.28, 68),
                                        (120, 0.28, 40)])
def test_pupil_symmetries(n, eps, nsub):
    m = geometry.pupil_mask(n, eps)
    assert np.array_equal(m, m[::-1, :])
    assert np.array_equal(m, m[:, ::-1])
    assert np.array_equal(m, m.T)
    # area within the discretisation of the annulus area
    area = math.pi / 4 * n * n * (1 - eps * eps)
    assert abs(m.sum() - area) < 4 * n
    v = geometry.valid_subaps(m, nsub)
    grid = np.zeros(nsub * nsub, dtype=bool)
    grid[v] = True
    grid = grid.reshape(nsub, nsub)
    assert np.array_equal(grid, grid[::-1, :]) and np.array_equal(grid, grid.T)


def test_quadrant_index_map_tiny():
    q = geometry.pyr_quadrant_index(np.array([0, 1, 2, 3], dtype=np.int32), 2)
    # detector 4x4; subap (a,b) -> Q1 (2+a, 2+b), Q2 (2+a, b), Q3 (a, b), Q4 (a, 2+b)
    assert q[0].tolist() == [10, 11, 14, 15]
    assert q[1].tolist() == [8, 9, 12, 13]
    assert q[2].tolist() == [0, 1, 4, 5]
    assert q[3].tolist() == [2, 3, 6, 7]


def test_mod_angles():
    c, s = geometry.mod_angles(4)
    assert np.allclose(c, [1, 0, -1, 0], atol=1e-15)
    assert np.allclose(s, [0, 1, 0, -1], atol=1e-15)   # counter-clockwise
    c, s = geometry.mod_angles(48)
    assert np.allclose(c * c + s * s, 1.0, atol=1e-15)
    assert abs(c.sum()) < 1e-13 and abs(s.sum()) < 1e-13
