"""The C ABI without a GPU: the library builds, loads, exports every declared
symbol, validates arguments on the host, and its host-side integer geometry
is bit-exact against the oracle."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

import synth
from oracle import geometry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sp():
    from paper_2602_06688_gb300 import build
    build.build()
    import paper_2602_06688_gb300 as pkg
    pkg.lib()
    return pkg


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(specula_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(sp):
    names = _declared()
    assert len(names) >= 18
    lib = sp.lib()
    for n in names:
        assert hasattr(lib, n), n
    # and the Python binding carries the same names
    for n in names:
        assert hasattr(sp, n), n


def test_strerror_and_version(sp):
    for code in range(0, -8, -1):
        assert sp.specula_strerror(code)
    assert sp.specula_strerror(12345) == "unknown status"
    assert sp.specula_version() >= 100


@pytest.mark.parametrize("name", ["pwfs8m_tiny", "pwfs8m", "mwfs39m", "pwfs39m", "soul220",
                                  "andes400"])
def test_host_geometry_bit_exact(sp, name):
    w = synth.workload(name)
    for s in w.sensors:
        p = s.pupil
        d = sp.pupil_desc(p)
        ref = geometry.pupil_mask(p.n_pix, p.obsc_frac)
        assert np.array_equal(sp.specula_pupil_mask_host(d), ref)
        n_sub = s.pwfs.n_sub if s.kind == "pwfs" else s.sh.n_sub
        got = sp.specula_valid_subaps_host(d, n_sub)
        assert np.array_equal(got, geometry.valid_subaps(ref, n_sub))


@pytest.mark.parametrize("n_mod", [1, 3, 12, 16, 24, 48])
def test_mod_table_bit_exact(sp, n_mod):
    c, s = sp.specula_mod_table_host(n_mod)
    rc, rs = geometry.mod_angles(n_mod)
    assert np.array_equal(c, rc) and np.array_equal(s, rs)
    assert np.array_equal(c.astype(np.float32), rc.astype(np.float32))


@pytest.mark.parametrize("n,obsc,nm", [(32, 0.0, 20), (64, 0.11, 200)])
def test_host_modal_basis_matches_oracle(sp, n, obsc, nm):
    from oracle import modal
    got = sp.specula_modal_basis_host(sp.PupilDesc(n, 0.1, obsc), nm)
    ref = modal.modal_basis(n, obsc, nm)
    # float64 on both sides; high radial orders lose a few digits to the
    # alternating factorial sums
    assert np.max(np.abs(got - ref)) <= 1e-8 * np.abs(ref).max()


def test_host_validation_returns_codes(sp):
    lib = sp.lib()
    bad = sp.PupilDesc(0, 0.1, 0.0)
    buf = np.zeros(16, dtype=np.uint8)
    assert lib.specula_pupil_mask_host(C.byref(bad), buf.ctypes.data_as(C.c_void_p)) == sp.EINVAL
    good = sp.PupilDesc(4, 0.1, 0.0)
    assert lib.specula_pupil_mask_host(C.byref(good), None) == sp.EINVAL
    nv = C.c_int32()
    idx = np.zeros(16, dtype=np.int32)
    assert lib.specula_valid_subaps_host(C.byref(good), 5, idx.ctypes.data_as(C.c_void_p),
                                         C.byref(nv)) == sp.EINVAL    # n_sub > n_pix
    assert lib.specula_mod_table_host(0, None, None) == sp.EINVAL
    # per-frame calls reject a null context before touching the device
    pw = sp.PwfsDesc(2, 12, 16, 64, 3.0)
    pu = sp.PupilDesc(64, 0.125, 0.0)
    dummy = C.c_void_p(16)
    assert lib.specula_pwfs_image(None, C.byref(pu), C.byref(pw), dummy, dummy, 1, dummy,
                                  None) == sp.EINVAL
    assert lib.specula_pwfs_plan(None, C.byref(pu), C.byref(pw)) == sp.EINVAL
    assert lib.specula_slopes(None, None, dummy, None, 1, dummy, None) == sp.EINVAL
    assert lib.specula_recon(None, None, dummy, 1, dummy, None) == sp.EINVAL
    assert lib.specula_atmo_extract(None, 1, None, None, None, None, 0.0, None, dummy,
                                    None) == sp.EINVAL
    assert lib.specula_ctx_create(None, 0) == sp.EINVAL
    assert lib.specula_ctx_destroy(None) == sp.EINVAL


def test_pyr_image_index_host_matches_oracle(sp):
    """Host image maps for the SOUL geometry and, at pad 2 with touching
    images, the quadrant layout; refused where image corners fall between
    detector pixels."""
    from oracle import geometry
    pu = sp.PupilDesc(80, 0.1025, 0.11)
    m = sp.specula_pyr_image_index_host(pu, 3, 96, 40)
    v = geometry.valid_subaps(geometry.pupil_mask(80, 0.11).astype(np.uint8), 40)
    assert np.array_equal(m, geometry.pyr_image_index(v, 40, 3, 96, 80))
    pu2 = sp.PupilDesc(64, 0.1, 0.0)
    v2 = geometry.valid_subaps(geometry.pupil_mask(64, 0.0).astype(np.uint8), 16)
    assert np.array_equal(sp.specula_pyr_image_index_host(pu2, 2, 64, 16),
                          geometry.pyr_quadrant_index(v2, 16))
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_pyr_image_index_host(pu, 3, 97, 40)       # not a multiple of b = 2
    assert e.value.status == sp.EUNSUPPORTED
    # the paper's own SOUL numbers: 220 px pupil, 40 subapertures of 5.5 px,
    # images 264 grid px = 48 detector px apart on the 120 px detector
    pu3 = sp.PupilDesc(220, 8.2 / 220, 0.11)
    v3 = geometry.valid_subaps(geometry.pupil_mask(220, 0.11).astype(np.uint8), 40)
    assert np.array_equal(sp.specula_valid_subaps_host(pu3, 40), v3)
    m3 = sp.specula_pyr_image_index_host(pu3, 3, 264, 40)
    assert np.array_equal(m3, geometry.pyr_image_index(v3, 40, 3, 264, 220))
    assert m3.min() // 120 == 16 and m3.max() // 120 == 103
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_pyr_image_index_host(pu3, 3, 265, 40)     # 265 / 5.5 is not whole
    assert e.value.status == sp.EUNSUPPORTED
    # the ANDES reading: 400 px pupil at pad 4, 100 subapertures of 4 px,
    # images 480 grid px = 120 detector px apart on the 400 px detector
    pu4 = sp.PupilDesc(400, 39.0 / 400, 0.28)
    v4 = geometry.valid_subaps(geometry.pupil_mask(400, 0.28).astype(np.uint8), 100)
    m4 = sp.specula_pyr_image_index_host(pu4, 4, 480, 100)
    assert np.array_equal(m4, geometry.pyr_image_index(v4, 100, 4, 480, 400))
    assert m4.min() // 400 == 90 and m4.max() // 400 == 309   # 200 -+ 60 -+ 50


@pytest.mark.parametrize("n,n_sub,obsc", [(22, 4, 0.0), (33, 6, 0.3), (100, 7, 0.2), (63, 10, 0.11)])
def test_valid_subaps_host_fractional(sp, n, n_sub, obsc):
    """Fractional subaperture sides: the host rule is the oracle's, exactly."""
    from oracle import geometry
    got = sp.specula_valid_subaps_host(sp.PupilDesc(n, 0.1, obsc), n_sub)
    assert np.array_equal(got, geometry.valid_subaps(geometry.pupil_mask(n, obsc), n_sub))
