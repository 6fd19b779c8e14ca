"""The allocation-free extraction entry point against the context-based one.

specula_atmo_extract_noalloc exists for callers that cannot allocate device
memory (hosts that only enqueue into their own graphs, real-time loops with
a fixed memory budget, embeddings that own all device memory).  It must give
the same phases as specula_atmo_extract, call after call, while its fixed
device array is reused.  This file is collected last on purpose.
"""
import ctypes as C
from types import SimpleNamespace as NS

import numpy as np
import pytest

from gpu_common import load_pkg, need_gpu

pytestmark = pytest.mark.gpu


def _case():
    rng = np.random.default_rng(11)
    layers = [NS(side=256, pitch_m=0.1, height_m=float(h), vx_mps=float(rng.uniform(-15, 15)),
                 vy_mps=float(rng.uniform(-15, 15))) for h in (0.0, 4e3, 9e3, 15e3)]
    src = NS(theta_x_rad=3e-5, theta_y_rad=-2e-5, height_m=90e3, wavelength_nm=589.0)
    screens = [rng.standard_normal((256, 256)).astype(np.float32) * 2.0 for _ in layers]
    return layers, src, screens, 160, 0.0525


def test_noalloc_matches_context_extraction_twice():
    torch = need_gpu()
    sp = load_pkg()
    layers, src, screens, n, pitch = _case()
    scr = [torch.tensor(s, device="cuda") for s in screens]
    L = [sp.layer_desc(l) for l in layers]
    pu = sp.PupilDesc(n, pitch, 0.0)
    with sp.Context(0) as ctx:
        for t in (0.0125, 0.3):          # two calls in a row reuse the fixed array
            ref = torch.empty(n, n, device="cuda")
            got = torch.full((n, n), float("nan"), device="cuda")
            sp.specula_atmo_extract(ctx, L, scr, sp.source_desc(src), pu, t, ref)
            sp.specula_atmo_extract_noalloc(L, scr, sp.source_desc(src), pu, t, got)
            torch.cuda.synchronize()
            # the extraction tolerance of the parity tests (4 ulp of the largest
            # screen value per layer); the two paths run the same kernels, so the
            # results are in fact identical
            tol = (500.0 / src.wavelength_nm) * sum(np.abs(s).max() for s in screens) * 4 * 2.0 ** -24
            diff = (got - ref).abs().max().item()
            assert diff <= tol
            assert torch.equal(got, ref)


def test_noalloc_rejects_sizes_beyond_its_array():
    """Sizes beyond the fixed array are refused before any launch; the calls
    get real buffers of the requested sizes, so a regression in the checks
    would fail the assertions (the output would change) rather than touch
    memory outside them."""
    torch = need_gpu()
    sp = load_pkg()
    lib = sp.lib()
    layers, src, screens, n, pitch = _case()
    scr = torch.tensor(screens[0], device="cuda")               # 256 x 256, as described
    L1 = (sp.LayerDesc * 1)(sp.layer_desc(layers[0]))
    ptr = (C.c_void_p * 1)(C.c_void_p(scr.data_ptr()))
    wide = 8193
    out = torch.full((wide, wide), 7.0, device="cuda")
    st = lib.specula_atmo_extract_noalloc(1, L1, ptr, C.byref(sp.source_desc(src)),
                                          C.byref(sp.PupilDesc(wide, 0.01, 0.0)), 0.0, None,
                                          C.c_void_p(out.data_ptr()), None)
    torch.cuda.synchronize()
    assert st == sp.EUNSUPPORTED
    assert bool((out == 7.0).all())
    del out
    many = (sp.LayerDesc * 65)(*([sp.layer_desc(layers[0])] * 65))
    ptrs = (C.c_void_p * 65)(*([C.c_void_p(scr.data_ptr())] * 65))
    out = torch.full((n, n), 7.0, device="cuda")
    st = lib.specula_atmo_extract_noalloc(65, many, ptrs, C.byref(sp.source_desc(src)),
                                          C.byref(sp.PupilDesc(n, pitch, 0.0)), 0.0, None,
                                          C.c_void_p(out.data_ptr()), None)
    torch.cuda.synchronize()
    assert st == sp.EUNSUPPORTED
    assert bool((out == 7.0).all())
