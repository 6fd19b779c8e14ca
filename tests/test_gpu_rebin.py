"""GPU parity of the area-weighted detector rebinning against the oracle.

Tolerance: an output pixel sums at most (ceil(b) + 1)^2 products of exact
integer weights and float32 inputs in float32, so |out - ref| <=
2 (n_terms + 2) eps_32 rebin(|img|) element-wise (rebin(|img|) is the sum of
the absolute terms)."""
import math

import numpy as np
import pytest

from gpu_common import close_checked, load_pkg, need_gpu
from oracle import pyramid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


@pytest.mark.parametrize("n_in,n_out,nb", [(960, 400, 1), (240, 100, 3), (30, 7, 2), (5, 3, 1),
                                          (24, 12, 2), (16, 40, 1), (1, 1, 1), (2048, 2047, 1)])
def test_rebin_matches_the_oracle(env, n_in, n_out, nb):
    torch, sp, ctx = env
    rng = np.random.default_rng(n_in * 7 + n_out)
    img = rng.random((nb, n_in, n_in)).astype(np.float32)
    out = torch.full((nb, n_out, n_out), float("nan"), device="cuda")
    sp.specula_rebin(ctx, torch.tensor(img, device="cuda"), n_out, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    terms = (math.ceil(n_in / n_out) + 1) ** 2
    for k in range(nb):
        ref = pyramid.rebin_area(img[k].astype(np.float64), n_out)
        bound = 2 * (terms + 2) * 2.0 ** -24 * pyramid.rebin_area(np.abs(img[k]).astype(np.float64), n_out)
        assert np.all(np.abs(got[k] - ref) <= bound + 1e-30)
        if n_in % n_out == 0:
            assert np.allclose(got[k], pyramid.bin_image(img[k].astype(np.float64), n_in // n_out),
                               rtol=1e-5, atol=0)


def test_rebin_arguments(env):
    torch, sp, ctx = env
    lib = sp.lib()
    import ctypes as C
    x = torch.zeros(4, 4, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = C.c_void_p(x.data_ptr())
    assert lib.specula_rebin(ctx.handle, p, 4, 2, 0, p, st) == sp.OK      # empty batch
    for n_in, n_out in ((0, 2), (4, 0), (4097, 2), (4, 4097)):
        assert lib.specula_rebin(ctx.handle, p, n_in, n_out, 1, p, st) == sp.EINVAL
