"""The learned reconstructor gains over the linear MVM on held-out frames.

Training pairs come from the GPU simulator (independent Kolmogorov screens,
r0 uniform in 0.06-0.20 m, the 8 m pyramid geometry); the network is trained
on the GPU by the library's own forward/backward kernels; the linear
reconstructor is the calibrated push-pull pseudo-inverse.  Reduced sample
count and model width for test time; bench.py runs the full configuration.
"""
import numpy as np
import pytest

import synth
from gpu_common import close_checked, load_pkg, need_gpu
from oracle import modal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pipe():
    torch = need_gpu()
    sp = load_pkg()
    from paper_2602_06688_gb300.learned import LearnedPipeline
    ctx = sp.Context(0)
    wl = synth.workload("learned8m")
    p = LearnedPipeline(ctx, wl, n_modes=200, hidden=(512, 512))
    yield torch, sp, ctx, p
    close_checked(sp, ctx)


def test_labels_are_modal_projections(pipe):
    torch, sp, ctx, p = pipe
    X, T = p.make_pairs(4, sample0=10 ** 6)
    # recompute the projection of the same phases in float64 from the oracle's basis
    n = p.n
    ph = torch.empty(4, n, n, device="cuda")
    scr = torch.empty(4, p.side, p.side, device="cuda")
    r0 = synth.uniform_draws(p.seed * 1000003 + 10 ** 6, 4, 0.06, 0.20)
    scale = torch.tensor((r0 ** (-5 / 6) * 500.0 / p.lam).astype(np.float32), device="cuda")
    sp.specula_screen_generate_batch(ctx, 4, p.side, p.pupil.pitch_m, 1.0, p.L0, p.seed, 10 ** 6, scr)
    sp.specula_random_phase(ctx, scr, 4, p.side, n, scale, ph)
    torch.cuda.synchronize()
    B = modal.modal_basis(n, p.sensor.pupil.obsc_frac, p.n_modes)
    mask = (B[0] != 0) | (modal.modal_basis(n, p.sensor.pupil.obsc_frac, 2)[1] != 0)
    from oracle import geometry
    mask = geometry.pupil_mask(n, p.sensor.pupil.obsc_frac)
    ref = modal.project(B, ph.cpu().numpy().astype(np.float64), mask)
    got = T.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.abs(ref).max()


def test_learned_beats_linear(pipe):
    torch, sp, ctx, p = pipe
    Xtr, Ttr = p.make_pairs(24000, sample0=0)
    Xte, Tte = p.make_pairs(2000, sample0=10 ** 6 + 100)
    hist = p.fit(Xtr, Ttr, epochs=8, batch=256, lr=1e-3)
    assert hist[-1] < hist[0]
    res = p.evaluate(Xte, Tte)
    # the network must reduce the modal residual of the linear reconstructor
    assert res["learned"] < 0.8 * res["linear"], res
    # the split-bf16 copy of R (tensor cores at this batch) leaves the same
    # residual as float32 R on the CUDA cores
    assert abs(res["linear_split_bf16"] - res["linear"]) <= 1e-4 * res["linear"], res
    a = p.linear(Xte).double()
    b = p.linear(Xte, split_bf16=True).double()
    assert float((a - b).norm() / a.norm()) <= 1e-4
