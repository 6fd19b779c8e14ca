"""GPU parity of the infinite phase screens against the FP64 oracle.

Tolerances:
* operators (float64 on both sides, GPU Jacobi vs LAPACK): the stencil
  covariance has condition numbers up to ~4e5 here, so A and B agree to
  1e-7 of their largest entry (float64 eigenvector error ~ kappa 1e-15);
  the float32 copies equal the float64 ones rounded once;
* one line (float32 dot products of m + side terms, strided lanes then a
  butterfly): |Z_gpu - Z| <= 2 (m + side) eps_32 (sum|A||X| + b_scale
  sum|B||b|) element-wise, against the oracle fed the GPU's float32
  operators and the same screen;
* in-kernel noise: the kernel evaluates the Box-Muller transform in float32
  (uniform rounded once, logf, sincospif: a few ulp), the oracle in float64;
  near u -> 1 the radius sqrt(-2 ln u) turns an absolute error of ~1e-7 in
  -2 ln u into up to ~4e-4, so the bound adds sum|B| (4e-4 + 1e-6 |b|);
* a grown sequence compounds that per-line error through the recursion;
  the check uses 1e-4 of the screen RMS after 60 lines.
"""
import numpy as np
import pytest

from gpu_common import close_checked, load_pkg, need_gpu
from oracle import atmo
from oracle import infinite as oinf

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    sp = load_pkg()
    ctx = sp.Context(0)
    yield torch, sp, ctx
    close_checked(sp, ctx)


def _np(t):
    return t.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("side,n_st,pitch,r0,L0", [(32, 2, 0.05, 0.15, 25.0),
                                                   (24, 3, 0.1, 0.1, 10.0),
                                                   (7, 1, 0.2, 0.2, 30.0)])
def test_operators_match_the_oracle(env, side, n_st, pitch, r0, L0):
    torch, sp, ctx = env
    A, B, A64, B64 = sp.specula_infscreen_operators(ctx, side, n_st, pitch, r0, L0,
                                                    want_f64=True)
    torch.cuda.synchronize()
    Ao, Bo = oinf.line_operators(side, n_st, pitch, r0, L0)
    assert np.max(np.abs(_np(A64) - Ao)) <= 1e-7 * np.abs(Ao).max()
    assert np.max(np.abs(_np(B64) - Bo)) <= 1e-7 * np.abs(Bo).max()
    assert np.array_equal(A.cpu().numpy(), A64.cpu().numpy().astype(np.float32))
    assert np.array_equal(B.cpu().numpy(), B64.cpu().numpy().astype(np.float32))


def _line_bound(A, B, X, b, bs, m, side):
    return 2 * (m + side) * EPS32 * (np.abs(A) @ np.abs(X) + bs * (np.abs(B) @ np.abs(b))) + 1e-30


@pytest.fixture(scope="module")
def ops(env):
    torch, sp, ctx = env
    side, n_st = 32, 2
    A, B = sp.specula_infscreen_operators(ctx, side, n_st, 0.05, 0.15, 25.0)
    return side, n_st, A, B


def test_one_line_per_task_with_given_noise(env, ops):
    """Three rings at once: a row upwards, a row downwards and a column;
    negative and wrapped line indices; other lines untouched."""
    torch, sp, ctx = env
    side, n_st, A, B = ops
    rng = np.random.default_rng(5)
    scr0 = [(rng.standard_normal((side, side)) * 20).astype(np.float32) for _ in range(3)]
    scr = [torch.tensor(x, device="cuda") for x in scr0]
    noise = rng.standard_normal((3, side)).astype(np.float32)
    spec = [(0, +1, 45, 1.0), (0, -1, -3, 0.7), (1, +1, 31, 1.3)]
    tasks = [(scr[i], A, B, bs, ax, d, i, L) for i, (ax, d, L, bs) in enumerate(spec)]
    sp.specula_infscreen_lines(ctx, side, n_st, tasks, noise=torch.tensor(noise, device="cuda"))
    torch.cuda.synchronize()
    A64, B64 = _np(A), _np(B)
    for i, (ax, d, L, bs) in enumerate(spec):
        ref = scr0[i].astype(np.float64)
        X = np.concatenate([oinf.get_line(ref, ax, L - d * k) for k in range(1, n_st + 1)])
        oinf.add_line(ref, A64, B64, ax, d, L, noise[i].astype(np.float64), bs)
        got = _np(scr[i])
        slot = L % side
        line_got = got[slot] if ax == 0 else got[:, slot]
        line_ref = ref[slot] if ax == 0 else ref[:, slot]
        bound = _line_bound(A64, B64, X, noise[i].astype(np.float64), bs, side * n_st, side)
        assert np.all(np.abs(line_got - line_ref) <= bound)
        mask = np.ones((side, side), bool)
        if ax == 0:
            mask[slot] = False
        else:
            mask[:, slot] = False
        assert np.array_equal(got[mask], scr0[i].astype(np.float64)[mask])


def test_philox_noise_lines(env, ops):
    """In-kernel noise: the oracle's Philox line noise gives the same line."""
    torch, sp, ctx = env
    side, n_st, A, B = ops
    rng = np.random.default_rng(6)
    scr0 = (rng.standard_normal((side, side)) * 20).astype(np.float32)
    scr = torch.tensor(scr0, device="cuda")
    L, seed, sid = -(1 << 33) - 5, 0x1234567890ABCDEF, 3
    sp.specula_infscreen_lines(ctx, side, n_st, [(scr, A, B, 1.0, 0, -1, sid, L)], seed=seed)
    torch.cuda.synchronize()
    A64, B64 = _np(A), _np(B)
    b = oinf.line_noise(seed, sid, L, side).astype(np.float32).astype(np.float64)
    ref = scr0.astype(np.float64)
    X = np.concatenate([oinf.get_line(ref, 0, L + k) for k in range(1, n_st + 1)])
    oinf.add_line(ref, A64, B64, 0, -1, L, b)
    slot = L % side
    bound = _line_bound(A64, B64, X, b, 1.0, side * n_st, side) \
        + np.abs(B64) @ (4e-4 + 1e-6 * np.abs(b))
    assert np.all(np.abs(_np(scr)[slot] - ref[slot]) <= bound)


def test_grown_sequence_matches_the_oracle(env, ops):
    """60 lines on one ring, rows and columns in both directions, one call per
    line, against the oracle run from the same start with the GPU's float32
    operators and the Philox noise."""
    torch, sp, ctx = env
    side, n_st, A, B = ops
    rng = np.random.default_rng(7)
    scr0 = (rng.standard_normal((side, side)) * 20).astype(np.float32)
    scr = torch.tensor(scr0, device="cuda")
    ref = scr0.astype(np.float64)
    A64, B64 = _np(A), _np(B)
    lo = {0: 0, 1: 0}
    seq = []
    for k in range(60):
        ax = k % 2
        d = -1 if (k // 7) % 2 else 1
        if d == 1:
            L = lo[ax] + side
            lo[ax] += 1
        else:
            lo[ax] -= 1
            L = lo[ax]
        seq.append((ax, d, L))
    for ax, d, L in seq:
        sp.specula_infscreen_lines(ctx, side, n_st, [(scr, A, B, 0.9, ax, d, 5 + ax, L)], seed=11)
        b = oinf.line_noise(11, 5 + ax, L, side).astype(np.float32).astype(np.float64)
        oinf.add_line(ref, A64, B64, ax, d, L, b, 0.9)
    torch.cuda.synchronize()
    got = _np(scr)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.sqrt(np.mean(ref ** 2))


def test_grown_strip_statistics_on_the_gpu(env):
    """2400 rows grown on the GPU from an FFT screen: the structure function
    along and across the growth direction follows 2 (C(0) - C(r))."""
    torch, sp, ctx = env
    side, n_st, pitch, r0, L0 = 32, 2, 0.1, 0.1, 8.0
    A, B = sp.specula_infscreen_operators(ctx, side, n_st, pitch, r0, L0)
    import synth
    scr = torch.empty(side, side, device="cuda")
    sp.specula_screen_generate(ctx, side, pitch, r0, L0,
                               torch.tensor(synth.screen_noise(3, side), device="cuda"),
                               synth.subharmonic_noise(3), scr)
    rows = []
    for k in range(2400):
        L = side + k
        sp.specula_infscreen_lines(ctx, side, n_st, [(scr, A, B, 1.0, 0, 1, 0, L)], seed=21)
        if (k + 1) % side == 0:
            blk = scr.cpu().numpy().astype(np.float64)
            first = L - side + 1
            rows += [blk[(first + j) % side] for j in range(side)]
    strip = np.array(rows[100:])
    c0 = oinf.vk_covariance(np.array([0.0]), r0, L0)[0]
    for lag in (1, 2, 4):
        theory = 2 * (c0 - oinf.vk_covariance(np.array([lag * pitch]), r0, L0)[0])
        along = oinf.structure_function(strip, lag)
        across = float(np.mean((strip[:, lag:] - strip[:, :-lag]) ** 2))
        assert abs(along / theory - 1) < 0.1, (lag, along / theory)
        assert abs(across / theory - 1) < 0.1, (lag, across / theory)


def test_infinite_frame_extraction_and_window(env):
    """The 8 m pyramid frame on infinite rings: after 2 s of flow the layers
    have grown hundreds of lines, the extraction of the rings matches the oracle
    extraction, and every line the footprint reads lies in the ring window."""
    torch, sp, ctx = env
    import synth
    from paper_2602_06688_gb300.frame import PwfsFrame
    wl = synth.workload("pwfs8m")
    fr = PwfsFrame(ctx, wl, infinite=dict(side=256, n_st=2, seed=4))
    for k in range(100):
        fr.frame(2.0 + k * fr.dt)
    torch.cuda.synchronize()
    t = 2.0 + 99 * fr.dt
    assert fr.inf.lines_grown > 200
    s = wl.sensors[0]
    for i, l in enumerate(wl.layers):
        for ax, th, v in ((0, s.source.theta_y_rad, l.vy_mps), (1, s.source.theta_x_rad, l.vx_mps)):
            i0, _ = atmo.layer_coords(s.pupil.n_pix, s.pupil.pitch_m, 256, l.pitch_m, l.height_m,
                                      th, v, s.source.height_m, t)
            lo = fr.inf.lo[i][ax]
            assert lo <= i0.min() and i0.max() + 1 <= lo + 255
    rings = [x.cpu().numpy().astype(np.float64) for x in fr.screens]
    ref = atmo.atmo_extract(rings, fr.layers, s.source, s.pupil.n_pix, s.pupil.pitch_m, t)
    tol = (500.0 / s.source.wavelength_nm) * sum(np.abs(x).max() for x in rings) * 4 * EPS32
    assert np.max(np.abs(_np(fr.phase) - ref)) <= tol
    assert np.all(np.isfinite(_np(fr.modes)))


def test_native_advance_equals_planned_calls(env):
    """specula_infscreen_advance produces bit-identical rings to the moves of
    specula_infscreen_plan issued as explicit line calls (rounds in layer
    order, stream id 2 layer + axis)."""
    torch, sp, ctx = env
    import synth
    wl = synth.workload("pwfs8m")
    s = wl.sensors[0]
    side, n_st = 256, 2
    A, B = sp.specula_infscreen_operators(ctx, side, n_st, wl.layers[0].pitch_m,
                                          wl.layers[0].r0_m, wl.layers[0].L0_m)
    layers = []
    for l in wl.layers:
        d = sp.layer_desc(l)
        d.side = side
        layers.append(d)
    src, pu = sp.source_desc(s.source), sp.pupil_desc(s.pupil)
    rng = np.random.default_rng(9)
    init = [torch.tensor((rng.standard_normal((side, side)) * 10).astype(np.float32),
                         device="cuda") for _ in layers]
    ra = [x.clone() for x in init]
    rb = [x.clone() for x in init]
    bs = [(wl.layers[0].r0_m / l.r0_m) ** (5 / 6) for l in wl.layers]
    lo_a = [0] * (2 * len(layers))
    lo_b = list(lo_a)
    for t in (0.3, 0.31, 0.5):
        sp.specula_infscreen_advance(ctx, layers, src, pu, side, n_st, 1, ra, [A] * 3, [B] * 3,
                                     bs, lo_a, t, seed=5)
        moves, lo_b = sp.specula_infscreen_plan(layers, src, pu, side, 1, t, lo_b, 100000)
        per = [[m for m in moves if m[0] == i] for i in range(len(layers))]
        for k in range(max(len(p) for p in per)):
            tasks = [(rb[i], A, B, bs[i], p[k][1], p[k][2], 2 * i + p[k][1], p[k][3])
                     for i, p in enumerate(per) if k < len(p)]
            sp.specula_infscreen_lines(ctx, side, n_st, tasks, seed=5)
        assert lo_a == lo_b
    torch.cuda.synchronize()
    assert sum(abs(v) for v in lo_a) > 20
    for x, y in zip(ra, rb):
        assert torch.equal(x, y)



def test_argument_checks(env):
    torch, sp, ctx = env
    import math
    bad_ops = [(1, 1, 0.1, 0.1, 10.0), (1025, 2, 0.1, 0.1, 10.0), (8, 5, 0.1, 0.1, 10.0),
               (8, 8, 0.1, 0.1, 10.0), (8, 2, 0.1, 0.1, math.inf), (8, 2, -0.1, 0.1, 10.0),
               (8, 2, 0.1, 0.0, 10.0)]
    for side, n_st, pitch, r0, L0 in bad_ops:
        with pytest.raises(sp.SpeculaError) as e:
            sp.specula_infscreen_operators(ctx, side, n_st, pitch, r0, L0)
        assert e.value.status == sp.EINVAL
    side, n_st = 16, 2
    A, B = sp.specula_infscreen_operators(ctx, side, n_st, 0.1, 0.1, 10.0)
    scr = torch.zeros(side, side, device="cuda")
    for task in [(scr, A, B, 1.0, 2, 1, 0, 5), (scr, A, B, 1.0, 0, 0, 0, 5),
                 (scr, A, B, float("nan"), 0, 1, 0, 5)]:
        with pytest.raises(sp.SpeculaError) as e:
            sp.specula_infscreen_lines(ctx, side, n_st, [task])
        assert e.value.status == sp.EINVAL
    with pytest.raises(sp.SpeculaError) as e:       # the same ring twice in one call
        sp.specula_infscreen_lines(ctx, side, n_st, [(scr, A, B, 1.0, 0, 1, 0, 5),
                                                     (scr, A, B, 1.0, 1, 1, 1, 5)])
    assert e.value.status == sp.EINVAL
    sp.specula_infscreen_lines(ctx, side, n_st, [])  # no task: a no-op
    torch.cuda.synchronize()
    assert bool((scr == 0).all())
