"""Host logic of the infinite-screen layers (no GPU): the native ring planner
(specula_infscreen_plan) that decides which lines a frame grows."""
import math

import numpy as np
import pytest

import synth
from oracle import atmo


@pytest.fixture(scope="module")
def sp():
    from paper_2602_06688_gb300 import build
    build.build()
    import paper_2602_06688_gb300 as sp
    return sp


def _descs(sp, wl, sensor, side):
    s = wl.sensors[sensor]
    layers = []
    for l in wl.layers:
        d = sp.layer_desc(l)
        d.side = side
        layers.append(d)
    return s, layers, sp.source_desc(s.source), sp.pupil_desc(s.pupil)


def test_plan_covers_the_extraction_footprint(sp):
    """After planning for time t, each window [lo, lo + side - 1] holds every
    line floor(u), floor(u) + 1 the oracle extraction reads (laser-star cone
    and off-axis source), and the moves are contiguous growth steps."""
    wl = synth.workload("mwfs39m")
    side = 1024
    for sensor in (0, 7):
        s, layers, src, pu = _descs(sp, wl, sensor, side)
        lo = [0] * (2 * len(layers))
        for t in (0.0, 0.004, 0.013, 0.5, 0.5, 0.1, 2.0):
            moves, lo2 = sp.specula_infscreen_plan(layers, src, pu, side, 1, t, lo, 200000)
            # contiguity: per (layer, axis) the lines follow one another from lo
            for li in range(len(layers)):
                for ax in (0, 1):
                    mv = [(d, L) for (l, a, d, L) in moves if l == li and a == ax]
                    w = lo[2 * li + ax]
                    for d, L in mv:
                        if d < 0:
                            w -= 1
                            assert L == w
                        else:
                            assert L == w + side
                            w += 1
                    assert w == lo2[2 * li + ax]
            # columns before rows within a layer
            for li in range(len(layers)):
                axes = [a for (l, a, d, L) in moves if l == li]
                assert axes == sorted(axes, reverse=True)
            lo = lo2
            for li, L in enumerate(wl.layers):
                for ax, th, v in ((1, s.source.theta_x_rad, L.vx_mps),
                                  (0, s.source.theta_y_rad, L.vy_mps)):
                    i0, _ = atmo.layer_coords(s.pupil.n_pix, s.pupil.pitch_m, side, L.pitch_m,
                                              L.height_m, th, v, s.source.height_m, t)
                    w = lo[2 * li + (1 if ax == 1 else 0)]
                    assert w <= i0.min() and i0.max() + 1 <= w + side - 1


def test_plan_errors_and_move_limit(sp):
    wl = synth.workload("pwfs8m")
    s, layers, src, pu = _descs(sp, wl, 0, 256)
    lo = [0] * 6
    # 10 s of flow needs thousands of lines: a small limit refuses and keeps lo
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_infscreen_plan(layers, src, pu, 256, 1, 10.0, lo, 10)
    assert e.value.status == sp.EUNSUPPORTED
    moves, lo2 = sp.specula_infscreen_plan(layers, src, pu, 256, 1, 10.0, lo, 100000)
    assert len(moves) == sum(abs(a - b) for a, b in zip(lo, lo2)) > 1000
    # a ring narrower than the footprint
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_infscreen_plan(layers, src, pu, 128, 1, 0.0, lo, 100)
    assert e.value.status == sp.EUNSUPPORTED
    with pytest.raises(sp.SpeculaError) as e:      # a jump of about 4e8 lines
        sp.specula_infscreen_plan(layers, src, pu, 256, 1, 1e6, lo, 100)
    assert e.value.status == sp.EUNSUPPORTED
    with pytest.raises(sp.SpeculaError) as e:
        sp.specula_infscreen_plan(layers, src, pu, 256, 1, math.nan, lo, 100)
    assert e.value.status == sp.EINVAL
    # no motion, no moves
    moves, lo3 = sp.specula_infscreen_plan(layers, src, pu, 256, 1, 10.0, lo2, 10)
    assert moves == [] and lo3 == lo2
    assert np.all(np.array(lo2[0::2]) != 0) or np.all(np.array(lo2[1::2]) != 0)
