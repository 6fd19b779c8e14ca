"""The modulation-point partition of one pyramid frame (host side, CPU): the
slot blocks cover every point once and are balanced, and on two gloo ranks
the summed partial images (each rank's points imaged by the oracle) equal
the full image."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_2602_06688_gb300.sharding import slot_points, slot_ranges  # noqa: E402


@pytest.mark.parametrize("n_mod", [1, 2, 3, 5, 12, 16, 24, 48])
def test_slot_ranges_partition_the_points(n_mod):
    nc = n_mod // 2 + 1
    for world in range(1, nc + 1):
        r = slot_ranges(n_mod, world)
        assert len(r) == world and r[0][0] == 0 and r[-1][1] == nc
        assert all(a < b for a, b in r) and all(r[k][1] == r[k + 1][0] for k in range(world - 1))
        pts = [m for a, b in r for c in range(a, b) for m in slot_points(n_mod, c)]
        assert sorted(pts) == list(range(n_mod))
        counts = [sum(len(slot_points(n_mod, c)) for c in range(a, b)) for a, b in r]
        assert max(counts) - min(counts) <= 2
    with pytest.raises(ValueError):
        slot_ranges(n_mod, nc + 1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    from oracle import geometry, pyramid
    from paper_2602_06688_gb300.sharding import slot_points, slot_ranges
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        n, n_mod = 24, 12
        amp = geometry.pupil_mask(n, 0.1).astype(np.float64)
        phase = np.random.default_rng(3).standard_normal((n, n))
        a, b = slot_ranges(n_mod, ws)[rank]
        pts = [m for c in range(a, b) for m in slot_points(n_mod, c)]
        part = pyramid.pwfs_intensity(amp, phase, 2, n_mod, 2.0, n, points=pts)
        t = torch.tensor(part)
        dist.all_reduce(t)
        out[rank] = t.numpy()
    finally:
        dist.destroy_process_group()


def test_two_ranks_sum_to_the_full_image():
    ws = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    from oracle import geometry, pyramid
    n = 24
    amp = geometry.pupil_mask(n, 0.1).astype(np.float64)
    phase = np.random.default_rng(3).standard_normal((n, n))
    full = pyramid.pwfs_intensity(amp, phase, 2, 12, 2.0, n)
    for r in range(ws):
        assert np.max(np.abs(res[r] - full)) <= 1e-12 * full.max()


# ---- the other partitions: SH by subaperture blocks, by sensor, by mode rows

from paper_2602_06688_gb300.sharding import (  # noqa: E402
    _all_gather_var, balanced_assignment, block_ranges, join_xy)


@pytest.mark.parametrize("n,world", [(0, 1), (1, 1), (7, 2), (10, 3), (3364, 4), (5, 5)])
def test_block_ranges_cover_and_balance(n, world):
    r = block_ranges(n, world)
    assert len(r) == world and r[0][0] == 0 and r[-1][1] == n
    assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
    sizes = [e - b for b, e in r]
    assert max(sizes) - min(sizes) <= 1


def test_balanced_assignment():
    costs = [5, 1, 3, 3, 2, 2]
    owners = balanced_assignment(costs, 2)
    assert sorted(i for o in owners for i in o) == list(range(len(costs)))
    loads = [sum(costs[i] for i in o) for o in owners]
    assert abs(loads[0] - loads[1]) <= max(costs)
    assert balanced_assignment(costs, 1) == [list(range(len(costs)))]


def _partition_rank(rank, ws, port, out):
    """Each rank computes, with the oracle, its share of (a) one SH sensor's
    slopes (a block of valid subapertures), (b) a multi-sensor system's
    slopes (its sensors), (c) the modes (its rows of R); the library's
    gather helpers assemble the full results on every rank."""
    sys.path.insert(0, ROOT)
    import synth
    from oracle import geometry, sh, slopes, system
    from paper_2602_06688_gb300.sharding import (SensorShards, _all_gather_var,
                                                 block_ranges, join_xy)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # (a) SH by subaperture blocks
        n, n_sub, sub_pix, fft_n = 64, 8, 8, 16
        amp = geometry.pupil_mask(n, 0.2).astype(np.float64)
        valid = geometry.valid_subaps(amp.astype(np.uint8), n_sub)
        phase = np.random.default_rng(5).standard_normal((n, n)) * 0.5
        ranges = block_ranges(len(valid), ws)
        b, e = ranges[rank]
        spots = sh.sh_spots(amp, phase, n_sub, sub_pix, fft_n, valid[b:e])
        part = torch.tensor(slopes.sh_slopes(spots))
        out[("sh", rank)] = join_xy(_all_gather_var(dist, None, part,
                                                    [2 * (q - p) for p, q in ranges])).numpy()
        # (b) by sensor
        wl = synth.workload("mwfs8m_small")
        scr = [np.random.default_rng(10 + k).standard_normal((l.side, l.side)) * 0.3
               for k, l in enumerate(wl.layers)]
        offs, total = system.slope_offsets(wl.sensors)
        sizes = [(offs + [total])[i + 1] - offs[i] for i in range(len(wl.sensors))]
        shards = SensorShards(sizes, sizes)
        mine = {i: torch.tensor(system.sensor_chain(scr, wl.layers, wl.sensors[i], 0.01)["slopes"])
                for i in shards.mine}
        out[("sys", rank)] = shards.join(mine).numpy()
        # (c) by mode rows
        R = np.random.default_rng(7).standard_normal((37, 50))
        s = np.random.default_rng(8).standard_normal(50)
        mr = block_ranges(37, ws)
        b, e = mr[rank]
        out[("rec", rank)] = torch.cat(_all_gather_var(dist, None, torch.tensor(R[b:e] @ s),
                                                       [q - p for p, q in mr])).numpy()
    finally:
        dist.destroy_process_group()


def test_two_ranks_assemble_sh_system_and_modes():
    ws = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_partition_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    import synth
    from oracle import geometry, sh, slopes, system
    n, n_sub, sub_pix, fft_n = 64, 8, 8, 16
    amp = geometry.pupil_mask(n, 0.2).astype(np.float64)
    valid = geometry.valid_subaps(amp.astype(np.uint8), n_sub)
    phase = np.random.default_rng(5).standard_normal((n, n)) * 0.5
    full_sh = slopes.sh_slopes(sh.sh_spots(amp, phase, n_sub, sub_pix, fft_n, valid))
    wl = synth.workload("mwfs8m_small")
    scr = [np.random.default_rng(10 + k).standard_normal((l.side, l.side)) * 0.3
           for k, l in enumerate(wl.layers)]
    full_sys, _ = system.system_slopes(scr, wl.layers, wl.sensors, 0.01)
    R = np.random.default_rng(7).standard_normal((37, 50))
    s = np.random.default_rng(8).standard_normal(50)
    for r in range(ws):
        assert np.array_equal(res[("sh", r)], full_sh)
        assert np.array_equal(res[("sys", r)], full_sys)
        assert np.max(np.abs(res[("rec", r)] - R @ s)) <= 1e-12 * np.abs(R).sum()
