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
