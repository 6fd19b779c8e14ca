"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): every
rank runs its own replica, the job's time is the slowest rank's, and the
value counts the frames of all ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r "took" 100 (r + 1) ms for 50 frames
        ms, value = bench.aggregate_ranks(100.0 * (rank + 1), 50, ws, dist, "cpu")
        out[rank] = (ms, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_rank_and_count_all_frames():
    ws = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        ms, value = res[r]
        assert ms == pytest.approx(200.0 / 50)           # the slower rank's span
        assert value == pytest.approx(ws * 50 / 0.2)     # all ranks' frames


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.aggregate_ranks(250.0, 50, 1)
    assert ms == 5.0 and value == pytest.approx(200.0)
