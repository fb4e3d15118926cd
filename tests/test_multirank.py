"""The N > 1 host logic of bench.py on CPU: two gloo ranks combine their
timings (slowest rank) and work (sum over ranks), and split the ensemble's
channels so that every channel is advanced by exactly one rank."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms, units = bench.combine_over_ranks(10.0 + 5.0 * rank, 100.0 * (rank + 1))
        share = bench.ensemble_share(256, rank, ws)
        out.put((rank, ms, units, share))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_two_gloo_ranks_combine_time_and_work(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    shares = []
    for rank, ms, units, share in res:
        assert ms == 15.0                       # the slowest rank's time
        assert units == 300.0                   # 100 + 200 cells
        shares += share
    assert sorted(shares) == list(range(256))   # each channel exactly once


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_over_ranks(3.5, 7) == (3.5, 7.0)
