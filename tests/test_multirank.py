"""The bench's N > 1 path on CPU: two gloo ranks aggregate independent
replicas (every rank's node updates over the slowest rank's time)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench._barrier(world)
        # rank r did (r + 1) * 1e6 updates in (r + 1) * 100 ms
        value, ms_max = bench.aggregate_replicas((rank + 1) * 1e6, (rank + 1) * 100.0, world)
        q.put((rank, value, ms_max))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, value, ms_max in got:
        assert ms_max == pytest.approx(200.0)
        assert value == pytest.approx(3e6 / 0.2)   # both ranks' updates over the slowest time


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    value, ms_max = bench.aggregate_replicas(5e6, 250.0, 1)
    assert ms_max == 250.0 and value == pytest.approx(5e6 / 0.25)
