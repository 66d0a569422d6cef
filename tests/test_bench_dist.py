"""Host-side multi-rank logic of bench.py on CPU (gloo, world size 2): the
whole-job rate is the sum of all ranks' units over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (r + 1) * 100 ms for (r + 1) * 1e6 units
    value, max_ms = bench.aggregate((rank + 1) * 100.0, (rank + 1) * 1e6, dist)
    q.put((rank, value, max_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, value, max_ms in res:
        assert max_ms == pytest.approx(200.0)
        assert value == pytest.approx(3e6 / 0.2)


def test_aggregate_single_rank():
    import bench
    value, ms = bench.aggregate(250.0, 5e5, None)
    assert ms == 250.0 and value == pytest.approx(2e6)
