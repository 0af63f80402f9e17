"""Host-side logic of the multi-GPU benchmark, with 2 gloo ranks on CPU: ranks take disjoint
events, the only collective is the max of the elapsed times, and the whole-job rate counts
every rank's events against the slowest rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        idx = bench.rank_event_indices(rank, 8)
        mine = 1.0 + rank          # rank 1 is slower
        worst = bench.max_over_ranks(mine, torch.device("cpu"))
        rate = bench.whole_job_rate(8 * 3, world, worst)
        q.put((rank, idx, worst, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_partition_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, i0, w0, v0), (r1, i1, w1, v1) = res
    assert not set(i0) & set(i1)                 # disjoint events
    assert w0 == w1 == 2.0                       # both ranks see the slowest time
    assert v0 == v1 == pytest.approx(8 * 3 * 2 / 2.0)
