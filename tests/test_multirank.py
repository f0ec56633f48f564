"""The multi-GPU path of the benchmark on CPU: two gloo ranks, the max-over-ranks step time
and the whole-job throughput of independent replicas (no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [2.0, 3.5][rank]              # rank 1 is the slower replica
    m = bench.max_over_ranks(ms, dist, "cpu")
    v = bench.replica_throughput(1000, world, m)
    dist.barrier()
    q.put((rank, m, v))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, m, v in res:
        assert m == pytest.approx(3.5)
        assert v == pytest.approx(2 * 1000 / 3.5e-3)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(1.25, None, "cpu") == 1.25
    assert bench.replica_throughput(10, 1, 1.0) == pytest.approx(1e4)
