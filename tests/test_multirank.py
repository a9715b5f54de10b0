"""World-size-2 gloo run of the benchmark's cross-rank logic on CPU: each
rank times its own replica, rank 0 reports the max over ranks and the
whole-job throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


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
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    dist.barrier()
    total, value = bench.aggregate_over_ranks(local_ms, steps=10, pairs_per_step=1000, world=world,
                                              dist=dist, device="cpu")
    seeds = [bench.replica_seed(2, r) for r in range(world)]
    q.put((rank, total, value, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, value, seeds in res:
        assert total == pytest.approx(150.0)
        assert value == pytest.approx(2 * 10 * 1000 / 0.150)
        assert len(set(seeds)) == 2  # distinct replica scenes
