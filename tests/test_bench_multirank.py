"""The bench's multi-rank aggregation (max over ranks, weak-scaling value)
on two gloo ranks on the CPU."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    def reduce_max(vals):
        t = torch.tensor(vals, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.tolist()
    # rank r is slower by (r+1): the slowest rank's time must be used
    times = [10.0 * (rank + 1), 100.0 * (rank + 1), 0.5 * (rank + 1)]
    agg = bench.aggregate(times, world, 1000, (50, 20, 20), reduce_max)
    dist.barrier()
    q.put((rank, agg))
    dist.destroy_process_group()


def test_two_rank_aggregate_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29611
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        agg = out[r]
        assert agg["ms32"] == 20.0 and agg["ms64"] == 200.0 and agg["e2e_s"] == 1.0
        assert agg["value"] == pytest.approx(2 * 1000 * 50 / 0.020)
        assert agg["value64"] == pytest.approx(2 * 1000 * 20 / 0.200)
        assert agg["e2e"] == pytest.approx(2 * 1000 * 20 / 1.0)
