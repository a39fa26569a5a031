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


def _lpt_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    cfg = dict(bench.PRESETS["batch256"])
    inst = bench.batch_instances(cfg)
    costs = [N * N * __import__("math").log2(N + 1) for (N, _, _, _, _) in inst]
    mine = bench.lpt_partition(costs, world)[rank]
    got = [None] * world
    dist.all_gather_object(got, mine)
    q.put((rank, got, costs))
    dist.destroy_process_group()


def test_two_rank_lpt_partition_of_the_batch_workload():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_lpt_worker, args=(r, 2, 29613, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, (g, c)) for r, g, c in (q.get(timeout=120) for _ in range(2)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (g0, costs), (g1, _) = out[0], out[1]
    assert g0 == g1                                   # every rank computes the same split
    a, b = g0
    assert sorted(a + b) == list(range(256)) and not set(a) & set(b)
    la, lb = sum(costs[i] for i in a), sum(costs[i] for i in b)
    assert abs(la - lb) <= max(costs)                 # LPT bound: within one item


def test_batch_instances_follow_the_recipe():
    import bench
    inst = bench.batch_instances(bench.PRESETS["batch256"])
    assert len(inst) == 256
    for N, al, ka, ta, sd in inst:
        assert N in (127, 255, 511, 1023, 2047)
        assert 1.1 <= al <= 1.9 and 0.5 <= ka <= 2.0 and ta == 1.0 / (N + 1)
    assert len({x[0] for x in inst}) == 5
    assert inst == bench.batch_instances(bench.PRESETS["batch256"])   # seeded


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    # the reference arm launched the way every arm is launched for N > 1
    # (torchrun, one process per GPU): rank 0 times the oracle and prints one
    # JSON line; the other rank exits 0 without work
    import json
    import socket
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1", "--N", "63"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-3000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
