"""Multi-process host logic of multi-GPU runs, on CPU with gloo (world size 2)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import synth
from paper_1711_11224_gb300.shard import lpt_assign, volume_cost


def test_lpt_partition_properties():
    shapes = synth.batch64_shapes()
    costs = [volume_cost(m, q) for m, q, _ in shapes]
    for world in (1, 2, 3, 4, 8):
        parts = lpt_assign(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))                       # every volume exactly once
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= sum(costs) / world + max(costs)        # Graham's bound for LPT
    assert lpt_assign(costs, 4) == lpt_assign(costs, 4)              # deterministic


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shapes = synth.batch64_shapes()
    costs = [volume_cost(m, q3) for m, q3, _ in shapes]
    mine = lpt_assign(costs, world)[rank]
    # each rank "times" its share; the job time is the max over ranks, the work the sum
    t = torch.tensor([float(sum(costs[i] for i in mine))], dtype=torch.float64)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    n = torch.tensor([len(mine)], dtype=torch.int64)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    dist.barrier()
    q.put((rank, mine, float(tmax.item()), int(n.item())))
    dist.destroy_process_group()


def test_two_rank_gloo_sharding():
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
    (r0, m0, t0, n0), (r1, m1, t1, n1) = res
    assert set(m0).isdisjoint(m1) and sorted(m0 + m1) == list(range(64))
    assert n0 == n1 == 64 and t0 == t1
