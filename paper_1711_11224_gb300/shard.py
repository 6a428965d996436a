"""Assignment of independent problems to GPUs (one process per GPU).

The batched workload has no data exchange between volumes, so a multi-GPU
run only partitions the volumes: longest-processing-time-first on the
convolution cost prod(m) x prod(2p+1), each volume to the least loaded rank.
The only collectives in such a run are a barrier and a max of the elapsed
times.
"""
from __future__ import annotations


def volume_cost(m, q):
    c = 1
    for v in m:
        c *= int(v)
    for v in q:
        c *= int(v)
    return c


def lpt_assign(costs, world):
    """Indices of the volumes of each rank (list of lists), greedy LPT; deterministic."""
    if world < 1:
        raise ValueError("world size must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        out[r].append(i)
        loads[r] += costs[i]
    return [sorted(v) for v in out]
