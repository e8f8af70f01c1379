"""Host-side logic of running on several GPUs of one node.

A single factorisation does not shard: its columns form one dependency DAG
over all of space, and a partition would need an exchange at each of its
hundreds of levels.  So the ranks run replicas (one process per GPU, each on
its own point set), and many independent point sets (batches, requests) are
split across ranks by cost with no collective on the data path; the ranks
only meet for a barrier around the timed region, the maximum of their
times, and a gather of small results on the host.

Everything here is plain ``torch.distributed`` on whatever backend the
process group has (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def rank_world() -> tuple[int, int]:
    """(rank, world size) from the launcher's environment (1 process: 0, 1)."""
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def init(backend: str = "nccl") -> tuple[int, int]:
    """Join the process group when launched with more than one rank."""
    rank, world = rank_world()
    if world > 1 and not dist.is_initialized():
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    return rank, world


def barrier():
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(values, device=None):
    """Elementwise maximum of a list of floats over all ranks."""
    vals = [float(v) for v in values]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return vals
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def sum_over_ranks(values, device=None):
    vals = [float(v) for v in values]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return vals
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(v) for v in t.tolist()]


def partition(costs, world: int) -> list[list[int]]:
    """Split independent units over `world` ranks by greedy balance: units in
    decreasing cost (ties by index) each go to the rank with the least total
    so far (ties to the lower rank).  Deterministic, so every rank computes
    the same split without communicating."""
    loads = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-float(costs[k]), k)):
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += float(costs[i])
    for p in parts:
        p.sort()
    return parts


def gather(obj):
    """Every rank's small host object, in rank order (a list of one without a
    process group)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out


def throughput(units_per_rank, times_per_rank_s) -> float:
    """Whole-job throughput: the units of all ranks over the slowest rank's
    time."""
    return float(sum(units_per_rank)) / float(max(times_per_rank_s))
