"""One process per GPU: how the evaluation is spread over ranks.

Configurations are independent (Eq. 1 neighbourhoods never cross configurations, and Eqs. 5-6
are sums of per-atom terms), so ranks exchange no data on the evaluation path.  Two layouts:

* replicas (weak scaling): every rank evaluates its own seeded workload of the same shape;
* shards (strong scaling): a batch is cut into contiguous ranges of whole configurations with
  about equal atom counts, one range per rank.

The only collectives are on timings and totals: the step time of a job is the maximum over
ranks, and its throughput is the units of all ranks divided by that time.
"""

import os

import numpy as np


def env():
    """(rank, world_size, local_rank) from the launcher's environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(base, rank):
    """Seed of a rank's replica: distinct per rank, the base seed on rank 0."""
    return int(base) + int(rank)


def shard_ranges(cfg_off, world):
    """Contiguous configuration ranges [(k0, k1)] per rank, cut where the running atom count
    crosses r * N / world; every configuration lands in exactly one range (empty ranges only
    when there are fewer configurations than ranks)."""
    off = np.asarray(cfg_off, dtype=np.int64)
    K = off.shape[0] - 1
    if K < 0 or world < 1:
        raise ValueError("need cfg_off of length >= 1 and world >= 1")
    N = int(off[-1])
    cuts = [0]
    for r in range(1, world):
        target = r * N / world
        # first configuration boundary at or after the target atom count
        k = int(np.searchsorted(off, target, side="left"))
        cuts.append(min(max(k, cuts[-1]), K))
    cuts.append(K)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def local_batch(batch, rank, world):
    """The rank's shard of a packed batch (pos, types, cells, cfg_off rebased to 0)."""
    from .synth import Batch

    k0, k1 = shard_ranges(batch.cfg_off, world)[rank]
    a0, a1 = int(batch.cfg_off[k0]), int(batch.cfg_off[k1])
    off = np.asarray(batch.cfg_off[k0:k1 + 1], dtype=np.int32) - a0
    return Batch(batch.pos[a0:a1].copy(), batch.types[a0:a1].copy(), batch.cells[k0:k1].copy(), off)


def max_over_ranks(value, device="cpu"):
    """Maximum of a float over the ranks of the default process group (the value itself alone)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device="cpu"):
    """Sum of a float over the ranks of the default process group (the value itself alone)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_all_ranks, ms_max):
    """Units per second of the whole job: all ranks' units over the slowest rank's time."""
    if ms_max <= 0:
        raise ValueError("step time must be positive")
    return float(units_all_ranks) / (ms_max * 1e-3)
