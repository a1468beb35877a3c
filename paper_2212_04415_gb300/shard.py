"""Sample sharding of the MLMC estimator over processes (Section 4).

The samples of a level are independent, so a run over several GPUs deals
each process whole batches of consecutive sample ids and exchanges nothing
while the samples run. Afterwards the per-batch FP64 sums (n, sum Y, sum Y^2)
that ``mlmc_estimate`` returns are gathered once on the host and added in
sample order, starting from zero: the same additions, in the same order, as a
single process that ran every batch makes, so the merged level totals are
bit-identical to that run's.
"""
from __future__ import annotations

import numpy as np


def split(n_samples, batch: int, world: int, rank: int):
    """(first_sample, count) per level for one process.

    Level l has ceil(N_l / batch) batches; process r takes a contiguous run of
    them (the first N_batches mod world processes one more), so every process
    holds whole batches and only the last batch of a level may be short.
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    if batch < 1:
        raise ValueError("batch must be >= 1")
    first, count = [], []
    for n in n_samples:
        n = int(n)
        if n < 0:
            raise ValueError("n_samples must be >= 0")
        nb = -(-n // batch)
        per, extra = divmod(nb, world)
        b0 = rank * per + min(rank, extra)
        b1 = b0 + per + (1 if rank < extra else 0)
        s0 = min(n, b0 * batch)
        first.append(s0)
        count.append(min(n, b1 * batch) - s0)
    return first, count


def merge(batch_sums_by_rank):
    """Level totals from every process's per-batch sums.

    ``batch_sums_by_rank[r][l]`` is the [n_batches, 3] array that process r's
    ``mlmc_estimate`` returned for level l; processes are listed in rank order,
    which is sample order under ``split``. The arrays are concatenated level
    by level in that order and handed to the library's ``mlmc_merge``, which
    adds them from zero (the additions of a single run) and forms the
    estimator Q_ML = sum_l Y_hat_l with its variance sum_l V_l / N_l (Eqs.
    MLMC_estimator, MLMC_error)."""
    import numpy as np

    from . import mlmc_merge
    n_levels = len(batch_sums_by_rank[0])
    per_level = [np.concatenate([np.asarray(r[l], np.float64).reshape(-1, 3) for r in batch_sums_by_rank])
                 for l in range(n_levels)]
    return mlmc_merge(per_level)


def allgather(obj, group=None):
    """Host-side gather of one picklable object per process (torch.distributed)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return [obj]
    out = [None] * dist.get_world_size(group)
    dist.all_gather_object(out, obj, group=group)
    return out


def sharded_mlmc_estimate(grids, bcs, max_steps, n_samples, mat, field, seed, batch, group=None, **kw):
    """``mlmc_estimate`` with this process's share of every level's samples,
    merged over the process group (one host-side gather at the end)."""
    import torch.distributed as dist
    from . import mlmc_estimate
    world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank(group) if world > 1 else 0
    first, count = split(n_samples, batch, world, rank)
    local = mlmc_estimate(grids, bcs, max_steps, count, mat, field, seed, batch, first_sample=first, **kw)
    merged = merge(allgather([bs for bs in local["batch_sums"]], group))
    merged["local"] = local
    merged["first_sample"], merged["count"] = first, count
    return merged
