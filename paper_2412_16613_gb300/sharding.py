"""Splitting one ensemble's runs over ranks (one GPU per rank) and combining results.

Runs are independent and every group of 32 runs draws from its own counter stream,
so a rank that holds runs [first_run, first_run + n_runs) (first_run a multiple of
32, passed as ssa_options.first_run) produces exactly the runs a single context
would.  The only exchange is the final sum of the per-snapshot histograms and run
counters (and the maximum of the longest-group counter); there is no collective on
the data path.  Under the state-following bound (pad_pow2 = 2) a run's draws also
depend on the other runs of its group, and whole-group shards keep those together.
"""
from __future__ import annotations

import numpy as np

GROUP = 32


def shard(total_runs: int, rank: int, world: int) -> tuple[int, int]:
    """(first_run, n_runs) of `rank`: contiguous whole groups, as even as possible."""
    if world < 1 or not 0 <= rank < world or total_runs < 0:
        raise ValueError("bad shard arguments")
    groups = -(-total_runs // GROUP)
    per, extra = divmod(groups, world)
    g0 = rank * per + min(rank, extra)
    g1 = g0 + per + (1 if rank < extra else 0)
    first = g0 * GROUP
    return first, max(0, min(g1 * GROUP, total_runs) - first)


def weak_shard(runs_per_rank: int, rank: int) -> tuple[int, int]:
    """Weak scaling: rank r holds runs [r R, (r + 1) R) of one larger ensemble (R a multiple of 32)."""
    if runs_per_rank % GROUP:
        raise ValueError("runs per rank must be a multiple of 32")
    return rank * runs_per_rank, runs_per_rank


# counter indices whose combination over ranks is a maximum (the longest group) or a bitwise or
# (the layouts that ran) rather than a sum
MAX_COUNTERS = (8,)
OR_COUNTERS = (9,)


def combine(hist: np.ndarray, counters: np.ndarray, dist=None):
    """Sum histograms and counters over the ranks of `dist` (torch.distributed), taking the
    maximum for the longest-group counter and the bitwise or for the layout counter.  Returns
    numpy arrays (unchanged without dist)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return hist, counters
    import torch
    counters = np.asarray(counters, dtype=np.uint64)
    h = torch.from_numpy(np.ascontiguousarray(hist, dtype=np.float64))
    c = torch.from_numpy(np.ascontiguousarray(counters, dtype=np.float64))
    cmax = c.clone()
    # the or of small bit sets as a maximum per bit
    bits = torch.tensor([float((int(counters[i]) >> b) & 1) for i in OR_COUNTERS if i < len(counters)
                         for b in range(8)], dtype=torch.float64)
    dist.all_reduce(h)
    dist.all_reduce(c)
    dist.all_reduce(cmax, op=dist.ReduceOp.MAX)
    if bits.numel():
        dist.all_reduce(bits, op=dist.ReduceOp.MAX)
    out_c = c.numpy().copy()
    for i in MAX_COUNTERS:
        if i < len(out_c):
            out_c[i] = cmax[i].item()
    for j, i in enumerate(k for k in OR_COUNTERS if k < len(out_c)):
        out_c[i] = sum(int(bits[8 * j + b].item()) << b for b in range(8))
    return h.numpy().astype(np.uint64), out_c.astype(np.uint64)
