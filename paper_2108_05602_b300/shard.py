"""Multi-process (one process per GPU) plumbing of the search.

The search partitions into independent units (scans, and within a scan
baselines x DM trials); the paper's MPI farm exchanges no data between
workers either (Sec. 2.4.1).  The one cross-unit step is the cross-baseline
match (a10), a host step over small candidate lists: when the baselines of
one scan are split over ranks, each rank searches its share with
min_baselines = 1 and rank 0 gathers the window-matched lists and runs
volks_cross_match once.  Benchmark timing uses a max over ranks and a sum of
trials.  All collectives here are host-side (gloo or NCCL through
torch.distributed) on KB-sized data, never on the visibilities.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple


def shard_range(n: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous block [lo, hi) of n units for `rank` of `world`; sizes
    differ by at most one, lower ranks take the extra units."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def reduce_step(trials: float, elapsed_s: float, device=None) -> Tuple[float, float]:
    """(sum of trials over ranks, max elapsed over ranks); identity when
    torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(trials), float(elapsed_s)
    t = torch.tensor([float(trials)], dtype=torch.float64, device=device)
    e = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(e, op=dist.ReduceOp.MAX)
    return t.item(), e.item()


def gather_candidates(cands: List[dict], bl_offset: int, dst: int = 0) -> Optional[List[dict]]:
    """Gather window-matched candidates of every rank's baseline shard to
    rank `dst`, renumbering baselines to the scan's global indices.  Returns
    the merged list on `dst`, None elsewhere."""
    import torch.distributed as dist
    mine = [dict(c, bl=c["bl"] + bl_offset) for c in cands]
    if not (dist.is_available() and dist.is_initialized()):
        return mine
    world, rank = dist.get_world_size(), dist.get_rank()
    got = [None] * world if rank == dst else None
    dist.gather_object(mine, got, dst=dst)
    if rank != dst:
        return None
    return [c for part in got for c in part]


def merge_shards(merged: Sequence[dict], min_baselines: int) -> List[dict]:
    """Cross-baseline match of the gathered lists (a10, in the library)."""
    from . import volks
    return volks.volks_cross_match(list(merged), min_baselines)
