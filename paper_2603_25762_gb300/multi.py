"""Host logic for running the solver on several GPUs of one node (one process per GPU).

Replicas of bSB are independent (SB algorithm solution: the solver runs many random
starts side by side and keeps the best), so the path shards by replica range and
needs no exchange while it runs:
  * rank r solves replicas base_r .. base_r + R - 1 with base_r = r * R (weak scaling);
  * afterwards one small all-gather picks, per block, the best cut over all ranks
    (ties: lowest global replica index) -- the same rule as inside one GPU;
  * timing reports the slowest rank (MAX).
Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU for tests).
"""
from __future__ import annotations

import numpy as np


def replica_range(rank: int, world: int, replicas_per_rank: int):
    """Global replica indices owned by `rank`: (first index, count)."""
    if not (0 <= rank < world) or replicas_per_rank < 1:
        raise ValueError("bad rank / world / replica count")
    return rank * replicas_per_rank, replicas_per_rank


def max_over_ranks(value: float, group=None) -> float:
    """Largest `value` over all ranks (the job's step time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def best_over_ranks(best_cut, best_replica, group=None):
    """Per block, the best (cut, global replica) over all ranks.

    best_cut     : float64[n_blocks], this rank's best cut per block
    best_replica : int64[n_blocks], its global replica index
    Returns (cut[n_blocks], replica[n_blocks], owner_rank[n_blocks]); ties in the cut go
    to the lowest global replica index, as within one GPU.
    """
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    cut = torch.as_tensor(np.asarray(best_cut, np.float64))
    rep = torch.as_tensor(np.asarray(best_replica, np.int64))
    if dist.get_backend(group) == "nccl":
        cut, rep = cut.cuda(), rep.cuda()
    cuts = [torch.empty_like(cut) for _ in range(world)]
    reps = [torch.empty_like(rep) for _ in range(world)]
    dist.all_gather(cuts, cut, group=group)
    dist.all_gather(reps, rep, group=group)
    C = torch.stack(cuts).cpu().numpy()
    P = torch.stack(reps).cpu().numpy()
    owner = np.zeros(C.shape[1], np.int64)
    for b in range(C.shape[1]):
        best = 0
        for r in range(1, world):
            if C[r, b] > C[best, b] or (C[r, b] == C[best, b] and P[r, b] < P[best, b]):
                best = r
        owner[b] = best
    idx = np.arange(C.shape[1])
    return C[owner, idx], P[owner, idx], owner
