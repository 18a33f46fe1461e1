"""Host logic for running the solver on several GPUs of one node (one process per GPU).

The path shards at two levels and needs no exchange while the solver runs:
  * Replicas of bSB are independent (SB algorithm solution: the solver runs many random
    starts side by side and keeps the best).  Rank r solves replicas base_r .. base_r +
    R - 1 with base_r = r * R (weak scaling); afterwards one small all-gather picks, per
    block, the best cut over all ranks (ties: lowest global replica index) -- the same
    rule as inside one GPU.
  * Phase blocks (connected components) are independent subproblems.  `block_shards`
    splits the blocks of a graph across ranks by their cost N_b^2 R (the dense-tile
    work of a block grows with the square of its size), each rank solves its share
    (qh_bsb_solve_blocks), and one all-gather of the per-block results lets every rank
    import the others' blocks (qh_solution_set_block) before phasing.
Timing reports the slowest rank (MAX).  Works with any torch.distributed backend (NCCL
on GPUs, gloo on CPU for tests).
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


def sum_over_ranks(value: float, group=None) -> float:
    """Sum of `value` over all ranks (e.g. the spin updates of block shards)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())


def pick_best(C, P):
    """Per block (column), the rank (row) with the best cut C; ties go to the lowest
    global replica index P.  Returns the owner rank of every block."""
    C, P = np.asarray(C), np.asarray(P)
    owner = np.zeros(C.shape[1], np.int64)
    for b in range(C.shape[1]):
        best = 0
        for r in range(1, C.shape[0]):
            if C[r, b] > C[best, b] or (C[r, b] == C[best, b] and P[r, b] < P[best, b]):
                best = r
        owner[b] = best
    return owner


def block_shards(block_sizes, world: int, replicas: int = 1):
    """Split phase blocks across `world` ranks by cost N_b^2 * replicas.

    Greedy longest-processing-time order: blocks by decreasing cost (ties: lower block
    index) each go to the rank with the least cost so far (ties: lower rank).  The
    result is the same on every rank.  Returns one ascending list of block indices per
    rank; the largest rank load is at most 4/3 of the best possible split."""
    if world < 1 or replicas < 1:
        raise ValueError("world and replicas must be >= 1")
    sizes = np.asarray(block_sizes, np.int64)
    cost = sizes.astype(np.float64) ** 2 * replicas
    order = sorted(range(sizes.shape[0]), key=lambda b: (-cost[b], b))
    load = np.zeros(world)
    shards = [[] for _ in range(world)]
    for b in order:
        r = int(np.argmin(load))  # first minimum: the lowest rank among equals
        shards[r].append(b)
        load[r] += cost[b]
    return [sorted(x) for x in shards]


def shard_loads(block_sizes, shards, replicas: int = 1):
    """Cost N_b^2 * replicas summed per rank."""
    sizes = np.asarray(block_sizes, np.float64)
    return [float((sizes[list(s)] ** 2).sum() * replicas) if s else 0.0 for s in shards]


def exchange_block_results(local: dict, group=None) -> dict:
    """All-gather of per-block results: `local` maps block index -> result (any
    picklable value, e.g. the dict Solution.block returns); every rank receives the
    union over all ranks.  A block reported by two ranks is an error."""
    import torch.distributed as dist
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, local, group=group)
    merged = {}
    for part in parts:
        for b, res in part.items():
            if b in merged:
                raise ValueError(f"block {b} solved by two ranks")
            merged[b] = res
    return merged


def solve_blocks_sharded(ctx, g, rank: int, world: int, group=None, **solve_kw):
    """Block-sharded solve of graph `g`: this rank solves its share of the blocks,
    the per-block results are exchanged, and the returned solution holds every block
    (the other ranks' blocks imported), ready for phasing."""
    R = int(solve_kw.get("replicas", 32))
    sizes = g.block_sizes()
    mine = block_shards(sizes, world, R)[rank]
    sol = ctx.solve(g, blocks=mine, **solve_kw)
    local = {}
    for b in mine:
        r = sol.block(b, int(sizes[b]))
        local[b] = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in r.items()}
    merged = exchange_block_results(local, group)
    for b, r in merged.items():
        if b not in local:
            sol.set_block(b, r["spins"], r["best_cut"], r["best_replica"], r["steps_run"],
                          r["iterations"])
    return sol


def combine_best_results(results, group=None) -> dict:
    """Replica sharding's exchange: `results` is this rank's per-block list of results
    (dicts with "best_cut", "best_replica" (global index) and "spins"); every rank
    receives, per block, the result of the rank holding the best cut (ties: lowest
    global replica index).  Only the winning ranks' spins travel."""
    import torch.distributed as dist
    cut, rep, owner = best_over_ranks([r["best_cut"] for r in results],
                                      [r["best_replica"] for r in results], group)
    rank = dist.get_rank(group)
    mine = {b: results[b] for b in range(len(results)) if owner[b] == rank}
    return exchange_block_results(mine, group)


def combine_replica_shards(sol, g, group=None):
    """Make `sol` (this rank's solve of its replica range) the combined solution of all
    ranks: blocks won by another rank are imported from it."""
    sizes = g.block_sizes()
    results = [sol.block(b, int(sizes[b])) for b in range(g.n_blocks)]
    merged = combine_best_results(results, group)
    for b, r in merged.items():
        # replica indices are global and disjoint across ranks: another index is
        # another rank's win
        if r["best_replica"] != results[b]["best_replica"]:
            sol.set_block(b, r["spins"], r["best_cut"], r["best_replica"], r["steps_run"],
                          r["iterations"])
    return sol


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
    owner = pick_best(C, P)
    idx = np.arange(C.shape[1])
    return C[owner, idx], P[owner, idx], owner
