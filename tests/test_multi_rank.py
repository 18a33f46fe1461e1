"""Two gloo ranks on the CPU: replica sharding and the cross-rank best-replica pick.

Each rank solves its own replica range of every phase block with the FP64 oracle
(no GPU); the combined per-block best must equal one process solving all replicas,
and the slowest rank's time must be what both ranks report.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, R, steps, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    from oracle import oracle as o
    from paper_2603_25762_gb300 import multi, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fr = synth.tiny_reads(1001)
    g = o.read_graph(fr, o.READ_SIGNED)
    base, n = multi.replica_range(rank, world, R)
    cuts, reps = [], []
    for b, nodes in enumerate(o.blocks_of(g)):
        best, _, _, br = o.bsb_solve(g.subgraph(nodes), list(range(base, base + n)), steps, 7, b)
        cuts.append(best)
        reps.append(base + br)
    cut, rep, owner = multi.best_over_ranks(cuts, reps)
    t = multi.max_over_ranks(1.0 + rank)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), cut=cut, rep=rep, owner=owner, t=t)
    dist.destroy_process_group()


def test_replica_range():
    from paper_2603_25762_gb300 import multi
    assert multi.replica_range(0, 2, 64) == (0, 64)
    assert multi.replica_range(1, 2, 64) == (64, 64)
    with pytest.raises(ValueError):
        multi.replica_range(2, 2, 64)


def test_two_gloo_ranks_match_one_process(tmp_path, oracle):
    import torch.multiprocessing as mp
    R, steps, world = 8, 400, 2
    mp.start_processes(_rank_main, args=(world, _free_port(), R, steps, str(tmp_path)),
                       nprocs=world, start_method="spawn", join=True)
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    for r in range(1, world):
        assert np.array_equal(res[r]["cut"], res[0]["cut"])
        assert np.array_equal(res[r]["rep"], res[0]["rep"])
    assert res[0]["t"] == res[1]["t"] == 2.0
    # one process over all 16 replicas
    from paper_2603_25762_gb300 import synth
    fr = synth.tiny_reads(1001)
    g = oracle.read_graph(fr, oracle.READ_SIGNED)
    for b, nodes in enumerate(oracle.blocks_of(g)):
        best, _, cuts, br = oracle.bsb_solve(g.subgraph(nodes), list(range(world * R)), steps, 7, b)
        assert res[0]["cut"][b] == best
        assert res[0]["rep"][b] == br


# ----------------------------------------------------------------------------- block sharding
def test_block_shards_cover_every_block_once_and_balance():
    from paper_2603_25762_gb300 import multi, synth
    sizes = np.array(synth.batched_blocks(1004).meta["block_reads"])
    for world in (1, 2, 3, 4, 8):
        sh = multi.block_shards(sizes, world, 256)
        assert sorted(b for s in sh for b in s) == list(range(sizes.shape[0]))
        assert all(s == sorted(s) for s in sh)
        loads = multi.shard_loads(sizes, sh, 256)
        assert max(loads) <= 4 / 3 * sum(loads) / world + 1e-9
        assert sh == multi.block_shards(sizes, world, 256)  # the same on every rank
    # one huge block: it takes a rank of its own, the rest share the others
    sh = multi.block_shards([5000, 10, 20, 30], 2)
    assert sh == [[0], [1, 2, 3]]
    with pytest.raises(ValueError):
        multi.block_shards(sizes, 0)


def _block_rank_main(rank, world, port, R, steps, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    from oracle import oracle as o
    from paper_2603_25762_gb300 import multi, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fr = synth.batched_blocks(1004, n_blocks=7, n_min=20, n_max=150)
    g = o.read_graph(fr, o.READ_SIGNED)
    blocks = o.blocks_of(g)
    mine = multi.block_shards([len(b) for b in blocks], world, R)[rank]
    local = {}
    for b in mine:  # the oracle stands in for this rank's GPU solve of its blocks
        best, s, _, br = o.bsb_solve(g.subgraph(blocks[b]), list(range(R)), steps, 3, b)
        local[b] = {"best_cut": best, "best_replica": br, "spins": s}
    merged = multi.exchange_block_results(local)
    np.savez(os.path.join(out_dir, f"blk{rank}.npz"), mine=np.array(mine),
             cut=np.array([merged[b]["best_cut"] for b in range(len(blocks))]),
             rep=np.array([merged[b]["best_replica"] for b in range(len(blocks))]),
             spins=np.concatenate([merged[b]["spins"] for b in range(len(blocks))]))
    dist.destroy_process_group()


def test_two_gloo_ranks_block_sharding_match_one_process(tmp_path, oracle):
    """Two ranks split the blocks by cost, solve their own and exchange the results:
    every rank ends with every block, equal to one process solving all of them."""
    import torch.multiprocessing as mp
    R, steps, world = 8, 300, 2
    mp.start_processes(_block_rank_main, args=(world, _free_port(), R, steps, str(tmp_path)),
                       nprocs=world, start_method="spawn", join=True)
    res = [np.load(tmp_path / f"blk{r}.npz") for r in range(world)]
    assert set(res[0]["mine"]).isdisjoint(set(res[1]["mine"]))
    assert len(res[0]["mine"]) > 0 and len(res[1]["mine"]) > 0
    for key in ("cut", "rep", "spins"):
        assert np.array_equal(res[0][key], res[1][key])
    from paper_2603_25762_gb300 import synth
    fr = synth.batched_blocks(1004, n_blocks=7, n_min=20, n_max=150)
    g = oracle.read_graph(fr, oracle.READ_SIGNED)
    spins = []
    for b, nodes in enumerate(oracle.blocks_of(g)):
        best, s, _, br = oracle.bsb_solve(g.subgraph(nodes), list(range(R)), steps, 3, b)
        assert res[0]["cut"][b] == best and res[0]["rep"][b] == br
        spins.append(s)
    assert np.array_equal(res[0]["spins"], np.concatenate(spins))


def test_pick_best_ties_go_to_the_lowest_replica():
    from paper_2603_25762_gb300 import multi
    C = np.array([[5.0, 7.0, 2.0], [5.0, 6.0, 3.0]])
    P = np.array([[70, 1, 9], [64, 0, 8]])
    assert list(multi.pick_best(C, P)) == [1, 0, 1]


def _combine_rank_main(rank, world, port, R, steps, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    from oracle import oracle as o
    from paper_2603_25762_gb300 import multi, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fr = synth.tiny_reads(1001)
    g = o.read_graph(fr, o.READ_SIGNED)
    base, n = multi.replica_range(rank, world, R)
    results = []
    for b, nodes in enumerate(o.blocks_of(g)):
        best, s, _, br = o.bsb_solve(g.subgraph(nodes), list(range(base, base + n)), steps, 7, b)
        results.append({"best_cut": best, "best_replica": base + br, "spins": s})
    merged = multi.combine_best_results(results)
    nb = len(results)
    np.savez(os.path.join(out_dir, f"cmb{rank}.npz"),
             cut=np.array([merged[b]["best_cut"] for b in range(nb)]),
             rep=np.array([merged[b]["best_replica"] for b in range(nb)]),
             spins=np.concatenate([merged[b]["spins"] for b in range(nb)]))
    dist.destroy_process_group()


def test_two_gloo_ranks_combined_solution_is_one_process(tmp_path, oracle):
    """The combined solution of two replica shards (best cut per block, with that
    replica's spins from the rank that holds it) equals one process over all replicas."""
    import torch.multiprocessing as mp
    R, steps, world = 8, 400, 2
    mp.start_processes(_combine_rank_main, args=(world, _free_port(), R, steps, str(tmp_path)),
                       nprocs=world, start_method="spawn", join=True)
    res = [np.load(tmp_path / f"cmb{r}.npz") for r in range(world)]
    for key in ("cut", "rep", "spins"):
        assert np.array_equal(res[0][key], res[1][key])
    from paper_2603_25762_gb300 import synth
    fr = synth.tiny_reads(1001)
    g = oracle.read_graph(fr, oracle.READ_SIGNED)
    spins = []
    for b, nodes in enumerate(oracle.blocks_of(g)):
        best, s, _, br = oracle.bsb_solve(g.subgraph(nodes), list(range(world * R)), steps, 7, b)
        assert res[0]["cut"][b] == best and res[0]["rep"][b] == br
        spins.append(s)
    assert np.array_equal(res[0]["spins"], np.concatenate(spins))
