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
