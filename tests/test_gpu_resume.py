"""Resume from a saved state.  Steps t0 .. t0+2n run in one call and as two calls of n
steps (the state x, y copied out and back in between, as a checkpoint would) give
bit-identical states, on every step-kernel family.  The product operand is not part
of the saved state: every kernel rebuilds it from x exactly as its epilogue writes it.

At the solve level, the SNP refinement's state after k solves (flip counts, the gauge of
the weights, the blocks still refining, their deformation) saved and resumed ends where
one uninterrupted loop ends.
"""
import numpy as np
import pytest

from paper_2603_25762_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_25762_gb300 import build, qhap
    build.build()
    return qhap


@pytest.fixture(scope="module")
def ctx(q):
    return q.Context(0)


CASES = [  # (precision, step kernel, storage, R, SB variant)
    (0, None, 1, 64, "ballistic"),
    (1, "cta-bn128-s2-x3", 1, 128, "ballistic"),
    (1, "persistent-bn64-tma-state", 1, 128, "discrete"),
    (1, "multistep-stream-tile", 1, 256, "ballistic"),
    (1, "multistep-jres-group", 1, 256, "adiabatic"),
    (3, None, 1, 128, "ballistic"),
    (0, "csr-lane8", 2, 64, "discrete"),
    (1, "csr-lane8", 2, 128, "ballistic"),
    (1, "csr-band8", 2, 128, "ballistic"),
]


@pytest.mark.parametrize("precision,kernel,storage,R,variant", CASES)
def test_split_step_range_is_bit_identical(q, ctx, precision, kernel, storage, R, variant):
    import torch
    fr = synth.batched_blocks(1004, n_blocks=4, n_min=80, n_max=300)
    g = ctx.build_graph(fr, mode=q.MODE_READ, storage=storage)
    n_pad, pidx, c0 = g.layout()
    rng = np.random.default_rng(9)
    x = np.zeros((R, n_pad), np.float32)
    y = np.zeros((R, n_pad), np.float32)
    real = pidx[pidx >= 0]
    x[:, real] = rng.uniform(-0.1, 0.1, (R, real.size))
    y[:, real] = rng.uniform(-0.1, 0.1, (R, real.size))
    dt = 0.25 if variant == "adiabatic" else 1.0  # aSB diverges at 0.5 from mid-schedule
    t0, n, steps = 101, 20, 400  # an odd t0: the operand's double buffer starts on its odd side
    kw = dict(dt=dt, c0=c0, step_kernel=kernel, variant=variant)
    xa, ya = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ctx.debug_steps(g, precision, R, xa, ya, t0, 2 * n, steps, **kw)
    xb, yb = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ctx.debug_steps(g, precision, R, xb, yb, t0, n, steps, **kw)
    saved = (xb.cpu().numpy().copy(), yb.cpu().numpy().copy())  # the checkpoint
    xc, yc = torch.from_numpy(saved[0]).cuda(), torch.from_numpy(saved[1]).cuda()
    ctx.debug_steps(g, precision, R, xc, yc, t0 + n, n, steps, **kw)
    assert not np.array_equal(saved[0], x)  # the steps moved the state
    assert np.isfinite(xa.cpu().numpy()).all() and np.isfinite(ya.cpu().numpy()).all()
    assert np.array_equal(xc.cpu().numpy(), xa.cpu().numpy())
    assert np.array_equal(yc.cpu().numpy(), ya.cpu().numpy())


# ----------------------------------------------------------------------------- refinement
def _refine_case(ctx, g, n_snps, k, **kw):
    """One SNP-mode solve with refine_max = kw's, and the same loop stopped after k
    solves, saved (refine_state) and resumed: both must end in the same place."""
    full = ctx.solve(g, **kw)
    part = ctx.solve(g, **dict(kw, refine_max=k))
    st = part.refine_state(g.n_nodes)
    assert st["iterations_done"] == k
    rest = ctx.solve(g, resume=st, **kw)
    sf, sr = full.refine_state(g.n_nodes), rest.refine_state(g.n_nodes)
    assert sr["iterations_done"] == sf["iterations_done"]
    for key in ("flips", "gauge", "refining", "solves", "deform", "tries"):
        assert np.array_equal(sr[key], sf[key]), key
    assert np.array_equal(rest.spins(g.n_nodes), full.spins(g.n_nodes))
    for b in range(g.n_blocks):
        bf, br = full.block(b), rest.block(b)
        assert br["best_cut"] == bf["best_cut"] and br["iterations"] == bf["iterations"], b
    hf, hr = ctx.phase(g, full, n_snps), ctx.phase(g, rest, n_snps)
    for a, c in zip(hf, hr):
        assert np.array_equal(a, c)
    return sf


@pytest.mark.parametrize("precision,storage,R,kernel", [(1, 1, 64, None), (0, 1, 64, None),
                                                        (1, 2, 128, "csr-band8")])
def test_refinement_checkpoint_resumes_to_the_same_result(q, ctx, precision, storage, R, kernel):
    """SNP refinement (flip counts C, sign inversions of the crossing edges) saved after
    k solves and resumed gives the flip counts, parity partition, final cuts and
    haplotypes of one uninterrupted loop."""
    fr = synth.region_reads(32, n_snps=400, region=130_000, n_reads=110, len_mean=8000,
                            len_sd=2000, flip_p=0.08, miss_p=0.0, qual=(7, 30))
    g = ctx.build_graph(fr, mode=q.MODE_SNP, storage=storage)
    kw = dict(replicas=R, steps=300, precision=precision, seed=6, refine_max=15,
              step_kernel=kernel)
    sf = _refine_case(ctx, g, fr.n_snps, 1, **kw)
    assert sf["solves"].max() >= 2  # the loop went on past the checkpoint in some block
    if sf["solves"].max() >= 3:
        _refine_case(ctx, g, fr.n_snps, 2, **kw)


def test_refinement_checkpoint_with_deformation(q, ctx):
    """The same with the deformed re-solves: the state carries each block's field and
    the re-solves it has used."""
    fr = synth.ont_region(1003, scale=0.06)
    g = ctx.build_graph(fr, mode=q.MODE_SNP)
    kw = dict(replicas=64, steps=300, precision=1, seed=3, refine_max=8, deform_h=0.025,
              deform_tries=2)
    sf = _refine_case(ctx, g, fr.n_snps, 1, **kw)
    assert sf["solves"].max() >= 2
    _refine_case(ctx, g, fr.n_snps, 2, **kw)


def test_refinement_state_rejections(q, ctx):
    fr = synth.region_reads(32, n_snps=150, region=50_000, n_reads=40, len_mean=8000,
                            len_sd=2000, flip_p=0.08, miss_p=0.0, qual=(7, 30))
    g = ctx.build_graph(fr, mode=q.MODE_SNP)
    kw = dict(replicas=64, steps=100, precision=1, seed=6, refine_max=4)
    st = ctx.solve(g, **dict(kw, refine_max=1)).refine_state(g.n_nodes)
    bad = dict(st, gauge=np.zeros_like(st["gauge"]))
    with pytest.raises(q.QhError) as e:
        ctx.solve(g, resume=bad, **kw)
    assert e.value.status == q.QH_EINVAL
    with pytest.raises(q.QhError):  # iterations_done must stay below refine_max
        ctx.solve(g, resume=st, **dict(kw, refine_max=1))
    with pytest.raises(q.QhError):  # a deformation field without deform_h
        ctx.solve(g, resume=dict(st, deform=np.full_like(st["deform"], 0.5)), **kw)
    gr = ctx.build_graph(fr, mode=q.MODE_READ)
    with pytest.raises(q.QhError):  # READ mode has no refinement
        ctx.solve(gr, replicas=64, steps=100, precision=1).refine_state(gr.n_nodes)
