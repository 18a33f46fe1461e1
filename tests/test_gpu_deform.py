"""The SNP refinement's deformation field on the GPU against the FP64 oracle, through
the C ABI: the state after a few steps with a field of a different strength in every
block, on each step-kernel family, and whole refinements with deformed re-solves.

Bars as for the plain steps: state within 1e-5 (FP32) / 1e-2 (BF16, FP8 after one step)
relative Frobenius of the oracle's; refinement cuts >= 0.999 x the oracle's.
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


def _rel_frob(a, b):
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / n if n > 0 else np.linalg.norm(a - b)


CASES = [  # (precision, step kernel, storage, R, steps compared, tolerance)
    (0, None, 1, 64, 3, 1e-5),
    (1, None, 1, 128, 3, 1e-2),
    (1, "cta-bn128-s2-x3", 1, 128, 3, 1e-2),
    (1, "cta-bn64-s2-x4", 1, 128, 3, 1e-2),
    (1, "persistent-bn128", 1, 128, 3, 1e-2),
    (1, "persistent-bn64-tma-state", 1, 128, 3, 1e-2),
    (1, "multistep-stream-tile", 1, 256, 3, 1e-2),
    (1, "multistep-jres-group", 1, 256, 3, 1e-2),
    (3, None, 1, 128, 1, 1e-2),
    (0, "csr-lane4", 2, 64, 3, 1e-5),
    (0, "csr-lane8", 2, 64, 3, 1e-5),
    (1, "csr-lane4", 2, 128, 3, 1e-2),
    (1, "csr-lane8", 2, 128, 3, 1e-2),
    (1, "csr-band8", 2, 128, 3, 1e-2),
]


@pytest.mark.parametrize("precision,kernel,storage,R,nsteps,tol", CASES)
def test_deformed_steps_match_oracle(q, ctx, oracle, precision, kernel, storage, R, nsteps, tol):
    import torch
    fr = synth.batched_blocks(1004, n_blocks=5, n_min=80, n_max=400)
    g = ctx.build_graph(fr, mode=q.MODE_READ, storage=storage)
    og = oracle.read_graph(fr, oracle.READ_SIGNED)
    blocks = oracle.blocks_of(og)
    n_pad, pidx, c0 = g.layout()
    # a field strength per block (a wrong block index shows), strong enough to matter
    field = 0.02 * (1 + np.arange(len(blocks)))
    steps, t0 = 200, 40
    rng = np.random.default_rng(31)
    x = np.zeros((R, n_pad), np.float32)
    y = np.zeros((R, n_pad), np.float32)
    refs = []
    for b, nodes in enumerate(blocks):
        x[:, pidx[nodes]] = rng.uniform(-0.1, 0.1, (R, len(nodes)))
        y[:, pidx[nodes]] = rng.uniform(-0.1, 0.1, (R, len(nodes)))
        sub = og.subgraph(nodes)
        xb = x[:, pidx[nodes]].astype(np.float64)
        yb = y[:, pidx[nodes]].astype(np.float64)
        x1, y1 = oracle.bsb_run(sub, xb, yb, t0, t0 + nsteps, steps, c0=float(c0[b]),
                                h=float(field[b]))
        x0, y0 = oracle.bsb_run(sub, xb, yb, t0, t0 + nsteps, steps, c0=float(c0[b]))
        assert _rel_frob(y1, y0) > 0.05  # the field is visible against the plain step
        refs.append((nodes, x1, y1))
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ctx.debug_steps(g, precision, R, xd, yd, t0, nsteps, steps, c0=c0, step_kernel=kernel,
                    field=field)
    xg, yg = xd.cpu().numpy().astype(np.float64), yd.cpu().numpy().astype(np.float64)
    for nodes, x1, y1 in refs:
        xgb, ygb = xg[:, pidx[nodes]], yg[:, pidx[nodes]]
        free = (np.abs(xgb) < 1.0) & (np.abs(x1) < 1.0)
        assert (~free & (np.abs(xgb) != np.abs(x1))).mean() <= 0.01
        x0 = x[:, pidx[nodes]]
        assert _rel_frob((xgb - x0)[free], (x1 - x0)[free]) <= tol
        assert _rel_frob(ygb[free], y1[free]) <= tol
    pad = np.ones(n_pad, bool)
    pad[pidx[pidx >= 0]] = False
    assert np.all(xg[:, pad] == 0) and np.all(yg[:, pad] == 0)


def _snp_case():
    return synth.region_reads(33, n_snps=400, region=150_000, n_reads=90, len_mean=9000,
                              len_sd=3000, flip_p=0.08, miss_p=0.0, qual=(7, 30))


@pytest.mark.parametrize("precision,storage", [(0, 1), (1, 1), (1, 2)])
def test_deformed_refinement_vs_oracle(q, ctx, oracle, precision, storage):
    fr = _snp_case()
    g = ctx.build_graph(fr, mode=q.MODE_SNP, storage=storage)
    kw = dict(replicas=64, steps=400, precision=precision, seed=6, refine_max=15)
    plain = ctx.solve(g, **kw)
    sol = ctx.solve(g, deform_h=0.02, deform_tries=2, **kw)
    res = oracle.phase_snp(fr, range(64), 400, seed=6, refine_max=15, deform_h=0.02,
                           deform_tries=2)
    og = res["graph"]
    extra = 0
    for b, nodes in enumerate(res["blocks"]):
        sub = og.subgraph(nodes)
        info = sol.block(b, len(nodes))
        p_or = np.where(res["C"][nodes] % 2 == 0, 1, -1).astype(np.int8)
        assert info["best_cut"] == pytest.approx(oracle.cut(sub, info["spins"]), rel=1e-12,
                                                 abs=1e-9)
        assert info["best_cut"] >= 0.999 * oracle.cut(sub, p_or) - 1e-9
        # the deformed refinement follows the plain one up to its first failed solve,
        # then only adds re-solves
        assert info["iterations"] >= plain.block(b)["iterations"]
        extra += info["iterations"] - plain.block(b)["iterations"]
    assert extra > 0  # re-solves happened
    assert res["solves"].sum() > len(res["blocks"])


def test_deform_options_validated(q, ctx):
    fr = _snp_case()
    g = ctx.build_graph(fr, mode=q.MODE_SNP)
    for bad in (dict(deform_h=-0.1, deform_tries=1), dict(deform_h=float("nan"), deform_tries=1),
                dict(deform_h=0.1, deform_tries=-1)):
        with pytest.raises(RuntimeError):
            ctx.solve(g, replicas=64, steps=50, precision=q.PREC_FP32, **bad)
    # read graphs have no refinement: the options are accepted and change nothing
    gr = ctx.build_graph(synth.tiny_reads(1001))
    a = ctx.solve(gr, replicas=64, steps=200, precision=q.PREC_FP32, seed=3)
    b = ctx.solve(gr, replicas=64, steps=200, precision=q.PREC_FP32, seed=3, deform_h=0.5,
                  deform_tries=3)
    assert np.array_equal(a.cuts(), b.cuts())
