"""Multi-step tensor-core kernels (momentum y held in TMEM across steps) against the
FP64 oracle, through the C ABI.

One launch runs a whole range of steps, and the row tiles of a block hand X_hat over
through release/acquire counters.  Bars as for the per-step kernels: the state after
a few steps within 1e-2 (relative Frobenius, BF16 operands) of the oracle's, best
cut >= 0.999 x the oracle's on the same seed, steps and replica indices.
"""
import numpy as np
import pytest

from paper_2603_25762_gb300 import synth

pytestmark = pytest.mark.gpu

MULTI = ["multistep-jres-group", "multistep-stream-tile", "multistep-jres-tile",
         "multistep-stream-group"]


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
    d = np.linalg.norm(a - b)
    n = np.linalg.norm(b)
    return d / n if n > 0 else d


def _state_case(q, ctx, oracle, fr, mode, precision, kernel, R, t0, nsteps, steps=200):
    import torch
    g = ctx.build_graph(fr, mode=mode)
    og = oracle.read_graph(fr, oracle.READ_SIGNED) if mode == q.MODE_READ else oracle.snp_graph(fr)
    blocks = oracle.blocks_of(og)
    n_pad, pidx, c0 = g.layout()
    x = np.zeros((R, n_pad), np.float32)
    y = np.zeros((R, n_pad), np.float32)
    rng = np.random.default_rng(8)
    refs = []
    for b, nodes in enumerate(blocks):
        x[:, pidx[nodes]] = rng.uniform(-0.1, 0.1, (R, len(nodes)))
        y[:, pidx[nodes]] = rng.uniform(-0.1, 0.1, (R, len(nodes)))
        x1, y1 = oracle.bsb_run(og.subgraph(nodes), x[:, pidx[nodes]].astype(np.float64),
                                y[:, pidx[nodes]].astype(np.float64), t0, t0 + nsteps, steps,
                                c0=float(c0[b]))
        refs.append((nodes, x1, y1))
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ctx.debug_steps(g, precision, R, xd, yd, t0, nsteps, steps, c0=c0, step_kernel=kernel)
    xg, yg = xd.cpu().numpy().astype(np.float64), yd.cpu().numpy().astype(np.float64)
    for nodes, x1, y1 in refs:
        xgb, ygb = xg[:, pidx[nodes]], yg[:, pidx[nodes]]
        free = (np.abs(xgb) < 1.0) & (np.abs(x1) < 1.0)
        assert (~free & (np.abs(xgb) != np.abs(x1))).mean() <= 0.01
        x0 = x[:, pidx[nodes]]
        assert _rel_frob((xgb - x0)[free], (x1 - x0)[free]) <= 1e-2
        assert _rel_frob(ygb[free], y1[free]) <= 1e-2
    # padding columns stay untouched
    pad = np.ones(n_pad, bool)
    pad[pidx[pidx >= 0]] = False
    assert np.all(xg[:, pad] == 0) and np.all(yg[:, pad] == 0)
    return g


@pytest.mark.parametrize("kernel", MULTI)
@pytest.mark.parametrize("t0,nsteps", [(50, 3), (51, 4), (0, 1)])
def test_multistep_state_matches_oracle(q, ctx, oracle, kernel, t0, nsteps):
    # several blocks of uneven size: per-block counters, row tiles per block 1..4
    fr = synth.batched_blocks(1004, n_blocks=6, n_min=60, n_max=450)
    _state_case(q, ctx, oracle, fr, q.MODE_READ, q.PREC_BF16, kernel, 256, t0, nsteps)


@pytest.mark.parametrize("kernel", MULTI)
def test_multistep_state_region_many_row_tiles(q, ctx, oracle, kernel):
    # one block spanning many row tiles: every step waits for all of them
    fr = synth.hifi_region(1002, scale=0.12)
    _state_case(q, ctx, oracle, fr, q.MODE_READ, q.PREC_BF16, kernel, 384, 100, 3)


def test_multistep_state_snp_hilo(q, ctx, oracle):
    # real-valued SNP weights with the BF16 hi + lo split of J
    fr = synth.ont_region(1003, scale=0.04)
    _state_case(q, ctx, oracle, fr, q.MODE_SNP, q.PREC_BF16X2, "multistep-stream-tile", 128,
                20, 3)


def _solve_case(q, ctx, oracle, fr, R, steps, seed, kernel, n_oracle=16, **kw):
    g = ctx.build_graph(fr, mode=q.MODE_READ)
    sol = ctx.solve(g, replicas=R, steps=steps, precision=q.PREC_BF16, seed=seed,
                    step_kernel=kernel, **kw)
    og = oracle.read_graph(fr, oracle.READ_SIGNED)
    spins = sol.spins(g.n_nodes)
    cuts = sol.cuts()
    for b, nodes in enumerate(oracle.blocks_of(og)):
        sub = og.subgraph(nodes)
        info = sol.block(b, len(nodes))
        assert info["best_cut"] == oracle.cut(sub, spins[nodes])
        # the GPU's best over the oracle's replica indices (same initial draws)
        best, _, _, _ = oracle.bsb_solve(sub, list(range(n_oracle)), steps, seed, b)
        same = cuts[b][:n_oracle].max()
        assert same >= 0.999 * best, (b, same, best)
    assert sol.timing()["kernel"] == kernel
    return g, sol


@pytest.mark.parametrize("kernel", MULTI)
def test_multistep_solve_tiny(q, ctx, oracle, kernel):
    _solve_case(q, ctx, oracle, synth.tiny_reads(1001), 128, 2000, 11, kernel)


@pytest.mark.parametrize("kernel", MULTI)
def test_multistep_solve_batched_blocks(q, ctx, oracle, kernel):
    fr = synth.batched_blocks(1004, n_blocks=10, n_min=20, n_max=400)
    g, _ = _solve_case(q, ctx, oracle, fr, 128, 600, 5, kernel)
    assert g.n_blocks >= 10


@pytest.mark.parametrize("kernel", MULTI)
def test_multistep_solve_region(q, ctx, oracle, kernel):
    _solve_case(q, ctx, oracle, synth.hifi_region(1002, scale=0.1), 256, 1000, 3, kernel)


@pytest.mark.parametrize("kernel", MULTI)
def test_multistep_early_stop_chunks(q, ctx, kernel):
    fr = synth.tiny_reads(1001)
    g = ctx.build_graph(fr)
    sol = ctx.solve(g, replicas=128, steps=3000, precision=q.PREC_BF16, seed=2, check_every=50,
                    patience=3, step_kernel=kernel)
    runs = [sol.block(b)["steps_run"] for b in range(g.n_blocks)]
    assert all(50 <= r <= 3000 for r in runs)
    assert min(runs) < 3000
    c = sol.cuts()
    for b in range(g.n_blocks):
        assert sol.block(b)["best_cut"] == c[b].max()


def _stop_case(q, ctx, g, R, steps, seed, kernel, check_every, patience, blocks=None):
    """The same early-stopping solve with the checks inside the multi-step launch and
    between launches (separate cut kernels): the trajectories are the same bits, so
    steps_run, every replica's cut, the picks and the spins must agree exactly."""
    kw = dict(replicas=R, steps=steps, precision=q.PREC_BF16, seed=seed,
              check_every=check_every, patience=patience, step_kernel=kernel, blocks=blocks)
    inside = ctx.solve(g, check_mode=0, **kw)
    between = ctx.solve(g, check_mode=1, **kw)
    ti, tb = inside.timing(), between.timing()
    # one launch per wave against one per check period
    assert ti["n_step_launches"] < tb["n_step_launches"]
    assert np.array_equal(inside.cuts(), between.cuts())
    assert np.array_equal(inside.spins(g.n_nodes), between.spins(g.n_nodes))
    runs = []
    for b in range(g.n_blocks):
        bi, bb = inside.block(b), between.block(b)
        for key in ("steps_run", "best_cut", "best_replica"):
            assert bi[key] == bb[key], (b, key, bi[key], bb[key])
        runs.append(bi["steps_run"])
    # the energy-check trace: the same best cut per block and check on both paths, a value
    # up to the check a block stopped at and NaN after it
    (cei, tri), (ceb, trb) = inside.check_trace(), between.check_trace()
    assert cei == ceb == check_every and tri.shape == ((steps - 1) // check_every, g.n_blocks)
    assert np.array_equal(tri, trb, equal_nan=True)
    for b in range(g.n_blocks):
        col = tri[:, b]
        if blocks is not None and b not in blocks:
            assert np.isnan(col).all()
            continue
        n_rec = runs[b] // check_every if runs[b] < steps else col.size
        assert np.isfinite(col[:n_rec]).all() and np.isnan(col[n_rec:]).all(), b
        if runs[b] < steps:  # stopped: its last `patience` checks did not beat the best before
            assert col[n_rec - patience:n_rec].max() <= col[:n_rec - patience].max(), b
    return runs


@pytest.mark.parametrize("kernel", MULTI)
def test_multistep_checks_inside_the_launch_tiny(q, ctx, kernel):
    g = ctx.build_graph(synth.tiny_reads(1001))
    runs = _stop_case(q, ctx, g, 128, 3000, 2, kernel, 50, 3)
    assert min(runs) < 3000 and all(r % 50 == 0 or r == 3000 for r in runs)


@pytest.mark.parametrize("kernel", MULTI)
def test_multistep_checks_inside_the_launch_blocks(q, ctx, kernel):
    # uneven blocks, each deciding on its own
    fr = synth.batched_blocks(1004, n_blocks=10, n_min=20, n_max=400)
    g = ctx.build_graph(fr)
    runs = _stop_case(q, ctx, g, 128, 1200, 5, kernel, 40, 2)
    assert min(runs) < 1200 and all(r % 40 == 0 for r in runs)
    # a partial solve stops the same way
    _stop_case(q, ctx, g, 128, 1200, 5, kernel, 40, 2, blocks=[1, 4, 7])


@pytest.mark.parametrize("kernel", ["multistep-stream-tile", "multistep-stream-group"])
def test_multistep_checks_inside_the_launch_region(q, ctx, kernel):
    # many row tiles of one block: the decision waits on every item of the block
    g = ctx.build_graph(synth.hifi_region(1002, scale=0.1))
    runs = _stop_case(q, ctx, g, 256, 2000, 3, kernel, 25, 2)
    assert min(runs) < 2000


def test_multistep_agrees_with_per_step_kernel(q, ctx):
    # same seed, steps and replicas: the two kernels round differently (y / (dt c0)
    # on chip), so the trajectories separate, but the best cuts are of equal quality
    fr = synth.hifi_region(1002, scale=0.1)
    g = ctx.build_graph(fr)
    a = ctx.solve(g, replicas=256, steps=1000, precision=q.PREC_BF16, seed=3,
                  step_kernel="cta-bn128-s3")
    for k in MULTI:
        b = ctx.solve(g, replicas=256, steps=1000, precision=q.PREC_BF16, seed=3, step_kernel=k)
        for blk in range(g.n_blocks):
            ca, cb = a.block(blk)["best_cut"], b.block(blk)["best_cut"]
            assert cb >= 0.999 * ca and ca >= 0.999 * cb, (k, blk, ca, cb)


def test_multistep_rejects_unfit_cases(q, ctx):
    import torch
    fr = synth.tiny_reads(1001)
    g = ctx.build_graph(fr)
    with pytest.raises(RuntimeError):  # replicas not a multiple of 128
        ctx.solve(g, replicas=64, steps=10, precision=q.PREC_BF16, step_kernel=MULTI[0])
    n_pad, _, c0 = g.layout()
    x = torch.zeros((128, n_pad), dtype=torch.float32, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(RuntimeError):  # dt * c0 = 0 cannot hold y / (dt c0)
        ctx.debug_steps(g, q.PREC_BF16, 128, x, y, 0, 2, 10, c0=np.zeros_like(c0),
                        step_kernel=MULTI[1])


def _wave_case(q, ctx, oracle, kernel, check_blocks):
    import torch
    # 40 blocks of 300-800 reads at R = 512: about 680 items, more than one wave holds
    fr = synth.batched_blocks(1007, n_blocks=40, n_min=300, n_max=800)
    g = ctx.build_graph(fr, mode=q.MODE_READ)
    og = oracle.read_graph(fr, oracle.READ_SIGNED)
    blocks = oracle.blocks_of(og)
    n_pad, pidx, c0 = g.layout()
    R, t0, nsteps, steps = 512, 30, 3, 200
    rng = np.random.default_rng(9)
    x = np.zeros((R, n_pad), np.float32)
    y = np.zeros((R, n_pad), np.float32)
    for nodes in blocks:
        x[:, pidx[nodes]] = rng.uniform(-0.1, 0.1, (R, len(nodes)))
        y[:, pidx[nodes]] = rng.uniform(-0.1, 0.1, (R, len(nodes)))
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ctx.debug_steps(g, q.PREC_BF16, R, xd, yd, t0, nsteps, steps, c0=c0, step_kernel=kernel)
    xg, yg = xd.cpu().numpy().astype(np.float64), yd.cpu().numpy().astype(np.float64)
    for b in check_blocks:
        nodes = blocks[b]
        x1, y1 = oracle.bsb_run(og.subgraph(nodes), x[:, pidx[nodes]].astype(np.float64),
                                y[:, pidx[nodes]].astype(np.float64), t0, t0 + nsteps, steps,
                                c0=float(c0[b]))
        xgb, ygb = xg[:, pidx[nodes]], yg[:, pidx[nodes]]
        free = (np.abs(xgb) < 1.0) & (np.abs(x1) < 1.0)
        assert (~free & (np.abs(xgb) != np.abs(x1))).mean() <= 0.01
        x0 = x[:, pidx[nodes]]
        assert _rel_frob((xgb - x0)[free], (x1 - x0)[free]) <= 1e-2
        assert _rel_frob(ygb[free], y1[free]) <= 1e-2
    return g, blocks


@pytest.mark.parametrize("kernel", MULTI)
def test_multistep_several_waves(q, ctx, oracle, kernel):
    g, blocks = _wave_case(q, ctx, oracle, kernel, [0, 1, 19, 20, 38, 39])
    assert sum(-(-len(b) // 128) for b in blocks) * 4 > 4 * 152  # more than one wave


def test_multistep_several_waves_solve(q, ctx, oracle):
    fr = synth.batched_blocks(1007, n_blocks=40, n_min=300, n_max=800)
    g = ctx.build_graph(fr, mode=q.MODE_READ)
    sol = ctx.solve(g, replicas=512, steps=400, precision=q.PREC_BF16, seed=4,
                    step_kernel="multistep-stream-group")
    og = oracle.read_graph(fr, oracle.READ_SIGNED)
    blocks = oracle.blocks_of(og)
    spins = sol.spins(g.n_nodes)
    cuts = sol.cuts()
    for b in [0, 13, 27, 39]:
        nodes = blocks[b]
        sub = og.subgraph(nodes)
        info = sol.block(b, len(nodes))
        assert info["best_cut"] == oracle.cut(sub, spins[nodes])
        best, _, _, _ = oracle.bsb_solve(sub, list(range(8)), 400, 4, b)
        assert cuts[b][:8].max() >= 0.999 * best, (b, cuts[b][:8].max(), best)


@pytest.mark.parametrize("kernel", ["multistep-stream-tile", "multistep-jres-group"])
def test_step_trace_events_are_ordered(q, ctx, kernel):
    """The tracing hook records every hand-off point of every live (step, item), in
    pipeline order on each SM's clock: accumulator free <= MMAs committed <= epilogue
    start <= epilogue end <= X_hat released; inputs released <= last load issued."""
    fr = synth.hifi_region(1002, scale=0.12)
    g = ctx.build_graph(fr)
    stamps, items = ctx.debug_run_trace(g, 256, kernel, 40, 10, 8)
    live = items >= 0
    assert live.any(axis=1).all()
    c = stamps[..., 16:27].astype(np.int64)
    for cta in range(stamps.shape[0]):
        for sl in np.nonzero(live[cta])[0]:
            ev = c[cta, :, sl]  # [nu, 11]
            assert (ev > 0).all(), (cta, sl)
            assert (ev[:, 8] <= ev[:, 9]).all() and (ev[:, 9] <= ev[:, 0]).all()
            assert (ev[:, 10] <= ev[:, 1]).all()
            assert (ev[:, 2] <= ev[:, 4]).all() and (ev[:, 4] <= ev[:, 5]).all()
            assert (ev[:, 5] <= ev[:, 6]).all() and (ev[:, 6] <= ev[:, 7]).all()
            assert (ev[:, 0] <= ev[:, 1]).all()
        assert (stamps[cta][:, ~live[cta]] == 0).all()
    with pytest.raises(q.QhError):
        ctx.debug_run_trace(g, 256, "cta-bn128-s3", 40, 10, 8)  # not a multi-step kernel
