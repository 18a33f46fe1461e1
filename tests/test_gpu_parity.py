"""GPU path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bars: integer graph weights and cuts bit-exact; SNP-graph weights within 1e-12
relative (FP64 in both, summation in the same fragment order, log10/exp10 from two
math libraries); per-step J x X relative Frobenius error <= 1e-5 (FP32 path) and
<= 1e-2 (BF16 path); best cut >= 0.999 x the oracle's on the same seed, steps and
replica indices.
"""
import numpy as np
import pytest

from paper_2603_25762_gb300 import metrics, synth

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


def _sorted_csr(rp, col, w):
    rows = np.repeat(np.arange(rp.shape[0] - 1), np.diff(rp))
    order = np.lexsort((col, rows))
    return rows[order], col[order], w[order]


def _oracle_edges(g):
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    return rows, g.col.astype(np.int64), g.w


def _small_region(seed=7, scale=0.1, **kw):
    return synth.hifi_region(seed=seed, scale=scale)


# ----------------------------------------------------------------------------- graph build
@pytest.mark.parametrize("make", [lambda: synth.tiny_reads(1001),
                                  lambda: synth.hifi_region(1002, scale=0.08),
                                  lambda: synth.tiny_reads(5, n_snps=60, n_reads=200, flip_p=0.2)])
@pytest.mark.parametrize("mode", [0, 1])
def test_read_graph_bitexact(q, ctx, oracle, make, mode):
    fr = make()
    g = ctx.build_graph(fr, mode=q.MODE_READ, weight_mode=mode)
    r1, c1, w1 = _sorted_csr(*g.edges())
    og = oracle.read_graph(fr, mode)
    r2, c2, w2 = _oracle_edges(og)
    assert np.array_equal(r1, r2) and np.array_equal(c1, c2)
    assert np.array_equal(w1, w2)


@pytest.mark.parametrize("mode", [0, 1])
def test_read_graph_wide_fragments_bitexact(q, ctx, oracle, mode):
    # fragments whose SNPs spread over more than 1,024 SNP indices (linked-read-like
    # spans) take the merge of both SNP lists instead of the allele window
    rng = np.random.default_rng(12)
    n, rows = 6000, []
    for i in range(150):
        k = int(rng.integers(2, 40))
        lo = int(rng.integers(0, n - 3000))
        span = int(rng.choice([200, 3000]))
        rows.append(np.sort(rng.choice(np.arange(lo, lo + span), size=k, replace=False)))
    ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    snp = np.concatenate(rows).astype(np.int32)
    allele = np.where(rng.random(snp.size) < 0.5, 1, -1).astype(np.int8)
    qual = np.full(snp.size, 30, np.uint8)
    fr = synth.Fragments(n, ptr, snp, allele, qual, np.zeros(len(rows), np.uint8),
                         np.arange(n), np.ones(n, np.int8))
    g = ctx.build_graph(fr, mode=q.MODE_READ, weight_mode=mode)
    r1, c1, w1 = _sorted_csr(*g.edges())
    r2, c2, w2 = _oracle_edges(oracle.read_graph(fr, mode))
    assert r1.size > 0
    assert np.array_equal(r1, r2) and np.array_equal(c1, c2) and np.array_equal(w1, w2)


@pytest.mark.parametrize("k", [10, 4])
def test_snp_graph_parity(q, ctx, oracle, k):
    fr = synth.ont_region(1003, scale=0.06)
    g = ctx.build_graph(fr, mode=q.MODE_SNP, linkage_k=k)
    r1, c1, w1 = _sorted_csr(*g.edges())
    og = oracle.snp_graph(fr, 0.1, k)
    r2, c2, w2 = _oracle_edges(og)
    assert np.array_equal(r1, r2) and np.array_equal(c1, c2)
    np.testing.assert_allclose(w1, w2, rtol=1e-12, atol=1e-15)


def test_snp_graph_porec_parity(q, ctx, oracle):
    fr = synth.chromosome_porec(1005, scale=0.004)
    assert fr.is_porec.sum() > 0
    g = ctx.build_graph(fr, mode=q.MODE_SNP, porec_alpha=0.1)
    r1, c1, w1 = _sorted_csr(*g.edges())
    og = oracle.snp_graph(fr, 0.1, 10)
    r2, c2, w2 = _oracle_edges(og)
    assert np.array_equal(r1, r2) and np.array_equal(c1, c2)
    np.testing.assert_allclose(w1, w2, rtol=1e-12, atol=1e-15)


def test_snp_graph_wide_rows_parity(q, ctx, oracle):
    # contacts spanning more than 12,288 SNP indices: those rows take the sorting path
    rng = np.random.default_rng(8)
    n = 30_000
    rows = []
    for i in range(300):
        k = int(rng.integers(2, 7))
        snps = np.sort(rng.choice(n, size=k, replace=False))
        rows.append(snps)
    ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    snp = np.concatenate(rows).astype(np.int32)
    allele = np.where(rng.random(snp.size) < 0.5, 1, -1).astype(np.int8)
    qual = rng.integers(7, 31, size=snp.size).astype(np.uint8)
    porec = (rng.random(len(rows)) < 0.5).astype(np.uint8)
    fr = synth.Fragments(n, ptr, snp, allele, qual, porec, np.arange(n), np.ones(n, np.int8))
    g = ctx.build_graph(fr, mode=q.MODE_SNP, porec_alpha=0.1)
    r1, c1, w1 = _sorted_csr(*g.edges())
    og = oracle.snp_graph(fr, 0.1, 10)
    r2, c2, w2 = _oracle_edges(og)
    assert np.array_equal(r1, r2) and np.array_equal(c1, c2)
    np.testing.assert_allclose(w1, w2, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("mode", ["read", "snp"])
def test_components_match_oracle(q, ctx, oracle, mode):
    fr = synth.region_reads(77, n_snps=800, region=600_000, n_reads=90, len_mean=6000,
                            len_sd=3000, flip_p=0.05, qual=(7, 30))
    if mode == "read":
        g = ctx.build_graph(fr, mode=q.MODE_READ)
        og = oracle.read_graph(fr, oracle.READ_SIGNED)
    else:
        g = ctx.build_graph(fr, mode=q.MODE_SNP)
        og = oracle.snp_graph(fr)
    blocks = oracle.blocks_of(og)
    bo, lo = g.blocks()
    assert g.n_blocks == len(blocks) and g.n_blocks > 1
    exp_b = -np.ones(og.n, np.int32)
    exp_l = np.zeros(og.n, np.int32)
    for b, nodes in enumerate(blocks):
        exp_b[nodes] = b
        exp_l[nodes] = np.arange(len(nodes))
    assert np.array_equal(bo, exp_b)
    assert np.array_equal(lo[exp_b >= 0], exp_l[exp_b >= 0])


def test_invalid_inputs_rejected(q, ctx):
    fr = synth.tiny_reads(3, n_snps=40, n_reads=10)
    bad = synth.Fragments(fr.n_snps, fr.frag_ptr, fr.snp.copy(), fr.allele, fr.qual, fr.is_porec,
                          fr.positions, fr.truth)
    bad.snp[3] = fr.n_snps + 5
    with pytest.raises(q.QhError) as e:
        ctx.build_graph(bad)
    assert e.value.status == q.QH_EINVAL
    bad2 = synth.Fragments(fr.n_snps, fr.frag_ptr, fr.snp, fr.allele.copy(), fr.qual,
                           fr.is_porec, fr.positions, fr.truth)
    bad2.allele[0] = 0
    with pytest.raises(q.QhError):
        ctx.build_graph(bad2)
    bad3 = synth.Fragments(fr.n_snps, fr.frag_ptr, fr.snp, fr.allele, fr.qual.copy(),
                           fr.is_porec, fr.positions, fr.truth)
    bad3.qual[2] = 3
    with pytest.raises(q.QhError):
        ctx.build_graph(bad3, mode=q.MODE_SNP)
    # a fragment range past the end of the entries (frag_ptr not monotone): rejected
    # before any of its entries is read
    fp4 = fr.frag_ptr.copy()
    fp4[1] = fp4[-1] + 40
    bad4 = synth.Fragments(fr.n_snps, fp4, fr.snp, fr.allele, fr.qual, fr.is_porec,
                           fr.positions, fr.truth)
    with pytest.raises(q.QhError) as e:
        ctx.build_graph(bad4)
    assert e.value.status == q.QH_EINVAL
    # the context stays usable after rejected inputs
    g = ctx.build_graph(fr)
    assert g.n_nodes == fr.n_frags


@pytest.mark.parametrize("storage", [1, 2])
def test_empty_and_edgeless_inputs(q, ctx, storage):
    empty = synth.Fragments(10, np.zeros(1, np.int64), np.zeros(0, np.int32),
                            np.zeros(0, np.int8), np.zeros(0, np.uint8), np.zeros(0, np.uint8),
                            np.arange(10), np.ones(10, np.int8))
    lone = synth.Fragments(10, np.array([0, 1, 2, 2], np.int64), np.array([1, 5], np.int32),
                           np.array([1, -1], np.int8), np.array([30, 30], np.uint8),
                           np.zeros(3, np.uint8), np.arange(10), np.ones(10, np.int8))
    # every step path on graphs without blocks: CSR storage adds the band-tile step and
    # an SNP-mode solve with deformed re-solves
    runs = [dict(replicas=64, precision=q.PREC_BF16), dict(replicas=32, precision=q.PREC_FP32)]
    if storage == 2:
        runs.append(dict(replicas=128, precision=q.PREC_BF16, step_kernel="csr-band8"))
    for fr in (empty, lone):
        for mode in (q.MODE_READ, q.MODE_SNP):
            g = ctx.build_graph(fr, mode=mode, storage=storage)
            assert g.n_blocks == 0
            for kw in runs:
                extra = dict(deform_h=0.05, deform_tries=2) if mode == q.MODE_SNP else {}
                sol = ctx.solve(g, steps=10, **kw, **extra)
                h1, h2, bid = ctx.phase(g, sol, 10)
                assert (h1 == 0).all() and (bid == -1).all()


# ----------------------------------------------------------------------------- J x X precision
def _rel_frob(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _matvec_case(q, ctx, oracle, fr, mode, precision, R, dense=False, seed=0, bf16_x=False,
                 storage=0):
    import torch
    if mode == q.MODE_READ:
        g = ctx.build_graph(fr, mode=mode, dense=dense, storage=storage)
        og = oracle.read_graph(fr, oracle.READ_SIGNED)
    else:
        g = ctx.build_graph(fr, mode=mode, dense=dense, storage=storage)
        og = oracle.snp_graph(fr)
    n_pad, pidx, _ = g.layout()
    rng = np.random.default_rng(seed)
    xv = rng.uniform(-1, 1, size=(R, og.n)).astype(np.float32)
    if bf16_x:  # values exactly representable in BF16: only J's representation errs
        import torch
        xv = torch.from_numpy(xv).to(torch.bfloat16).float().numpy()
    x = np.zeros((R, n_pad), np.float32)
    inb = pidx >= 0
    x[:, pidx[inb]] = xv[:, inb]
    xd = torch.from_numpy(x).cuda()
    zd = torch.zeros_like(xd)
    ctx.debug_matvec(g, precision, R, xd, zd)
    z = zd.cpu().numpy()[:, pidx[inb]]
    from scipy.sparse import csr_matrix
    J = -csr_matrix((og.w, og.col, og.row_ptr), shape=(og.n, og.n))
    zref = (J @ xv.astype(np.float64).T).T[:, inb]
    return _rel_frob(z.astype(np.float64), zref)


@pytest.mark.parametrize("dense", [False, True])
def test_matvec_read_graph(q, ctx, oracle, dense):
    fr = synth.hifi_region(1002, scale=0.08)
    e32 = _matvec_case(q, ctx, oracle, fr, q.MODE_READ, q.PREC_FP32, 64, dense)
    e16 = _matvec_case(q, ctx, oracle, fr, q.MODE_READ, q.PREC_BF16, 128, dense)
    assert e32 <= 1e-5, e32
    assert e16 <= 1e-2, e16


def _states_along_schedule(q, ctx, g, R, steps):
    """The solver's own states at t = 0, steps / 2 and steps - 1: the initial draws, then
    FP32 steps (x of the early schedule is small, of the late one mostly at the walls)."""
    import torch
    n_pad = g.layout()[0]
    x = torch.zeros((R, n_pad), dtype=torch.float32, device="cuda")
    y = torch.zeros_like(x)
    ctx.debug_init_state(g, R, x, y, seed=3)
    out, t = [x.cpu().numpy().copy()], 0
    for t1 in (steps // 2, steps - 1):
        ctx.debug_steps(g, q.PREC_FP32, R, x, y, t, t1 - t, steps)
        t = t1
        out.append(x.cpu().numpy().copy())
    return out


@pytest.mark.parametrize("storage", [0, 2])
def test_matvec_along_the_schedule(q, ctx, oracle, storage):
    """J x X at the schedule points the measurement plan samples (t = 0, steps / 2,
    steps - 1), on the solver's own states: relative Frobenius error against FP64
    <= 1e-5 for FP32 and <= 1e-2 for BF16 (and FP8 on tile storage)."""
    import torch
    from scipy.sparse import csr_matrix
    fr = synth.hifi_region(1002, scale=0.1)
    g = ctx.build_graph(fr, storage=storage)
    og = oracle.read_graph(fr, oracle.READ_SIGNED)
    n_pad, pidx, _ = g.layout()
    inb = pidx >= 0
    J = -csr_matrix((og.w, og.col, og.row_ptr), shape=(og.n, og.n))
    R, steps = 128, 1000
    precs = [(q.PREC_FP32, 1e-5), (q.PREC_BF16, 1e-2)]
    if storage == 0:
        precs.append((q.PREC_FP8, 1e-2))
    for k, x in enumerate(_states_along_schedule(q, ctx, g, R, steps)):
        xv = x[:, pidx[inb]].astype(np.float64)
        zref = (J @ xv.T).T[:, inb]
        for prec, bar in precs:
            zd = torch.zeros((R, n_pad), dtype=torch.float32, device="cuda")
            ctx.debug_matvec(g, prec, R, torch.from_numpy(x).cuda(), zd)
            err = _rel_frob(zd.cpu().numpy()[:, pidx[inb]].astype(np.float64), zref)
            assert err <= bar, (k, prec, err)
        if k == 2:
            assert (np.abs(xv) == 1.0).mean() > 0.5  # the late state sits at the walls


@pytest.mark.parametrize("mode", ["read", "snp"])
def test_matvec_fp8(q, ctx, oracle, mode):
    # e4m3 with J and x each split into hi + lo parts: within the 1e-2 bar
    if mode == "read":
        fr, m = synth.hifi_region(1002, scale=0.08), q.MODE_READ
    else:
        fr, m = synth.ont_region(1003, scale=0.06), q.MODE_SNP
    e8 = _matvec_case(q, ctx, oracle, fr, m, q.PREC_FP8, 128)
    assert e8 <= 1e-2, e8


def test_matvec_exact_operands(q, ctx, oracle):
    # integer |w| <= 256 is exact in one BF16 operand; real SNP weights use J = hi + lo
    fr = synth.hifi_region(1002, scale=0.08)
    e_read = _matvec_case(q, ctx, oracle, fr, q.MODE_READ, q.PREC_BF16, 64, bf16_x=True)
    assert e_read <= 1e-6, e_read
    fs = synth.ont_region(1003, scale=0.06)
    e_snp = _matvec_case(q, ctx, oracle, fs, q.MODE_SNP, q.PREC_BF16X2, 64, bf16_x=True)
    assert e_snp <= 3e-5, e_snp
    e_hi = _matvec_case(q, ctx, oracle, fs, q.MODE_SNP, q.PREC_BF16, 64, bf16_x=True)
    assert 3e-5 < e_hi <= 1e-2, e_hi  # hi tiles only: J itself rounded to BF16


def test_matvec_snp_graph_hilo(q, ctx, oracle):
    fr = synth.ont_region(1003, scale=0.06)
    e32 = _matvec_case(q, ctx, oracle, fr, q.MODE_SNP, q.PREC_FP32, 64)
    e16 = _matvec_case(q, ctx, oracle, fr, q.MODE_SNP, q.PREC_BF16, 64)
    e2 = _matvec_case(q, ctx, oracle, fr, q.MODE_SNP, q.PREC_BF16X2, 64)
    assert e32 <= 1e-5, e32
    assert e16 <= 1e-2, e16
    assert e2 <= e16 and e2 <= 1e-2, (e2, e16)


# ----------------------------------------------------------------------------- one bSB step
@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-2), (3, 1e-2)])
def test_steps_match_oracle(q, ctx, oracle, precision, tol, storage):
    if precision == 3 and storage == 2:
        pytest.skip("FP8 runs on tile storage only")
    _steps_case(q, ctx, oracle, precision, tol, storage, 64 if precision != 3 else 128)


@pytest.mark.parametrize("R,kernel", [(12, "csr-lane4"), (24, "csr-lane8"), (64, "csr-lane4"),
                                      (192, "csr-lane8"), (384, "csr-lane8"), (384, "csr-lane4"),
                                      (128, "csr-band8"), (256, "csr-band8")])
@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-2)])
def test_csr_steps_replica_counts(q, ctx, oracle, precision, tol, R, kernel):
    if kernel == "csr-band8" and precision == 0:
        pytest.skip("the band-tile step takes BF16 operands")
    # the CSR step's lane layouts: 4 replicas per lane (R = 384: three passes), and
    # 8 per lane with 8 (R = 24), 2 (R = 192, two passes) and 1 (R = 384, two passes)
    # neighbours per warp at once
    _steps_case(q, ctx, oracle, precision, tol, 2, R, kernel)


def test_csr_variant_rejections(q, ctx):
    import torch
    fr = synth.tiny_reads(1001)
    gc = ctx.build_graph(fr, storage=q.STORAGE_CSR)
    gt = ctx.build_graph(fr)
    with pytest.raises(RuntimeError):  # 8 replicas per lane needs R % 8 == 0
        ctx.solve(gc, replicas=12, steps=10, precision=q.PREC_BF16, step_kernel="csr-lane8")
    with pytest.raises(RuntimeError):  # a CSR variant on tile storage
        ctx.solve(gt, replicas=64, steps=10, precision=q.PREC_BF16, step_kernel="csr-lane4")
    with pytest.raises(RuntimeError):  # a tile variant on CSR storage
        ctx.solve(gc, replicas=64, steps=10, precision=q.PREC_BF16, step_kernel="cta-bn128-s3")
    with pytest.raises(RuntimeError):  # the band-tile step: BF16 operands, R % 128 == 0
        ctx.solve(gc, replicas=128, steps=10, precision=q.PREC_FP32, step_kernel="csr-band8")
    with pytest.raises(RuntimeError):
        ctx.solve(gc, replicas=64, steps=10, precision=q.PREC_BF16, step_kernel="csr-band8")
    n_pad, _, c0 = gc.layout()
    x = torch.zeros((12, n_pad), dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError):
        ctx.debug_steps(gc, q.PREC_FP32, 12, x, torch.zeros_like(x), 0, 1, 10, c0=c0,
                        step_kernel="csr-lane8")
    sol = ctx.solve(gc, replicas=12, steps=10, precision=q.PREC_FP32, step_kernel="csr-lane4")
    assert sol.timing()["kernel"] == "csr-lane4-fp32"


def _steps_case(q, ctx, oracle, precision, tol, storage, R, kernel=None):
    import torch
    fr = synth.hifi_region(1002, scale=0.06)
    g = ctx.build_graph(fr, mode=q.MODE_READ, storage=storage)
    og = oracle.read_graph(fr, oracle.READ_SIGNED)
    blocks = oracle.blocks_of(og)
    n_pad, pidx, c0 = g.layout()
    # FP8's product error (~0.4% per step, within the 1e-2 per-step bar) compounds over
    # steps: its state is compared after one step, the others after three
    steps, nsteps, t0 = 200, (3 if precision != 3 else 1), 50
    x = np.zeros((R, n_pad), np.float32)
    y = np.zeros((R, n_pad), np.float32)
    refs = []
    rng = np.random.default_rng(4)
    # FP32 starts anywhere in the box (walls included); BF16 starts at the solver's
    # initial amplitude, where no element reaches the wall within three steps, so a
    # rounding difference cannot flip a clamp decision
    amp = (0.9, 0.2) if precision == 0 else (0.1, 0.1)
    for b, nodes in enumerate(blocks):
        xb = rng.uniform(-amp[0], amp[0], (R, len(nodes)))
        yb = rng.uniform(-amp[1], amp[1], (R, len(nodes)))
        x[:, pidx[nodes]] = xb
        y[:, pidx[nodes]] = yb
        sub = og.subgraph(nodes)
        x1, y1 = oracle.bsb_run(sub, x[:, pidx[nodes]].astype(np.float64),
                                y[:, pidx[nodes]].astype(np.float64), t0, t0 + nsteps, steps,
                                c0=float(c0[b]))
        refs.append((nodes, x1, y1))
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ctx.debug_steps(g, precision, R, xd, yd, t0, nsteps, steps, c0=c0, step_kernel=kernel)
    xg, yg = xd.cpu().numpy(), yd.cpu().numpy()
    for nodes, x1, y1 in refs:
        xgb, ygb = xg[:, pidx[nodes]].astype(np.float64), yg[:, pidx[nodes]].astype(np.float64)
        # an element whose last update lands within rounding of the wall may clamp on one
        # side only; compare the elements that neither side clamped, count the others
        free = (np.abs(xgb) < 1.0) & (np.abs(x1) < 1.0)
        assert (~free & (np.abs(xgb) != np.abs(x1))).mean() <= 0.01
        dx = (xgb - x[:, pidx[nodes]])[free]
        dxr = (x1 - x[:, pidx[nodes]])[free]
        assert _rel_frob(dx, dxr) <= tol
        assert _rel_frob(ygb[free], y1[free]) <= tol


# ----------------------------------------------------------------------------- full solve
def _check_solve(q, ctx, oracle, fr, precision, R, steps, seed, n_oracle=None, storage=0,
                 step_kernel=None):
    g = ctx.build_graph(fr, mode=q.MODE_READ, storage=storage)
    sol = ctx.solve(g, replicas=R, steps=steps, precision=precision, seed=seed,
                    step_kernel=step_kernel)
    og = oracle.read_graph(fr, oracle.READ_SIGNED)
    blocks = oracle.blocks_of(og)
    spins = sol.spins(g.n_nodes)
    n_or = n_oracle or R
    ridx = list(range(n_or))
    cuts = sol.cuts()
    for b, nodes in enumerate(blocks):
        sub = og.subgraph(nodes)
        info = sol.block(b, len(nodes))
        # exact cut evaluation of the GPU's chosen spins
        assert info["best_cut"] == oracle.cut(sub, spins[nodes])
        assert np.array_equal(info["spins"], spins[nodes])
        assert info["best_cut"] == cuts[b].max()
        # same seed, steps and replica indices on both sides: the GPU's best over the
        # oracle's replicas (identical initial draws), not over its larger R
        best, _, _, _ = oracle.bsb_solve(sub, ridx, steps, seed, b)
        same = cuts[b][:n_or].max()
        assert same >= 0.999 * best, (b, same, best)
    return g, sol


@pytest.mark.parametrize("precision", [0, 1, 3])
def test_solve_tiny_vs_oracle(q, ctx, oracle, precision):
    fr = synth.tiny_reads(1001)
    R = 32 if precision == 0 else 64
    _check_solve(q, ctx, oracle, fr, precision, R, 2000, seed=11)


@pytest.mark.parametrize("precision", [0, 1, 3])
def test_solve_region_vs_oracle(q, ctx, oracle, precision):
    fr = synth.hifi_region(1002, scale=0.1)
    _check_solve(q, ctx, oracle, fr, precision, 128, 1000, seed=3, n_oracle=16)


def test_batched_blocks_vs_oracle(q, ctx, oracle):
    fr = synth.batched_blocks(1004, n_blocks=10, n_min=20, n_max=400)
    g, sol = _check_solve(q, ctx, oracle, fr, q.PREC_BF16, 64, 600, seed=5, n_oracle=16)
    assert g.n_blocks >= 10


def test_solution_cuts_are_exact_and_deterministic(q, ctx, oracle):
    fr = synth.tiny_reads(1001)
    g = ctx.build_graph(fr)
    s1 = ctx.solve(g, replicas=64, steps=500, precision=q.PREC_BF16, seed=9)
    s2 = ctx.solve(g, replicas=64, steps=500, precision=q.PREC_BF16, seed=9)
    assert np.array_equal(s1.cuts(), s2.cuts())
    assert np.array_equal(s1.spins(g.n_nodes), s2.spins(g.n_nodes))
    c = s1.cuts()
    for b in range(g.n_blocks):
        info = s1.block(b)
        assert info["best_cut"] == c[b].max()
        assert info["best_replica"] == int(np.argmax(c[b]))


# ----------------------------------------------------------------------------- bSB setup
def _init_state_case(q, ctx, oracle, g, og, R, base, seed, it):
    import torch
    n_pad, pidx, _ = g.layout()
    x = torch.full((R, n_pad), float("nan"), dtype=torch.float32, device="cuda")
    y = torch.full_like(x, float("nan"))
    ctx.debug_init_state(g, R, x, y, replica_base=base, seed=seed, it=it)
    xg, yg = x.cpu().numpy(), y.cpu().numpy()
    pad = np.ones(n_pad, bool)
    pad[pidx[pidx >= 0]] = False
    assert np.all(xg[:, pad] == 0) and np.all(yg[:, pad] == 0)
    for b, nodes in enumerate(oracle.blocks_of(og)):
        xo, yo = oracle.bsb_init(len(nodes), list(range(base, base + R)), seed, b, it)
        # drawn in FP64, rounded once to FP32 on the GPU: bit-identical after that rounding
        assert np.array_equal(xg[:, pidx[nodes]], xo.astype(np.float32)), b
        assert np.array_equal(yg[:, pidx[nodes]], yo.astype(np.float32)), b


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("base,it", [(0, 0), (64, 0), (3, 5)])
def test_init_state_matches_oracle_draws(q, ctx, oracle, storage, base, it):
    """The initial x, y of every replica equal the oracle's SplitMix64 draws bit for bit
    (after the one FP32 rounding), keyed by block, refinement iteration and the global
    replica index, so a replica range starting at replica_base is the oracle's range."""
    fr = synth.batched_blocks(1004, n_blocks=5, n_min=30, n_max=300)
    g = ctx.build_graph(fr, storage=storage)
    og = oracle.read_graph(fr, oracle.READ_SIGNED)
    _init_state_case(q, ctx, oracle, g, og, 64, base, seed=1234567, it=it)


def test_init_state_snp_graph(q, ctx, oracle):
    fr = synth.ont_region(1003, scale=0.05)
    g = ctx.build_graph(fr, mode=q.MODE_SNP)
    _init_state_case(q, ctx, oracle, g, oracle.snp_graph(fr), 32, 0, seed=9, it=2)


@pytest.mark.parametrize("mode", ["read", "snp"])
def test_default_c0_matches_oracle(q, ctx, oracle, mode):
    """The default coupling scale c0 = 0.5 / (sigma sqrt(N)) of every block, from the
    GPU's block sums (FP64), against the oracle's per-block sums."""
    if mode == "read":
        fr = synth.batched_blocks(1004, n_blocks=6, n_min=40, n_max=500)
        g, og = ctx.build_graph(fr), oracle.read_graph(fr, oracle.READ_SIGNED)
    else:
        fr = synth.ont_region(1003, scale=0.06)
        g, og = ctx.build_graph(fr, mode=q.MODE_SNP), oracle.snp_graph(fr)
    _, _, c0 = g.layout()
    blocks = oracle.blocks_of(og)
    assert len(blocks) == g.n_blocks
    for b, nodes in enumerate(blocks):
        ref = oracle.default_c0(og.subgraph(nodes))
        assert c0[b] == pytest.approx(ref, rel=1e-12), b


# ----------------------------------------------------------------------------- early stop
@pytest.mark.parametrize("precision,R", [(0, 32), (1, 64)])
def test_early_stop_steps_run_matches_oracle(q, ctx, oracle, precision, R):
    """Early stop on a stalled best energy (check every 50 steps, patience 3): each
    block stops after exactly the oracle's number of steps on the same replicas, and
    its best cut is the oracle's to 0.999."""
    fr = synth.tiny_reads(1001)
    g = ctx.build_graph(fr)
    steps, seed, ce, pat = 3000, 2, 50, 3
    sol = ctx.solve(g, replicas=R, steps=steps, precision=precision, seed=seed, check_every=ce,
                    patience=pat)
    og = oracle.read_graph(fr, oracle.READ_SIGNED)
    spins = sol.spins(g.n_nodes)
    for b, nodes in enumerate(oracle.blocks_of(og)):
        sub = og.subgraph(nodes)
        best, _, _, _, sr = oracle.bsb_solve_early_stop(sub, list(range(R)), steps, seed, ce,
                                                        pat, block=b)
        info = sol.block(b)
        assert sr < steps
        assert info["steps_run"] == sr, (b, info["steps_run"], sr)
        assert info["best_cut"] == oracle.cut(sub, spins[nodes])
        assert info["best_cut"] >= 0.999 * best


def test_check_trace_matches_oracle(q, ctx, oracle):
    """The energy-check trace (Results: the energy against the iterations) at FP32: each
    check's best cut over the replicas equals the oracle's, whose replicas are advanced
    check by check and cut-evaluated exactly (same seed, steps and replica indices)."""
    fr = synth.tiny_reads(1001)
    g = ctx.build_graph(fr)
    R, steps, seed, ce = 32, 600, 2, 50
    sol = ctx.solve(g, replicas=R, steps=steps, precision=q.PREC_FP32, seed=seed,
                    check_every=ce, patience=1000)  # checks on, no block stops
    got_ce, tr = sol.check_trace()
    assert got_ce == ce and tr.shape == ((steps - 1) // ce, g.n_blocks)
    og = oracle.read_graph(fr, oracle.READ_SIGNED)
    for b, nodes in enumerate(oracle.blocks_of(og)):
        sub = og.subgraph(nodes)
        x, y = oracle.bsb_init(sub.n, list(range(R)), seed, b)
        t = 0
        for c in range(tr.shape[0]):
            x, y = oracle.bsb_run(sub, x, y, t, (c + 1) * ce, steps)
            t = (c + 1) * ce
            best = max(oracle.cut(sub, np.where(x[r] >= 0, 1, -1).astype(np.int8))
                       for r in range(R))
            assert tr[c, b] == pytest.approx(best, rel=1e-3), (b, c, tr[c, b], best)


@pytest.mark.parametrize("precision,R,pat,kernel", [(0, 32, 0, None), (0, 32, 3, None),
                                                     (1, 64, 0, None),
                                                     (1, 128, 3, "multistep-stream-tile")])
def test_track_best_matches_oracle(q, ctx, oracle, precision, R, pat, kernel):
    """The best result during the run (checks every 25 steps, with and without early
    stop): the GPU keeps a best cut of at least 0.999 x the oracle's kept one on the
    same replicas, its spins give exactly that cut, it is never below the final
    state's, the final state's per-replica cuts are still reported, and early stop
    comes at the oracle's step."""
    fr = synth.tiny_reads(1001)
    g = ctx.build_graph(fr)
    steps, seed, ce = 1500, 2, 25
    kw = dict(replicas=R, steps=steps, precision=precision, seed=seed, check_every=ce,
              patience=pat, step_kernel=kernel)
    sol = ctx.solve(g, track_best=True, **kw)
    fin = ctx.solve(g, **kw)
    og = oracle.read_graph(fr, oracle.READ_SIGNED)
    spins = sol.spins(g.n_nodes)
    assert np.array_equal(sol.cuts(), fin.cuts())
    for b, nodes in enumerate(oracle.blocks_of(og)):
        sub = og.subgraph(nodes)
        best, _, _, _, sr = oracle.bsb_solve_early_stop(sub, list(range(R)), steps, seed, ce,
                                                        pat, block=b, track_best=True)
        info, ref = sol.block(b), fin.block(b)
        assert info["steps_run"] == ref["steps_run"]
        if precision == 0 or kernel is None:
            assert info["steps_run"] == sr, (b, info["steps_run"], sr)
        assert info["best_cut"] == oracle.cut(sub, spins[nodes])
        assert info["best_cut"] >= ref["best_cut"]
        assert info["best_cut"] >= 0.999 * best, (b, info["best_cut"], best)


def _two_schedule_fragments():
    """One block of more than 5,000 reads (AUTO schedule: 1,000 steps) and one small
    block (500 steps) on disjoint SNPs."""
    big = synth.region_reads(77, n_snps=9000, region=3_000_000, n_reads=5200)
    small = synth.tiny_reads(1001)
    ptr = np.concatenate([big.frag_ptr, small.frag_ptr[1:] + big.frag_ptr[-1]])
    return synth.Fragments(big.n_snps + small.n_snps, ptr.astype(np.int64),
                           np.concatenate([big.snp, small.snp + big.n_snps]).astype(np.int32),
                           np.concatenate([big.allele, small.allele]),
                           np.concatenate([big.qual, small.qual]),
                           np.zeros(ptr.shape[0] - 1, np.uint8),
                           np.concatenate([big.positions, small.positions + 4_000_000]),
                           np.concatenate([big.truth, small.truth]))


def test_early_stop_respects_each_block_schedule(q, ctx, oracle):
    """AUTO schedule with blocks of 500 and 1,000 steps: the short block is checked only
    while its own schedule runs, as in the oracle (patience 12 cannot be reached in its
    nine checks, so it runs all 500 steps)."""
    fr = _two_schedule_fragments()
    g = ctx.build_graph(fr)
    sizes = g.block_sizes()
    assert sorted(sizes)[-1] >= 5000 and sorted(sizes)[0] < 5000
    sol = ctx.solve(g, replicas=64, precision=q.PREC_BF16, seed=4, schedule=q.SCHED_AUTO,
                    check_every=50, patience=12)
    og = oracle.read_graph(fr, oracle.READ_SIGNED)
    for b, nodes in enumerate(oracle.blocks_of(og)):
        info = sol.block(b)
        if len(nodes) >= 5000:
            assert info["steps_run"] <= 1000
            continue
        _, _, _, _, sr = oracle.bsb_solve_early_stop(og.subgraph(nodes), list(range(64)), 500,
                                                     4, 50, 12, block=b)
        assert sr == 500
        assert info["steps_run"] == sr, (b, info["steps_run"])


def test_auto_schedule_steps(q, ctx):
    fr = synth.tiny_reads(1001)
    g = ctx.build_graph(fr)
    sol2 = ctx.solve(g, replicas=64, precision=q.PREC_FP32, seed=2, schedule=q.SCHED_AUTO)
    assert all(sol2.block(b)["steps_run"] == 500 for b in range(g.n_blocks))


# ----------------------------------------------------------------------------- CSR storage
@pytest.mark.parametrize("mode", ["read", "snp"])
def test_csr_storage_matvec(q, ctx, oracle, mode):
    if mode == "read":
        fr, m = synth.hifi_region(1002, scale=0.08), q.MODE_READ
    else:
        fr, m = synth.ont_region(1003, scale=0.06), q.MODE_SNP
    e32 = _matvec_case(q, ctx, oracle, fr, m, q.PREC_FP32, 64, storage=q.STORAGE_CSR)
    e16 = _matvec_case(q, ctx, oracle, fr, m, q.PREC_BF16, 64, storage=q.STORAGE_CSR)
    assert e32 <= 1e-5, e32
    assert e16 <= 1e-2, e16


def test_csr_band_matvec_exact_on_bf16_inputs(q, ctx, oracle):
    # integer read weights (exact in BF16) and x exact in BF16: the band product on the
    # tensor cores plus the remainder leave only FP32 accumulation error
    fr = synth.hifi_region(1002, scale=0.1)
    for R in (128, 256):
        e = _matvec_case(q, ctx, oracle, fr, q.MODE_READ, q.PREC_BF16, R, bf16_x=True,
                         storage=q.STORAGE_CSR)
        assert e <= 1e-6, (R, e)


def test_csr_band_split_covers_every_entry(q, ctx):
    # band (three tiles per row tile) + remainder = the stored entries, on a graph with
    # long-range contacts; the default BF16 step at R = 128 is the band-tile step
    fr = synth.chromosome_porec(1005, scale=0.03)
    g = ctx.build_graph(fr, mode=q.MODE_SNP, storage=q.STORAGE_CSR)
    sol = ctx.solve(g, replicas=128, steps=20, precision=q.PREC_BF16, seed=1, refine_max=1)
    assert sol.timing()["kernel"] == "csr-band8-bf16"
    sol64 = ctx.solve(g, replicas=64, steps=20, precision=q.PREC_BF16, seed=1, refine_max=1)
    assert sol64.timing()["kernel"] == "csr-lane8-bf16"


@pytest.mark.parametrize("R", [12, 24, 192, 384])
def test_csr_matvec_replica_counts(q, ctx, oracle, R):
    fr = synth.ont_region(1003, scale=0.06)
    e32 = _matvec_case(q, ctx, oracle, fr, q.MODE_SNP, q.PREC_FP32, R, storage=q.STORAGE_CSR)
    e16 = _matvec_case(q, ctx, oracle, fr, q.MODE_SNP, q.PREC_BF16, R, storage=q.STORAGE_CSR)
    assert e32 <= 1e-5, e32
    assert e16 <= 1e-2, e16


@pytest.mark.parametrize("kernel", [None, "csr-lane4", "csr-lane8", "csr-band8"])
@pytest.mark.parametrize("precision", [0, 1])
def test_csr_storage_solve_vs_oracle(q, ctx, oracle, precision, kernel):
    if kernel == "csr-band8" and precision == 0:
        pytest.skip("the band-tile step takes BF16 operands")
    _check_solve(q, ctx, oracle, synth.tiny_reads(1001), precision,
                 128 if kernel == "csr-band8" else 64, 2000, seed=11,
                 storage=q.STORAGE_CSR, step_kernel=kernel)
    g, sol = _check_solve(q, ctx, oracle, synth.hifi_region(1002, scale=0.1), precision, 128,
                          1000, seed=3, n_oracle=16, storage=q.STORAGE_CSR, step_kernel=kernel)
    assert g.n_tiles == 0 and sol.timing()["kernel"].startswith(kernel or "csr-")


def test_csr_storage_early_stop(q, ctx):
    fr = synth.tiny_reads(1001)
    g = ctx.build_graph(fr, storage=q.STORAGE_CSR)
    for prec in (0, 1):
        sol = ctx.solve(g, replicas=64, steps=3000, precision=prec, seed=2, check_every=50,
                        patience=3)
        runs = [sol.block(b)["steps_run"] for b in range(g.n_blocks)]
        assert all(50 <= r <= 3000 for r in runs) and min(runs) < 3000


@pytest.mark.parametrize("precision,R,kernel", [(0, 64, None), (1, 64, None),
                                                (1, 128, "csr-band8")])
def test_csr_storage_snp_refinement(q, ctx, oracle, precision, R, kernel):
    # the band-tile step refreshes its band tiles and remainder after each sign inversion
    # (its case spans four row tiles, so off-diagonal band tiles are in play)
    if kernel == "csr-band8":
        fr = synth.region_reads(32, n_snps=400, region=140_000, n_reads=100, len_mean=8000,
                                len_sd=2000, flip_p=0.08, miss_p=0.0, qual=(7, 30))
    else:
        fr = synth.region_reads(32, n_snps=150, region=50_000, n_reads=40, len_mean=8000,
                                len_sd=2000, flip_p=0.08, miss_p=0.0, qual=(7, 30))
    g = ctx.build_graph(fr, mode=q.MODE_SNP, storage=q.STORAGE_CSR)
    sol = ctx.solve(g, replicas=R, steps=300, precision=precision, seed=6, refine_max=15,
                    step_kernel=kernel)
    res = oracle.phase_snp(fr, range(R), 300, seed=6, refine_max=15)
    og = res["graph"]
    for b, nodes in enumerate(res["blocks"]):
        sub = og.subgraph(nodes)
        info = sol.block(b, len(nodes))
        p_or = np.where(res["C"][nodes] % 2 == 0, 1, -1).astype(np.int8)
        assert info["best_cut"] == pytest.approx(oracle.cut(sub, info["spins"]), rel=1e-12, abs=1e-9)
        assert info["best_cut"] >= 0.999 * oracle.cut(sub, p_or) - 1e-9


@pytest.mark.parametrize("storage", [1, 2])
def test_rebuilt_graphs_never_replay_stale_loops(q, ctx, storage):
    # the captured step loop is reused only while every pointer it bakes in is unchanged:
    # rebuild the same input with device allocations in between (addresses shift), with
    # the early-stop cut kernels inside the loop, and expect identical results
    import torch
    fr = synth.hifi_region(1002, scale=0.06)
    ref, pads = None, []
    for i in range(4):
        pads.append(torch.empty((i + 1) * 3_000_000, dtype=torch.uint8, device="cuda"))
        g = ctx.build_graph(fr, storage=storage)
        pads.append(torch.empty(1_000_000 * (4 - i), dtype=torch.uint8, device="cuda"))
        sol = ctx.solve(g, replicas=64, steps=200, precision=q.PREC_BF16, seed=4, check_every=40,
                        patience=50)
        cuts = sol.cuts()
        sol.free()
        g.free()
        if ref is None:
            ref = cuts
        assert np.array_equal(cuts, ref), i


def test_chromosome_porec_picks_csr(q, ctx):
    fr = synth.chromosome_porec(1005, scale=0.5)
    g = ctx.build_graph(fr, mode=q.MODE_SNP, porec_alpha=0.1)
    assert g.n_tiles == 0, "long-range contacts scatter over most tiles: CSR expected"
    assert g.n_blocks >= 1 and g.block_sizes().max() > 0.9 * fr.n_snps
    sol = ctx.solve(g, replicas=64, steps=50, precision=q.PREC_BF16, seed=1, refine_max=1)
    h1, h2, bid = ctx.phase(g, sol, fr.n_snps)
    assert sol.timing()["kernel"] == "csr-lane8-bf16"
    assert (h1 != 0).mean() > 0.9


# ----------------------------------------------------------------------------- phase
@pytest.mark.parametrize("precision", [0, 1])
def test_phase_read_matches_oracle_and_truth(q, ctx, oracle, precision):
    fr = synth.tiny_reads(21, flip_p=0.0)
    g = ctx.build_graph(fr)
    sol = ctx.solve(g, replicas=64, steps=1000, precision=precision, seed=3)
    h1, h2, bid = ctx.phase(g, sol, fr.n_snps)
    se, he = metrics.switch_hamming(h1, bid, fr.truth)
    assert se == 0.0 and he == 0.0
    assert np.array_equal(h2, -h1)
    # voting on the GPU's spins equals the oracle's voting on the same spins
    bo, _ = g.blocks()
    oh1, osb = oracle.vote(fr, sol.spins(g.n_nodes), bo, g.n_blocks)
    assert np.array_equal(h1, oh1) and np.array_equal(bid, osb)


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_phase_snp_refinement(q, ctx, oracle, precision):
    fr = synth.region_reads(31, n_snps=150, region=50_000, n_reads=50, len_mean=8000,
                            len_sd=2000, flip_p=0.0, miss_p=0.0, qual=(10, 30))
    g = ctx.build_graph(fr, mode=q.MODE_SNP)
    sol = ctx.solve(g, replicas=64, steps=300, precision=precision, seed=5, refine_max=15)
    h1, h2, bid = ctx.phase(g, sol, fr.n_snps)
    se, he = metrics.switch_hamming(h1, bid, fr.truth)
    assert se == 0.0 and he == 0.0
    # noisy input: the parity partition's cut matches the oracle's refinement within 0.999
    fr2 = synth.region_reads(32, n_snps=150, region=50_000, n_reads=40, len_mean=8000,
                             len_sd=2000, flip_p=0.08, miss_p=0.0, qual=(7, 30))
    g2 = ctx.build_graph(fr2, mode=q.MODE_SNP)
    sol2 = ctx.solve(g2, replicas=64, steps=300, precision=precision, seed=6, refine_max=15)
    res = oracle.phase_snp(fr2, range(64), 300, seed=6, refine_max=15)
    og = res["graph"]
    for b, nodes in enumerate(res["blocks"]):
        sub = og.subgraph(nodes)
        p_or = np.where(res["C"][nodes] % 2 == 0, 1, -1).astype(np.int8)
        info = sol2.block(b, len(nodes))
        p_gpu = info["spins"]
        assert info["best_cut"] == pytest.approx(oracle.cut(sub, p_gpu), rel=1e-12, abs=1e-9)
        assert info["best_cut"] >= 0.999 * oracle.cut(sub, p_or) - 1e-9
        assert info["best_cut"] >= 0.999 * res["first_cuts"][b] - 1e-9


# ----------------------------------------------------------------------------- full size
@pytest.mark.slow
def test_full_size_hifi_region(q, ctx, oracle):
    """The 7,200-read / 12,000-SNP workload at 1,024 replicas: exact graph, BF16 and FP32
    J x X precision on all rows, and exact cut evaluation of the solve's spins."""
    fr = synth.hifi_region(1002)
    g = ctx.build_graph(fr)
    og = oracle.read_graph(fr, oracle.READ_SIGNED)
    r1, c1, w1 = _sorted_csr(*g.edges())
    r2, c2, w2 = _oracle_edges(og)
    assert np.array_equal(c1, c2) and np.array_equal(w1, w2)
    e16 = _matvec_case(q, ctx, oracle, fr, q.MODE_READ, q.PREC_BF16, 1024)
    e32 = _matvec_case(q, ctx, oracle, fr, q.MODE_READ, q.PREC_FP32, 256)
    assert e16 <= 1e-2 and e32 <= 1e-5
    sol = ctx.solve(g, replicas=1024, steps=1000, precision=q.PREC_BF16, seed=1)
    spins = sol.spins(g.n_nodes)
    for b, nodes in enumerate(oracle.blocks_of(og)):
        sub = og.subgraph(nodes)
        info = sol.block(b)
        assert info["best_cut"] == oracle.cut(sub, spins[nodes])


def test_real_weight_cuts_match_fp64(q, ctx, oracle):
    # SNP weights are real: the many-replica pick sums them in compensated FP32, the
    # reported cut is the FP64 cut of the partition.  With one refinement iteration the
    # partition is the picked replica's spins, so the two must agree to ~1e-11.
    fr = synth.ont_region(1003, scale=0.04)
    g = ctx.build_graph(fr, mode=q.MODE_SNP)
    sol = ctx.solve(g, replicas=128, steps=300, precision=q.PREC_BF16, seed=6, refine_max=1)
    og = oracle.snp_graph(fr)
    spins = sol.spins(g.n_nodes)
    c = sol.cuts()
    for b, nodes in enumerate(oracle.blocks_of(og)):
        info = sol.block(b, len(nodes))
        exact = oracle.cut(og.subgraph(nodes), spins[nodes])
        assert info["best_cut"] == pytest.approx(exact, rel=1e-12, abs=1e-9)
        picked = c[b][info["best_replica"]]
        assert picked == c[b].max()
        if picked <= 0:  # the refinement test stops before flipping: no partition
            continue
        assert picked == pytest.approx(exact, rel=1e-10, abs=1e-8)


# ----------------------------------------------------------------------------- failure detection
@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_expires_and_context_survives(q, ctx, oracle, which):
    # a wait that nothing completes (an mbarrier phase, a release counter) gives up
    # after about a second with QH_ETIMEOUT; the next call on the context works
    import time
    t0 = time.perf_counter()
    with pytest.raises(q.QhError) as e:
        ctx.debug_wait_timeout(which)
    assert e.value.status == 4  # QH_ETIMEOUT
    assert 0.2 < time.perf_counter() - t0 < 30
    _check_solve(q, ctx, oracle, synth.tiny_reads(1001), q.PREC_BF16, 64, 500, seed=11)


# ----------------------------------------------------------------------------- sharding
@pytest.mark.parametrize("precision,kernel,R", [(0, None, 32), (1, "cta-bn64-s2-x4", 64),
                                                (1, "multistep-stream-tile", 128)])
def test_replica_ranges_combine_to_one_solve(q, ctx, precision, kernel, R):
    """Replica sharding: replicas base .. base + R - 1 of a solve at replica_base are
    exactly those replicas of one solve over 2R (same draws, same per-replica
    arithmetic), and the cross-rank pick over the two halves is that solve's pick."""
    from paper_2603_25762_gb300 import multi
    fr = synth.batched_blocks(1004, n_blocks=4, n_min=60, n_max=400)
    g = ctx.build_graph(fr)
    kw = dict(steps=400, precision=precision, seed=8, step_kernel=kernel)
    full = ctx.solve(g, replicas=2 * R, **kw)
    halves = [ctx.solve(g, replicas=R, replica_base=base, **kw) for base in (0, R)]
    cf = full.cuts()
    assert np.array_equal(halves[0].cuts(), cf[:, :R])
    assert np.array_equal(halves[1].cuts(), cf[:, R:])
    C = np.array([[h.block(b)["best_cut"] for b in range(g.n_blocks)] for h in halves])
    P = np.array([[h.block(b)["best_replica"] for b in range(g.n_blocks)] for h in halves])
    owner = multi.pick_best(C, P)
    for b in range(g.n_blocks):
        ref = full.block(b)
        assert C[owner[b], b] == ref["best_cut"] and P[owner[b], b] == ref["best_replica"]


def _block_subset_case(q, ctx, fr, mode, **kw):
    from paper_2603_25762_gb300 import multi
    g = ctx.build_graph(fr, mode=mode)
    sizes = g.block_sizes()
    full = ctx.solve(g, **kw)
    shards = multi.block_shards(sizes, 2, kw["replicas"])
    assert shards[0] and shards[1]
    part = [ctx.solve(g, blocks=s, **kw) for s in shards]
    # before the exchange: each part has its own blocks only
    h1p, _, bidp = ctx.phase(g, part[0], fr.n_snps)
    for b in shards[1]:
        info = part[0].block(b, int(sizes[b]))
        assert info["best_replica"] == -1 and info["steps_run"] == 0
        assert not np.any(info["spins"])
        assert not np.any(bidp == b)
    # import the other part's blocks, as the all-gather of a sharded run does
    for b in shards[1]:
        r = part[1].block(b, int(sizes[b]))
        part[0].set_block(b, r["spins"], r["best_cut"], r["best_replica"], r["steps_run"],
                          r["iterations"])
    for b in range(g.n_blocks):
        a, ref = part[0].block(b, int(sizes[b])), full.block(b, int(sizes[b]))
        for key in ("best_cut", "best_replica", "steps_run", "iterations"):
            assert a[key] == ref[key], (b, key)
        assert np.array_equal(a["spins"], ref["spins"]), b
    h1, h2, bid = ctx.phase(g, part[0], fr.n_snps)
    r1, r2, rbid = ctx.phase(g, full, fr.n_snps)
    assert np.array_equal(h1, r1) and np.array_equal(h2, r2) and np.array_equal(bid, rbid)
    return g


@pytest.mark.parametrize("kernel", ["cta-bn128-s3", "multistep-stream-group",
                                    "multistep-jres-tile"])
def test_block_subsets_combine_to_the_full_solve_read(q, ctx, kernel):
    """Block sharding: two disjoint block subsets (split by cost), solved separately and
    merged with qh_solution_set_block, give exactly the full solve and its phasing."""
    fr = synth.batched_blocks(1004, n_blocks=7, n_min=40, n_max=420)
    _block_subset_case(q, ctx, fr, q.MODE_READ, replicas=128, steps=300, precision=q.PREC_BF16,
                       seed=5, step_kernel=kernel)


def test_block_subsets_combine_to_the_full_solve_snp(q, ctx):
    fr = synth.batched_blocks(1004, n_blocks=5, n_min=30, n_max=200)
    _block_subset_case(q, ctx, fr, q.MODE_SNP, replicas=32, steps=300, precision=q.PREC_FP32,
                       seed=5, refine_max=4)


def test_block_subset_arguments_checked(q, ctx):
    fr = synth.batched_blocks(1004, n_blocks=3, n_min=40, n_max=100)
    g = ctx.build_graph(fr)
    for bad in ([0, 0], [g.n_blocks], [-1]):
        with pytest.raises(q.QhError) as e:
            ctx.solve(g, replicas=64, steps=10, precision=q.PREC_BF16, blocks=bad)
        assert e.value.status == q.QH_EINVAL
    empty = ctx.solve(g, replicas=64, steps=10, precision=q.PREC_BF16, blocks=[])
    _, _, bid = ctx.phase(g, empty, fr.n_snps)
    assert np.all(bid == -1)
    with pytest.raises(q.QhError):
        empty.set_block(0, np.zeros(g.block_sizes()[0], np.int8), 1.0, 0, 10, 1)  # spins 0
