"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

No GPU: these run on the CPU and check the oracle itself (hand-worked examples,
closed forms, brute force, an independent ODE integration, library routines).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from paper_2603_25762_gb300 import metrics, synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _frags_from_M(M, qual=None, porec=None):
    M = np.asarray(M)
    ptr, snp, al, q = [0], [], [], []
    for i, row in enumerate(M):
        nz = np.nonzero(row)[0]
        snp += nz.tolist()
        al += row[nz].tolist()
        q += ([30] * nz.size) if qual is None else list(np.asarray(qual)[i][nz])
        ptr.append(len(snp))
    return synth.Fragments(M.shape[1], np.array(ptr, np.int64), np.array(snp, np.int32),
                           np.array(al, np.int8), np.array(q, np.uint8),
                           np.zeros(M.shape[0], np.uint8) if porec is None
                           else np.asarray(porec, np.uint8),
                           np.arange(M.shape[1], dtype=np.int64),
                           np.ones(M.shape[1], np.int8))


def _dense_M(fr):
    M = np.zeros((fr.n_frags, fr.n_snps), np.int64)
    rows = np.repeat(np.arange(fr.n_frags), np.diff(fr.frag_ptr))
    M[rows, fr.snp] = fr.allele
    return M


def _brute_maxcut(W):
    n = W.shape[0]
    best = -np.inf
    # spin 0 fixed to +1 (global flip symmetry); enumerate the rest in chunks
    for bits in range(1 << (n - 1)):
        s = np.ones(n)
        for k in range(n - 1):
            if bits >> k & 1:
                s[k + 1] = -1
        c = 0.25 * (W.sum() - s @ W @ s)
        best = max(best, c)
    return best


def _brute_maxcut_fast(W):
    n = W.shape[0]
    idx = np.arange(1 << (n - 1), dtype=np.int64)
    S = np.ones((idx.size, n))
    for k in range(n - 1):
        S[:, k + 1] = np.where((idx >> k) & 1, -1.0, 1.0)
    vals = 0.25 * (W.sum() - np.einsum("ri,ij,rj->r", S, W, S))
    return vals.max()


# ----------------------------------------------------------------------------- RNG
def test_splitmix64_published_vectors(oracle):
    # SplitMix64 first output from state 0 and the published sequence for seed 1234567
    assert oracle.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert [oracle.splitmix64(1234567, i) for i in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_init_values_range_and_grid(oracle):
    v = np.array([oracle.init_value(7, b, 0, r, i, w) for b in range(2) for r in range(4)
                  for i in range(50) for w in range(2)])
    assert v.min() >= -0.1 and v.max() < 0.1
    u = (v + 0.1) / 0.2 * 2 ** 24
    assert np.allclose(u, np.round(u), atol=1e-6)
    assert len(np.unique(v)) > 0.99 * v.size


# ----------------------------------------------------------------------------- read graph
def test_read_graph_hand_example(oracle):
    g = json.load(open(os.path.join(GOLD, "read_graph_hand.json")))
    fr = _frags_from_M(g["M"])
    assert (oracle.read_graph_dense(fr, oracle.READ_CONFLICT) == np.array(g["conflict"])).all()
    W = oracle.read_graph_dense(fr, oracle.READ_SIGNED)
    assert (W == np.array(g["signed"])).all()
    csr = oracle.read_graph(fr, oracle.READ_SIGNED)
    assert (csr.dense() == W).all()
    s = np.array(g["argmax_spins"], np.int8)
    assert oracle.cut(csr, s) == g["max_cut"]
    assert W.sum() == g["sum_W_signed"]
    assert s @ W @ s == g["sTWs_signed_at_argmax"]
    assert _brute_maxcut(W.astype(float)) == g["max_cut"]
    wc = oracle.CSR.from_dense(np.array(g["conflict"]))
    assert _brute_maxcut(np.array(g["conflict"], float)) == g["max_cut"]
    assert oracle.cut(wc, s) == g["max_cut"]
    hap1, sb = oracle.vote(fr, s, np.zeros(3, np.int32), 1)
    assert hap1.tolist() == g["vote_hap1_with_S1_r0_r2"]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_read_graph_matches_matrix_identities(oracle, seed):
    fr = synth.tiny_reads(seed=seed, n_snps=120, n_reads=40, flip_p=0.1, miss_p=0.1)
    M = _dense_M(fr)
    Ws = oracle.read_graph_dense(fr, oracle.READ_SIGNED)
    Wc = oracle.read_graph_dense(fr, oracle.READ_CONFLICT)
    signed = -(M @ M.T)
    np.fill_diagonal(signed, 0)
    assert (Ws == signed).all()
    overlap = np.abs(M) @ np.abs(M).T
    np.fill_diagonal(overlap, 0)
    agree = (overlap - signed) // 2
    conflict = (overlap + signed) // 2
    assert (Wc == conflict).all() and (agree >= 0).all()
    for mode, Wd in ((oracle.READ_SIGNED, Ws), (oracle.READ_CONFLICT, Wc)):
        csr = oracle.read_graph(fr, mode)
        assert (csr.dense() == Wd).all()
        assert np.all(np.diff(csr.row_ptr) >= 0)


def test_read_graph_rejects_bad_input(oracle):
    fr = _frags_from_M([[1, 1, 0], [0, -1, 1]])
    fr.allele = fr.allele.copy()
    fr.allele[0] = 2
    with pytest.raises(ValueError):
        oracle.read_graph_dense(fr)
    fr2 = _frags_from_M([[1, 1, 0], [0, -1, 1]])
    fr2.snp = fr2.snp.copy()
    fr2.snp[1] = 0  # not strictly increasing inside a fragment
    with pytest.raises(ValueError):
        oracle.read_graph(fr2)


def test_read_graph_empty_and_singleton_fragments(oracle):
    fr = _frags_from_M([[0, 0, 0], [1, 0, 0], [0, 0, 0]])
    W = oracle.read_graph_dense(fr)
    assert (W == 0).all()
    g = oracle.read_graph(fr)
    assert g.nnz == 0
    assert oracle.blocks_of(g) == []


# ----------------------------------------------------------------------------- SNP graph
def _llr_closed_form(qa, qb):
    # P_cis + P_trans = 1 and P_cis - P_trans = (2 q_u - 1)(2 q_v - 1), so
    # log10(P_cis / P_trans) = 2 atanh(d) / ln 10 with d = (1 - 2 e_u)(1 - 2 e_v), e = 10^(-Q/10)
    d = (1 - 2 * 10 ** (-qa / 10)) * (1 - 2 * 10 ** (-qb / 10))
    return 2 * math.atanh(d) / math.log(10)


@pytest.mark.parametrize("qa,qb", [(10, 10), (20, 20), (30, 30), (7, 7), (10, 20), (4, 93),
                                   (13, 29)])
def test_snp_edge_two_snp_closed_form(oracle, qa, qb):
    for sa, sb in ((1, 1), (1, -1), (-1, -1)):
        fr = _frags_from_M([[sa, sb]], qual=[[qa, qb]])
        g = oracle.snp_graph(fr)
        W = g.dense()
        expect = -(sa * sb) * _llr_closed_form(qa, qb)
        assert W[0, 1] == pytest.approx(expect, rel=1e-13)
        assert W[1, 0] == W[0, 1]


def test_snp_edge_hand_computed_values(oracle):
    # Q = 10, equal alleles: q = 0.9, P_cis = 0.82, P_trans = 0.18, w = -log10(0.82 / 0.18);
    # and the three-SNP fragment normalised by |S_i| - 1 = 2 (Eq. edge_weight_SNP)
    fr = _frags_from_M([[1, 1]], qual=[[10, 10]])
    assert oracle.snp_graph(fr).dense()[0, 1] == pytest.approx(-0.6585413472804108, rel=1e-14)
    fr3 = _frags_from_M([[1, 1, -1]], qual=[[10, 20, 30]])
    W = oracle.snp_graph(fr3).dense()
    assert W[0, 1] == pytest.approx(-_llr_closed_form(10, 20) / 2, rel=1e-13)
    assert W[0, 2] == pytest.approx(+_llr_closed_form(10, 30) / 2, rel=1e-13)
    assert W[1, 2] == pytest.approx(+_llr_closed_form(20, 30) / 2, rel=1e-13)


def test_snp_edge_additivity_porec_alpha_and_linkage(oracle):
    rng = np.random.default_rng(5)
    M = np.array([[1, -1, 1, 1, -1]])
    Q = rng.integers(7, 31, size=(1, 5))
    one = oracle.snp_graph(_frags_from_M(M, qual=Q)).dense()
    two = oracle.snp_graph(_frags_from_M(np.vstack([M, M]), qual=np.vstack([Q, Q]))).dense()
    assert np.allclose(two, 2 * one, rtol=1e-15, atol=0)
    pc = oracle.snp_graph(_frags_from_M(M, qual=Q, porec=[1]), porec_alpha=0.1).dense()
    assert np.allclose(pc, 0.1 * one, rtol=1e-14, atol=0)
    # linkage depth 5/10 on |S| = 5: each SNP links to the next floor(5*4/10) = 2 SNPs,
    # normalisation stays |S| - 1
    half = oracle.snp_graph(_frags_from_M(M, qual=Q), linkage_k=5).dense()
    mask = np.zeros((5, 5), bool)
    for u in range(5):
        for v in range(u + 1, min(5, u + 3)):
            mask[u, v] = mask[v, u] = True
    assert np.array_equal(half != 0, mask)
    assert np.allclose(half[mask], one[mask], rtol=1e-15)


def test_snp_graph_rejects_bad_quality(oracle):
    with pytest.raises(ValueError):
        oracle.snp_graph(_frags_from_M([[1, 1]], qual=[[3, 20]]))
    with pytest.raises(ValueError):
        oracle.snp_graph(_frags_from_M([[1, 1]], qual=[[20, 94]]))


def test_snp_graph_truth_signs_without_errors(oracle):
    # error-free reads: cis pairs (same truth) get negative weight, trans pairs positive
    fr = synth.region_reads(11, n_snps=200, region=60_000, n_reads=60, len_mean=8000,
                            len_sd=2000, flip_p=0.0, miss_p=0.0, qual=(7, 30))
    W = oracle.snp_graph(fr).dense()
    t = fr.truth.astype(float)
    nz = W != 0
    assert np.all(np.sign(W[nz]) == -np.outer(t, t)[nz])


def test_snp_graph_gauge_under_allele_flips(oracle):
    """Flipping the alleles at a set T of SNPs in every fragment gives exactly D W D
    (d = -1 on T): each edge term carries the allele product M_iu M_iv, the quality
    terms do not depend on the allele, and the summation order is unchanged.  With
    Pore-C fragments and a linkage depth below 10."""
    import dataclasses
    fr = synth.region_reads(12, n_snps=150, region=50_000, n_reads=50, len_mean=8000,
                            len_sd=2000, flip_p=0.05, miss_p=0.0, qual=(7, 30))
    rng = np.random.default_rng(3)
    fr = dataclasses.replace(fr, is_porec=(rng.random(fr.n_frags) < 0.3).astype(np.uint8))
    T = rng.random(fr.n_snps) < 0.4
    frt = dataclasses.replace(fr, allele=np.where(T[fr.snp], -fr.allele, fr.allele).astype(fr.allele.dtype))
    d = np.where(T, -1.0, 1.0)
    for k in (10, 6):
        W = oracle.snp_graph(fr, linkage_k=k).dense()
        Wt = oracle.snp_graph(frt, linkage_k=k).dense()
        assert np.count_nonzero(W) > 0
        assert np.array_equal(Wt, d[:, None] * W * d[None, :])


# ----------------------------------------------------------------------------- components
def test_components_match_scipy(oracle):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    fr = synth.region_reads(3, n_snps=600, region=400_000, n_reads=70, len_mean=6000,
                            len_sd=3000, flip_p=0.05, miss_p=0.0)
    g = oracle.read_graph(fr, oracle.READ_SIGNED)
    nc, lab = oracle.components(g)
    A = csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(g.n, g.n))
    nc2, lab2 = connected_components(A, directed=False)
    assert nc == nc2
    # same partition, numbered by smallest vertex
    first = {}
    for v, c in enumerate(lab2):
        first.setdefault(c, len(first))
    assert np.array_equal(lab, np.array([first[c] for c in lab2]))
    assert nc > 1


# ----------------------------------------------------------------------------- bSB dynamics
def test_bsb_matches_ode_integration(oracle):
    """Symplectic-Euler bSB converges (first order) to the bSB ODE solved by scipy."""
    from scipy.integrate import solve_ivp
    rng = np.random.default_rng(0)
    n = 5
    J = rng.normal(size=(n, n))  # deliberately asymmetric: catches a transposed product
    np.fill_diagonal(J, 0)
    g = oracle.CSR.from_dense(-J)  # w = -J
    a0, c0, T = 1.0, 0.15, 6.0
    x0 = rng.uniform(-0.05, 0.05, n)
    y0 = rng.uniform(-0.05, 0.05, n)

    def rhs2(t, u):
        x, y = u[:n], u[n:]
        at = a0 * t / T
        dy = -(a0 - at) * x + c0 * (J @ x)
        return np.concatenate([a0 * y, dy])

    ref = solve_ivp(rhs2, (0, T), np.concatenate([x0, y0]), rtol=1e-11, atol=1e-13).y[:, -1]
    assert np.abs(ref[:n]).max() < 1.0  # wall never reached: pure dynamics
    errs = []
    for steps in (3000, 6000):
        dt = T / steps
        x, y = oracle.bsb_run(g, x0[None], y0[None], 0, steps, steps, dt=dt, a0=a0, c0=c0)
        errs.append(np.abs(np.concatenate([x[0], y[0]]) - ref).max() / np.abs(ref).max())
    assert errs[1] < 2e-3
    assert 1.6 < errs[0] / errs[1] < 2.4  # first-order convergence to the ODE


def test_bsb_wall_invariant(oracle):
    rng = np.random.default_rng(1)
    W = synth.random_graph(3, 12, p=0.5)
    g = oracle.CSR.from_dense(W)
    x0 = rng.uniform(-0.1, 0.1, (4, 12))
    y0 = rng.uniform(-0.1, 0.1, (4, 12))
    x, y = oracle.bsb_run(g, x0, y0, 0, 150, 300, dt=1.0, a0=1.0, c0=0.3)
    assert np.abs(x).max() <= 1.0
    at_wall = np.abs(x) == 1.0
    assert at_wall.any()
    assert np.all(y[at_wall] == 0.0)


def test_bsb_gauge_invariance_exact(oracle):
    """Solving D J D from D x0 gives exactly D x(t): sign flips are exact in FP64."""
    W = synth.random_graph(4, 14, p=0.4, integer=False)
    g = oracle.CSR.from_dense(W)
    rng = np.random.default_rng(2)
    d = np.where(rng.random(14) < 0.5, -1.0, 1.0)
    gd = oracle.CSR.from_dense(d[:, None] * W * d[None, :])
    x0 = rng.uniform(-0.1, 0.1, (3, 14))
    y0 = rng.uniform(-0.1, 0.1, (3, 14))
    c0 = oracle.default_c0(g)
    x1, y1 = oracle.bsb_run(g, x0, y0, 0, 400, 400, c0=c0)
    x2, y2 = oracle.bsb_run(gd, x0 * d, y0 * d, 0, 400, 400, c0=c0)
    assert np.array_equal(x2, x1 * d) and np.array_equal(y2, y1 * d)


def test_default_c0_definition(oracle):
    """Definition check, not a pin: the paper prints no c0, and the oracle's c0 is the
    normalisation of the bSB literature it cites.  This only guards the sums (both
    triangles, N (N - 1) pairs) against an indexing slip."""
    W = synth.random_graph(9, 10, p=0.6, integer=False)
    g = oracle.CSR.from_dense(W)
    n = 10
    sigma = np.sqrt((W ** 2).sum() / (n * (n - 1)))
    assert oracle.default_c0(g) == pytest.approx(0.5 / (sigma * np.sqrt(n)), rel=1e-14)


# ----------------------------------------------------------------------------- cut / energy
def test_cut_identity_and_energy(oracle):
    W = synth.random_graph(5, 16, p=0.5, integer=False)
    g = oracle.CSR.from_dense(W)
    rng = np.random.default_rng(3)
    for _ in range(5):
        s = np.where(rng.random(16) < 0.5, -1, 1).astype(np.int8)
        sf = s.astype(float)
        assert oracle.cut(g, s) == pytest.approx(0.25 * (W.sum() - sf @ W @ sf), abs=1e-10)
        assert oracle.ising_energy(g, s) == pytest.approx(-0.5 * sf @ (-W) @ sf, abs=1e-10)


def _ring(n):
    W = np.zeros((n, n))
    for i in range(n):
        W[i, (i + 1) % n] = W[(i + 1) % n, i] = 1
    return W


@pytest.mark.parametrize("name,W,opt", [
    ("C8", _ring(8), 8), ("C9", _ring(9), 8), ("C12", _ring(12), 12), ("C13", _ring(13), 12),
    ("K7", np.ones((7, 7)) - np.eye(7), 12), ("K10", np.ones((10, 10)) - np.eye(10), 25),
    ("K34", np.block([[np.zeros((3, 3)), np.ones((3, 4))], [np.ones((4, 3)), np.zeros((4, 4))]]),
     12),
])
def test_bsb_closed_form_maxcut(oracle, name, W, opt):
    g = oracle.CSR.from_dense(W)
    best, s, cuts, br = oracle.bsb_solve(g, list(range(32)), 1000, seed=17)
    assert best == opt
    assert _brute_maxcut_fast(W) == opt


def test_bsb_brute_force(oracle):
    hits, total = 0, 0
    for seed in range(12):
        n = 10 + seed % 7
        W = synth.random_graph(100 + seed, n, p=0.5, integer=(seed % 2 == 0))
        g = oracle.CSR.from_dense(W)
        opt = _brute_maxcut_fast(W)
        best, s, cuts, br = oracle.bsb_solve(g, list(range(32)), 2000, seed=seed)
        assert best == pytest.approx(oracle.cut(g, s))
        assert best >= 0.99 * opt - 1e-9
        assert cuts[br] == best and np.all(cuts[:br] < best)  # ties -> lowest replica
        hits += abs(best - opt) < 1e-9
        total += 1
    assert hits >= 0.9 * total


def test_bsb_planted_partition_error_free(oracle):
    fr = synth.tiny_reads(seed=21, flip_p=0.0)
    res = oracle.phase_read(fr, oracle.READ_SIGNED, range(16), 1000, seed=3)
    g = res["graph"]
    for b, nodes in enumerate(res["blocks"]):
        sub = g.subgraph(nodes)
        planted = sub.w[sub.w > 0].sum() / 2
        assert res["cuts"][b] == planted
    se, he = metrics.switch_hamming(res["hap1"], res["snp_block"], fr.truth)
    assert se == 0.0 and he == 0.0


# ----------------------------------------------------------------------------- voting / parity
def test_vote_rule_cases(oracle):
    cases = json.load(open(os.path.join(GOLD, "vote_cases.json")))["cases"]
    n = len(cases)
    rows, spins = [], []
    for j, c in enumerate(cases):
        for a in c["S1"]:
            r = np.zeros(n, np.int64)
            r[j] = a
            rows.append(r)
            spins.append(1)
        for a in c["S2"]:
            r = np.zeros(n, np.int64)
            r[j] = a
            rows.append(r)
            spins.append(-1)
    fr = _frags_from_M(np.array(rows))
    hap1, sb = oracle.vote(fr, np.array(spins, np.int8), np.zeros(len(rows), np.int32), 1)
    assert hap1.tolist() == [c["hap1"] for c in cases]
    assert sb.tolist() == [0 if c["hap1"] != 0 else -1 for c in cases]


def test_vote_block_assignment_majority(oracle):
    # SNP 0 covered by 2 reads of block 1 and 1 read of block 0 -> block 1 votes
    fr = _frags_from_M([[1], [-1], [1]])
    hap1, sb = oracle.vote(fr, np.array([1, 1, -1], np.int8), np.array([0, 1, 1], np.int32), 2)
    assert sb.tolist() == [1] and hap1.tolist() == [-1]


def test_parity_swap(oracle):
    hap1 = oracle.parity(np.array([0, 1, 2, 3, 0]), np.array([1, 1, 1, 1, 0]))
    assert hap1.tolist() == [1, -1, 1, -1, 0]


def test_refinement_invariant_and_error_free_phase(oracle):
    fr = synth.region_reads(31, n_snps=150, region=50_000, n_reads=50, len_mean=8000,
                            len_sd=2000, flip_p=0.0, miss_p=0.0, qual=(10, 30))
    res = oracle.phase_snp(fr, range(8), 300, seed=5, refine_max=15)
    se, he = metrics.switch_hamming(res["hap1"], res["snp_block"], fr.truth)
    assert se == 0.0 and he == 0.0
    # noisy input: the final parity partition never cuts less of the ungauged graph
    fr2 = synth.region_reads(32, n_snps=150, region=50_000, n_reads=40, len_mean=8000,
                             len_sd=2000, flip_p=0.08, miss_p=0.0, qual=(7, 30))
    res2 = oracle.phase_snp(fr2, range(4), 150, seed=6, refine_max=15)
    g = res2["graph"]
    for b, nodes in enumerate(res2["blocks"]):
        sub = g.subgraph(nodes)
        p = np.where(res2["C"][nodes] % 2 == 0, 1, -1).astype(np.int8)
        assert oracle.cut(sub, p) >= res2["first_cuts"][b] - 1e-9
        assert 1 <= res2["iters"][b] <= 15


# ----------------------------------------------------------------------------- metrics
def test_metrics_paper_example():
    g = json.load(open(os.path.join(GOLD, "metrics_paper_example.json")))
    se, he = metrics.string_example(g["inferred"], g["reference"])
    assert se == pytest.approx(g["se"]) and he == pytest.approx(g["he"])


def test_n50_hand_case():
    assert metrics.n50([50_000, 30_000, 20_000]) == 50_000
    assert metrics.n50([10, 10, 10, 10]) == 10
    assert metrics.n50([]) == 0


# ----------------------------------------------------------------------------- dSB and aSB
def test_asb_matches_ode_integration(oracle):
    """Adiabatic SB: symplectic Euler converges (first order) to its ODE, cubic detuning
    included, and it has no walls."""
    from scipy.integrate import solve_ivp
    rng = np.random.default_rng(10)
    n = 5
    J = rng.normal(size=(n, n))  # asymmetric: catches a transposed product
    np.fill_diagonal(J, 0)
    g = oracle.CSR.from_dense(-J)
    a0, c0, T = 1.0, 0.4, 8.0
    x0 = rng.uniform(-0.3, 0.3, n)
    y0 = rng.uniform(-0.3, 0.3, n)

    def rhs(t, u):
        x, y = u[:n], u[n:]
        at = a0 * t / T
        return np.concatenate([a0 * y, -(x * x + a0 - at) * x + c0 * (J @ x)])

    ref = solve_ivp(rhs, (0, T), np.concatenate([x0, y0]), rtol=1e-11, atol=1e-13).y[:, -1]
    assert np.abs(ref[:n]).max() > 0.3  # the cubic term matters at this amplitude
    errs = []
    for steps in (3000, 6000):
        dt = T / steps
        x, y = oracle.bsb_run(g, x0[None], y0[None], 0, steps, steps, dt=dt, a0=a0, c0=c0,
                              variant="adiabatic")
        errs.append(np.abs(np.concatenate([x[0], y[0]]) - ref).max() / np.abs(ref).max())
    assert errs[1] < 2e-3
    assert 1.6 < errs[0] / errs[1] < 2.4


def test_asb_has_no_walls(oracle):
    W = synth.random_graph(3, 8, p=0.6)
    g = oracle.CSR.from_dense(W)
    x0 = np.full((1, 8), 0.9)
    y0 = np.full((1, 8), 2.0)
    xa, ya = oracle.bsb_run(g, x0, y0, 0, 1, 10, dt=0.5, c0=0.0, variant="adiabatic")
    xb, yb = oracle.bsb_run(g, x0, y0, 0, 1, 10, dt=0.5, c0=0.0, variant="ballistic")
    assert (np.abs(xa) > 1.0).all() and (ya != 0).all()
    assert (np.abs(xb) == 1.0).all() and (yb == 0).all()


def test_dsb_from_binary_states_equals_bsb(oracle):
    """On x in {-1, +1}^n, sgn(x) = x: one discrete step equals one ballistic step."""
    W = synth.random_graph(5, 16, p=0.5, integer=False)
    g = oracle.CSR.from_dense(W)
    rng = np.random.default_rng(11)
    x0 = np.where(rng.random((4, 16)) < 0.5, -1.0, 1.0)
    y0 = rng.uniform(-0.1, 0.1, (4, 16))
    c0 = oracle.default_c0(g)
    xd, yd = oracle.bsb_run(g, x0, y0, 7, 8, 40, c0=c0, variant="discrete")
    xb, yb = oracle.bsb_run(g, x0, y0, 7, 8, 40, c0=c0, variant="ballistic")
    assert np.array_equal(xd, xb) and np.array_equal(yd, yb)


def test_dsb_coupling_sees_only_signs(oracle):
    """Two states with the same signs differ, after a discrete step, exactly as they do
    without coupling (c0 = 0): the coupling term cancels.  The ballistic step does not."""
    W = synth.random_graph(6, 12, p=0.6, integer=False)
    g = oracle.CSR.from_dense(W)
    rng = np.random.default_rng(12)
    x1 = rng.uniform(0.05, 0.3, (2, 12)) * np.where(rng.random((2, 12)) < 0.5, -1, 1)
    x2 = x1 * rng.uniform(0.2, 0.9, (2, 12))  # same signs, other magnitudes
    y0 = rng.uniform(-0.05, 0.05, (2, 12))
    c0 = oracle.default_c0(g)

    def diff(variant, cc):
        xa, ya = oracle.bsb_run(g, x1, y0, 3, 4, 20, c0=cc, variant=variant)
        xb, yb = oracle.bsb_run(g, x2, y0, 3, 4, 20, c0=cc, variant=variant)
        assert np.abs(xa).max() < 1.0 and np.abs(xb).max() < 1.0  # away from the walls
        return np.concatenate([xa - xb, ya - yb])

    np.testing.assert_allclose(diff("discrete", c0), diff("discrete", 0.0), rtol=0, atol=1e-15)
    assert np.abs(diff("ballistic", c0) - diff("ballistic", 0.0)).max() > 1e-3


@pytest.mark.parametrize("variant,dt", [("discrete", 1.0), ("adiabatic", 0.5)])
def test_sb_variants_gauge_invariance_exact(oracle, variant, dt):
    W = synth.random_graph(4, 14, p=0.4, integer=False)
    g = oracle.CSR.from_dense(W)
    rng = np.random.default_rng(13)
    d = np.where(rng.random(14) < 0.5, -1.0, 1.0)
    gd = oracle.CSR.from_dense(d[:, None] * W * d[None, :])
    x0 = rng.uniform(-0.1, 0.1, (3, 14))
    y0 = rng.uniform(-0.1, 0.1, (3, 14))
    c0 = oracle.default_c0(g)
    x1, y1 = oracle.bsb_run(g, x0, y0, 0, 300, 300, dt=dt, c0=c0, variant=variant)
    x2, y2 = oracle.bsb_run(gd, x0 * d, y0 * d, 0, 300, 300, dt=dt, c0=c0, variant=variant)
    assert np.array_equal(x2, x1 * d) and np.array_equal(y2, y1 * d)


@pytest.mark.parametrize("variant,dt", [("discrete", 1.0), ("adiabatic", 0.5)])
def test_sb_variants_brute_force(oracle, variant, dt):
    """dSB and aSB reach the exhaustive-search optimum of small mixed-sign graphs."""
    rng = np.random.default_rng(14)
    hit, worst = 0, 1.0
    for inst in range(12):
        n = 11
        A = np.triu(rng.integers(-3, 4, (n, n)), 1)
        A = (A + A.T).astype(float)
        g = oracle.CSR.from_dense(A)
        best, s, _, _ = oracle.bsb_solve(g, list(range(32)), 2000, inst, dt=dt, variant=variant)
        opt = -np.inf
        for bits in range(1 << (n - 1)):
            sp = np.array([1 if (bits >> i) & 1 else -1 for i in range(n)])
            opt = max(opt, 0.25 * (A.sum() - sp @ A @ sp))
        assert best == oracle.cut(g, s)
        hit += best >= opt - 1e-9
        worst = min(worst, best / opt)
    assert hit >= 11 and worst >= 0.9, (hit, worst)


# ----------------------------------------------------------------------------- deformation
def test_deformed_bsb_matches_ode_integration(oracle):
    """bSB with the deformation field h (1 - t/T) d_i converges (first order) to its ODE."""
    from scipy.integrate import solve_ivp
    rng = np.random.default_rng(20)
    n = 5
    J = rng.normal(size=(n, n))  # asymmetric: catches a transposed product
    np.fill_diagonal(J, 0)
    g = oracle.CSR.from_dense(-J)
    a0, c0, T, h = 1.0, 0.15, 6.0, 0.02
    d = np.array([1.0, -1.0, -1.0, 1.0, 1.0])
    x0 = rng.uniform(-0.05, 0.05, n)
    y0 = rng.uniform(-0.05, 0.05, n)

    def rhs(t, u):
        x, y = u[:n], u[n:]
        return np.concatenate([a0 * y, -(a0 - a0 * t / T) * x + c0 * (J @ x)
                               + h * (1 - t / T) * d])

    ref = solve_ivp(rhs, (0, T), np.concatenate([x0, y0]), rtol=1e-11, atol=1e-13).y[:, -1]
    assert np.abs(ref[:n]).max() < 1.0
    x_plain, _ = oracle.bsb_run(g, x0[None], y0[None], 0, 6000, 6000, dt=T / 6000, a0=a0, c0=c0)
    assert np.abs(x_plain[0] - ref[:n]).max() > 0.01  # the field changes the trajectory
    errs = []
    for steps in (3000, 6000):
        x, y = oracle.bsb_run(g, x0[None], y0[None], 0, steps, steps, dt=T / steps, a0=a0,
                              c0=c0, h=h, hdir=d)
        errs.append(np.abs(np.concatenate([x[0], y[0]]) - ref).max() / np.abs(ref).max())
    assert errs[1] < 2e-3
    assert 1.6 < errs[0] / errs[1] < 2.4


def test_deformation_uniform_field_is_field_along_the_gauge(oracle):
    """A field along d on J equals, spin for spin, the uniform field on D J D from D x0:
    the refinement's uniform field in the gauged frame is a field along the incumbent."""
    W = synth.random_graph(4, 14, p=0.4, integer=False)
    g = oracle.CSR.from_dense(W)
    rng = np.random.default_rng(21)
    d = np.where(rng.random(14) < 0.5, -1.0, 1.0)
    gd = oracle.CSR.from_dense(d[:, None] * W * d[None, :])
    x0 = rng.uniform(-0.1, 0.1, (3, 14))
    y0 = rng.uniform(-0.1, 0.1, (3, 14))
    c0 = oracle.default_c0(g)
    x1, y1 = oracle.bsb_run(g, x0, y0, 0, 400, 400, c0=c0, h=0.05, hdir=d)
    x2, y2 = oracle.bsb_run(gd, x0 * d, y0 * d, 0, 400, 400, c0=c0, h=0.05)
    assert np.array_equal(x2, x1 * d) and np.array_equal(y2, y1 * d)
    x3, y3 = oracle.bsb_run(g, x0, y0, 0, 400, 400, c0=c0, h=0.0, hdir=d)
    x4, y4 = oracle.bsb_run(g, x0, y0, 0, 400, 400, c0=c0)
    assert np.array_equal(x3, x4) and np.array_equal(y3, y4)


def test_deformation_field_direction_and_decay(oracle):
    """Without couplings the field alone moves every spin toward d; its strength falls
    to zero at the end of the schedule (the last step adds nothing to y)."""
    n = 6
    g = oracle.CSR.from_dense(np.zeros((n, n)))
    d = np.array([1.0, -1.0, 1.0, -1.0, -1.0, 1.0])
    x0 = np.zeros((1, n))
    y0 = np.zeros((1, n))
    x, _ = oracle.bsb_run(g, x0, y0, 0, 100, 100, dt=0.5, c0=0.0, h=0.2, hdir=d)
    assert np.array_equal(np.sign(x[0]), d)
    # last step of the schedule, from rest at x = 0: the field term is h (1 - (T-1)/T)
    T = 50
    x1, y1 = oracle.bsb_run(g, x0, y0, T - 1, T, T, dt=1.0, c0=0.0, h=0.5, hdir=d)
    np.testing.assert_allclose(y1[0], 0.5 / T * d, rtol=0, atol=1e-15)
    x2, y2 = oracle.bsb_run(g, x0, y0, 0, 1, T, dt=1.0, c0=0.0, h=0.5, hdir=d)
    np.testing.assert_allclose(y2[0], 0.5 * d, rtol=0, atol=1e-15)


def test_refine_deformation_retries_count_toward_refine_max(oracle):
    """Every weight negative: no cut is positive, so each solve fails.  The plain
    refinement stops after one solve; with deformation it re-solves deform_tries times
    (never beyond refine_max) and accepts nothing."""
    rng = np.random.default_rng(22)
    n = 10
    A = -np.triu(rng.uniform(0.5, 2.0, (n, n)), 1)
    A = A + A.T
    g = oracle.CSR.from_dense(A)
    for h, tries, rmax, solves in [(0.0, 3, 15, 1), (0.05, 3, 15, 4), (0.05, 3, 2, 2),
                                   (0.05, 0, 15, 1)]:
        st = {}
        Cc, acc, first, _ = oracle.refine(g, range(8), 200, 3, 0, rmax, deform_h=h,
                                          deform_tries=tries, stats=st)
        assert acc == 0 and st["solves"] == solves and not Cc.any(), (h, tries, rmax, st)
        assert first <= 0.0


def test_refine_with_deformation_matches_plain_when_cuts_stay_positive(oracle):
    """The deformation only acts after a failed solve: on an error-free read set (each
    refinement ends in one accepted partition, then a failed solve) the accepted
    partitions, and so the phase, are those of the plain refinement."""
    fr = synth.region_reads(40, n_snps=60, region=30_000, n_reads=30, len_mean=6000,
                            len_sd=1500, flip_p=0.0, miss_p=0.0, qual=(20, 30))
    a = oracle.phase_snp(fr, range(8), 300, seed=2, refine_max=15)
    b = oracle.phase_snp(fr, range(8), 300, seed=2, refine_max=15, deform_h=0.02, deform_tries=2)
    assert np.array_equal(a["hap1"], b["hap1"])
    assert (b["solves"] >= a["solves"]).all()


@pytest.mark.parametrize("variant,dt", [("discrete", 1.0), ("adiabatic", 0.25)])
def test_refinement_with_sb_variants(oracle, variant, dt):
    """The refinement runs every solve with the chosen SB variant: its first solve is
    that variant's solve of the ungauged block (a different solve from bSB's), and the
    final parity partition never cuts less than that first solve.  dSB phases error-free
    reads exactly.  aSB (dt 0.25: at 0.5 its explicit cubic term collapses every
    replica on these SNP graphs) is weaker and leaves a few errors."""
    fr = synth.region_reads(31, n_snps=150, region=50_000, n_reads=50, len_mean=8000,
                            len_sd=2000, flip_p=0.0, miss_p=0.0, qual=(10, 30))
    res = oracle.phase_snp(fr, range(8), 300, seed=5, refine_max=15, dt=dt, variant=variant)
    se, he = metrics.switch_hamming(res["hap1"], res["snp_block"], fr.truth)
    if variant == "discrete":
        assert se == 0.0 and he == 0.0
    else:
        assert se < 0.2 and he < 0.2
    fr2 = synth.region_reads(32, n_snps=150, region=50_000, n_reads=40, len_mean=8000,
                             len_sd=2000, flip_p=0.08, miss_p=0.0, qual=(7, 30))
    res2 = oracle.phase_snp(fr2, range(4), 150, seed=6, refine_max=15, dt=dt, variant=variant)
    g = res2["graph"]
    differs = 0
    for b, nodes in enumerate(res2["blocks"]):
        sub = g.subgraph(nodes)
        best, _, _, _ = oracle.bsb_solve(sub, range(4), 150, 6, b, 0, dt=dt, variant=variant)
        plain, _, _, _ = oracle.bsb_solve(sub, range(4), 150, 6, b, 0, dt=dt)
        assert res2["first_cuts"][b] == best
        differs += best != plain
        p = np.where(res2["C"][nodes] % 2 == 0, 1, -1).astype(np.int8)
        assert oracle.cut(sub, p) >= res2["first_cuts"][b] - 1e-9
    assert differs > 0


@pytest.mark.parametrize("variant,dt", [("ballistic", 1.0), ("discrete", 1.0), ("adiabatic", 0.5)])
def test_sb_spin_flip_symmetry_exact(oracle, variant, dt):
    """Every SB variant is odd in (x, y): the flipped start gives the flipped run, bit for
    bit (negation commutes with IEEE rounding; the wall, sgn and the cubic term are
    odd; no initial value is exactly zero).  The deformation field is not odd, and
    breaks it."""
    W = synth.random_graph(5, 16, p=0.4, integer=False)
    g = oracle.CSR.from_dense(W)
    rng = np.random.default_rng(17)
    x0 = rng.uniform(-0.1, 0.1, (4, 16))
    y0 = rng.uniform(-0.1, 0.1, (4, 16))
    c0 = oracle.default_c0(g)
    x1, y1 = oracle.bsb_run(g, x0, y0, 0, 200, 200, dt=dt, c0=c0, variant=variant)
    x2, y2 = oracle.bsb_run(g, -x0, -y0, 0, 200, 200, dt=dt, c0=c0, variant=variant)
    assert np.array_equal(x2, -x1) and np.array_equal(y2, -y1)
    assert np.abs(x1).max() > 0.5  # the run got somewhere
    # mid-schedule, before the walls take every vertex (the field decays to 0 at the end)
    xm, ym = oracle.bsb_run(g, x0, y0, 0, 60, 200, dt=dt, c0=c0, variant=variant, h=0.05)
    xf, yf = oracle.bsb_run(g, -x0, -y0, 0, 60, 200, dt=dt, c0=c0, variant=variant, h=0.05)
    assert not (np.array_equal(xf, -xm) and np.array_equal(yf, -ym))


# ----------------------------------------------------------------------------- hand-worked steps
def test_bsb_two_steps_hand_values(oracle):
    """Two bSB steps worked by hand in exact fractions (tests/golden): pins the order of
    the half-steps (y from x_t, then x from y_{t+1}), a(t) indexed at t, the row-wise
    product z_i = sum_j J_ij x_j on an asymmetric J, and the wall."""
    gold = json.load(open(os.path.join(GOLD, "bsb_two_steps_hand.json")))
    for case in gold["cases"]:
        J = np.array(case["J"], np.float64)
        g = oracle.CSR.from_dense(-J)  # the oracle takes w = -J
        x = np.array([case["x0"]])
        y = np.array([case["y0"]])
        for t, key in enumerate(["after_step_0", "after_step_1"]):
            x, y = oracle.bsb_run(g, x, y, t, t + 1, case["steps"], dt=case["dt"],
                                  a0=case["a0"], c0=case["c0"])
            assert np.array_equal(x[0], np.array(case[key]["x"])), (case["name"], key)
            assert np.array_equal(y[0], np.array(case[key]["y"])), (case["name"], key)


# ----------------------------------------------------------------------------- early stop
def test_early_stop_off_equals_plain_solve(oracle):
    fr = synth.tiny_reads(1001)
    g = oracle.read_graph(fr, oracle.READ_SIGNED)
    sub = g.subgraph(oracle.blocks_of(g)[0])
    ref = oracle.bsb_solve(sub, list(range(8)), 400, 5)
    for ce, pat in [(0, 3), (50, 0), (50, 100)]:  # off, off, never reached
        best, s, cuts, br, sr = oracle.bsb_solve_early_stop(sub, list(range(8)), 400, 5, ce, pat)
        assert sr == 400
        assert best == ref[0] and br == ref[3]
        assert np.array_equal(s, ref[1]) and np.array_equal(cuts, ref[2])


@pytest.mark.parametrize("check_every,patience", [(10, 1), (25, 3), (40, 4)])
def test_early_stop_two_node_closed_form(oracle, check_every, patience):
    """One edge of weight 3: every check can at best see the cut 3, and some replica
    already splits the two vertices at the first check, so the best never improves
    after it: the stall count reaches `patience` at check 1 + patience exactly."""
    g = oracle.CSR.from_dense(np.array([[0.0, 3.0], [3.0, 0.0]]))
    steps = 2000
    best, s, cuts, br, sr = oracle.bsb_solve_early_stop(g, list(range(32)), steps, 9,
                                                         check_every, patience)
    assert sr == check_every * (1 + patience)
    assert best == 3.0 and s[0] != s[1]


def test_early_stop_result_is_the_truncated_run(oracle):
    """A block that stops keeps the state it reached: the result equals a plain run of
    the same schedule cut off after steps_run steps, evaluated with numpy."""
    fr = synth.tiny_reads(1001)
    g = oracle.read_graph(fr, oracle.READ_SIGNED)
    sub = g.subgraph(oracle.blocks_of(g)[0])
    reps, steps, seed = list(range(16)), 3000, 2
    best, s, cuts, br, sr = oracle.bsb_solve_early_stop(sub, reps, steps, seed, 50, 3)
    assert 0 < sr < steps and sr % 50 == 0
    x, y = oracle.bsb_init(sub.n, reps, seed, 0)
    x, _ = oracle.bsb_run(sub, x, y, 0, sr, steps)
    W = sub.dense()
    S = np.where(x >= 0, 1.0, -1.0)
    ref = 0.25 * (W.sum() - np.einsum("ri,ij,rj->r", S, W, S))
    assert np.array_equal(cuts, ref)
    assert best == ref.max() and br == int(np.argmax(ref))
    # the stopping check is the patience-th check in a row without a better best cut
    xs, ys = oracle.bsb_init(sub.n, reps, seed, 0)
    seen, stall, t = -np.inf, 0, 0
    while True:
        xs, ys = oracle.bsb_run(sub, xs, ys, t, t + 50, steps)
        t += 50
        Sx = np.where(xs >= 0, 1.0, -1.0)
        c = (0.25 * (W.sum() - np.einsum("ri,ij,rj->r", Sx, W, Sx))).max()
        if c > seen:
            seen, stall = c, 0
        else:
            stall += 1
            if stall == 3:
                break
    assert t == sr


# ----------------------------------------------------------------------------- best during the run
def test_track_best_is_the_best_over_the_checks(oracle):
    """track_best: the best cut reached at any check or at the end, recomputed here from
    plain runs cut off at every check (numpy cuts), with the earliest check and the
    lowest replica winning ties; the final state's cuts are still reported."""
    fr = synth.tiny_reads(1001)
    g = oracle.read_graph(fr, oracle.READ_SIGNED)
    sub = g.subgraph(oracle.blocks_of(g)[0])
    reps, steps, seed, ce = list(range(12)), 600, 4, 20
    W = sub.dense()
    x, y = oracle.bsb_init(sub.n, reps, seed, 0)
    kept, kept_r, kept_s = -np.inf, -1, None
    for t in range(ce, steps + 1, ce):
        x, y = oracle.bsb_run(sub, x, y, t - ce, t, steps)
        S = np.where(x >= 0, 1.0, -1.0)
        c = 0.25 * (W.sum() - np.einsum("ri,ij,rj->r", S, W, S))
        if t == steps:
            final = c
            r = int(np.argmax(c))
            if c[r] > kept:  # the end counts as the last check
                kept, kept_r, kept_s = c[r], r, S[r]
        else:
            r = int(np.argmax(c))
            if c[r] > kept:
                kept, kept_r, kept_s = c[r], r, S[r]
    best, s, cuts, br, sr = oracle.bsb_solve_early_stop(sub, reps, steps, seed, ce, 0,
                                                         track_best=True)
    assert sr == steps
    assert np.array_equal(cuts, final)
    assert best == kept and br == kept_r and np.array_equal(s, kept_s.astype(np.int8))
    assert best >= final.max()
    # without checks, or without track_best, the final state decides
    plain = oracle.bsb_solve(sub, reps, steps, seed)
    for ce2, tb in [(0, True), (ce, False)]:
        b2, s2, _, br2, _ = oracle.bsb_solve_early_stop(sub, reps, steps, seed, ce2, 0,
                                                         track_best=tb)
        assert b2 == plain[0] and br2 == plain[3] and np.array_equal(s2, plain[1])


def test_track_best_with_early_stop(oracle):
    """With early stop too: the stop comes at the same step as without track_best, and
    the kept result is at least the stopped state's best."""
    fr = synth.tiny_reads(1001)
    g = oracle.read_graph(fr, oracle.READ_SIGNED)
    sub = g.subgraph(oracle.blocks_of(g)[0])
    reps, steps, seed = list(range(16)), 3000, 2
    b0, _, c0_, _, sr0 = oracle.bsb_solve_early_stop(sub, reps, steps, seed, 50, 3)
    b1, s1, c1, br1, sr1 = oracle.bsb_solve_early_stop(sub, reps, steps, seed, 50, 3,
                                                        track_best=True)
    assert sr1 == sr0 and np.array_equal(c1, c0_)
    assert b1 >= b0 and b1 == oracle.cut(sub, s1)
