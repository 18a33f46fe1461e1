"""ctypes wrapper around the FP64 C oracle (qhap_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the smoke check and the CPU
baseline leg of the benchmark.  Nothing on the product path imports it.

Each function cites the Methods passage of the QHap paper that it restates; the
composed pipelines (`phase_read`, `phase_snp`) chain them in the paper's order:
graph construction -> connected components (singletons dropped) -> bSB per
component -> voting (read-based) or iterative refinement + parity (SNP-based).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qhap_oracle.c")
_LIB = os.path.join(_HERE, "libqhap_oracle.so")

READ_CONFLICT = 0
READ_SIGNED = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _setup(_lib)
    return _lib


P = C.c_void_p
I32, I64, U64, D = C.c_int32, C.c_int64, C.c_uint64, C.c_double


def _setup(L):
    L.qo_init_value.restype = D
    L.qo_init_value.argtypes = [U64, I64, I32, I32, I64, C.c_int]
    L.qo_splitmix64.restype = U64
    L.qo_splitmix64.argtypes = [U64, U64]
    L.qo_read_graph_dense.restype = C.c_int
    L.qo_read_graph_dense.argtypes = [I32, I32, P, P, P, C.c_int, P]
    L.qo_read_graph_csr.restype = I64
    L.qo_read_graph_csr.argtypes = [I32, I32, P, P, P, C.c_int, C.POINTER(P), C.POINTER(P),
                                    C.POINTER(P)]
    L.qo_snp_graph_csr.restype = I64
    L.qo_snp_graph_csr.argtypes = [I32, I32, P, P, P, P, P, D, C.c_int, C.POINTER(P),
                                   C.POINTER(P), C.POINTER(P)]
    L.qo_free.restype = None
    L.qo_free.argtypes = [P]
    L.qo_components.restype = I32
    L.qo_components.argtypes = [I32, P, P, P, P]
    L.qo_bsb_run.restype = None
    L.qo_bsb_run.argtypes = [I32, P, P, P, I32, P, P, I32, I32, I32, D, D, D]
    L.qo_bsb_init.restype = None
    L.qo_bsb_init.argtypes = [I32, I32, P, U64, I64, I32, P, P]
    L.qo_default_c0.restype = D
    L.qo_default_c0.argtypes = [I32, P, P]
    L.qo_cut.restype = D
    L.qo_cut.argtypes = [I32, P, P, P, P]
    L.qo_ising_energy.restype = D
    L.qo_ising_energy.argtypes = [I32, P, P, P, P]
    L.qo_bsb_solve.restype = D
    L.qo_bsb_solve.argtypes = [I32, P, P, P, I32, P, I32, D, D, D, U64, I64, I32, P, P, P]
    L.qo_sb_run.restype = None
    L.qo_sb_run.argtypes = [I32, P, P, P, I32, P, P, I32, I32, I32, D, D, D, I32]
    L.qo_sb_solve.restype = D
    L.qo_sb_solve_es.restype = D
    L.qo_sb_solve_es.argtypes = [I32, P, P, P, I32, P, I32, D, D, D, U64, I64, I32, I32, I32, P, P,
                                 P, P, I32, I32]
    L.qo_sb_solve.argtypes = [I32, P, P, P, I32, P, I32, D, D, D, U64, I64, I32, P, P, P, I32]
    L.qo_refine.restype = I32
    L.qo_refine.argtypes = [I32, P, P, P, I32, P, I32, D, D, D, U64, I64, I32, P, P]
    L.qo_sb_run_h.restype = None
    L.qo_sb_run_h.argtypes = [I32, P, P, P, I32, P, P, I32, I32, I32, D, D, D, I32, D, P]
    L.qo_sb_solve_h.restype = D
    L.qo_sb_solve_h.argtypes = [I32, P, P, P, I32, P, I32, D, D, D, U64, I64, I32, P, P, P, I32, D]
    L.qo_refine_h.restype = I32
    L.qo_refine_h.argtypes = [I32, P, P, P, I32, P, I32, D, D, D, U64, I64, I32, P, P, D, I32, P]
    L.qo_refine_v.restype = I32
    L.qo_refine_v.argtypes = [I32, P, P, P, I32, P, I32, D, D, D, U64, I64, I32, P, P, D, I32, P,
                              I32]
    L.qo_vote.restype = None
    L.qo_vote.argtypes = [I32, I32, P, P, P, P, P, I32, P, P]
    L.qo_parity.restype = None
    L.qo_parity.argtypes = [I32, P, P, P]


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class CSR:
    """Symmetric sparse graph: row_ptr int64[n+1], col int32[nnz], w float64[nnz]."""

    def __init__(self, n, row_ptr, col, w):
        self.n = int(n)
        self.row_ptr = _c(row_ptr, np.int64)
        self.col = _c(col, np.int32)
        self.w = _c(w, np.float64)

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    def dense(self):
        W = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        W[rows, self.col] = self.w
        return W

    @staticmethod
    def from_dense(W):
        W = np.asarray(W, dtype=np.float64)
        n = W.shape[0]
        mask = W != 0
        rp = np.concatenate([[0], np.cumsum(mask.sum(1))]).astype(np.int64)
        rows, cols = np.nonzero(mask)
        return CSR(n, rp, cols.astype(np.int32), W[rows, cols])

    def subgraph(self, nodes):
        """Induced subgraph on `nodes` (sorted), renumbered 0..len-1."""
        nodes = np.asarray(nodes, dtype=np.int64)
        pos = -np.ones(self.n, np.int64)
        pos[nodes] = np.arange(nodes.shape[0])
        rp, cols, ws = [0], [], []
        for u in nodes:
            s, e = self.row_ptr[u], self.row_ptr[u + 1]
            c = pos[self.col[s:e]]
            keep = c >= 0
            cols.append(c[keep])
            ws.append(self.w[s:e][keep])
            rp.append(rp[-1] + int(keep.sum()))
        col = np.concatenate(cols) if cols else np.zeros(0, np.int64)
        w = np.concatenate(ws) if ws else np.zeros(0)
        return CSR(nodes.shape[0], np.array(rp, np.int64), col.astype(np.int32), w)


def _take_csr(n, nnz, rp, col, w):
    L = lib()
    if nnz < 0:
        raise ValueError(f"oracle rejected the input (status {-nnz})")
    r = np.ctypeslib.as_array(C.cast(rp, C.POINTER(C.c_int64)), shape=(n + 1,)).copy()
    c = (np.ctypeslib.as_array(C.cast(col, C.POINTER(C.c_int32)), shape=(nnz,)).copy()
         if nnz else np.zeros(0, np.int32))
    ww = (np.ctypeslib.as_array(C.cast(w, C.POINTER(C.c_double)), shape=(nnz,)).copy()
          if nnz else np.zeros(0))
    for ptr in (rp, col, w):
        L.qo_free(ptr)
    return CSR(n, r, c, ww)


def init_value(seed, block, it, replica, node, which):
    return lib().qo_init_value(seed, block, it, replica, node, which)


def splitmix64(key, n):
    return lib().qo_splitmix64(key, n)


def read_graph_dense(fr, mode=READ_SIGNED):
    """Read-based graph, Eqs. delta / w_ab (CONFLICT) or W = -M M^T (SIGNED)."""
    m = fr.n_frags
    W = np.zeros((m, m), np.int64)
    fp, snp, al = _c(fr.frag_ptr, np.int64), _c(fr.snp, np.int32), _c(fr.allele, np.int8)
    rc = lib().qo_read_graph_dense(m, fr.n_snps, _p(fp), _p(snp), _p(al), mode, _p(W))
    if rc:
        raise ValueError(f"oracle rejected the input (status {rc})")
    return W


def read_graph(fr, mode=READ_SIGNED):
    fp, snp, al = _c(fr.frag_ptr, np.int64), _c(fr.snp, np.int32), _c(fr.allele, np.int8)
    rp, col, w = P(), P(), P()
    nnz = lib().qo_read_graph_csr(fr.n_frags, fr.n_snps, _p(fp), _p(snp), _p(al), mode,
                                  C.byref(rp), C.byref(col), C.byref(w))
    return _take_csr(fr.n_frags, nnz, rp, col, w)


def snp_graph(fr, porec_alpha=0.1, linkage_k=10):
    """SNP-based graph, Eq. edge_weight_SNP with the Pore-C alpha and linkage depth k/10."""
    fp, snp, al = _c(fr.frag_ptr, np.int64), _c(fr.snp, np.int32), _c(fr.allele, np.int8)
    q, pc = _c(fr.qual, np.uint8), _c(fr.is_porec, np.uint8)
    rp, col, w = P(), P(), P()
    nnz = lib().qo_snp_graph_csr(fr.n_frags, fr.n_snps, _p(fp), _p(snp), _p(al), _p(q), _p(pc),
                                 porec_alpha, linkage_k, C.byref(rp), C.byref(col), C.byref(w))
    return _take_csr(fr.n_snps, nnz, rp, col, w)


def components(g: CSR):
    """BFS components over w != 0 edges, numbered by smallest vertex."""
    lab = np.zeros(g.n, np.int32)
    nc = lib().qo_components(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), _p(lab))
    return nc, lab


def blocks_of(g: CSR):
    """Phase blocks: components with >= 2 vertices, in order of smallest vertex."""
    nc, lab = components(g)
    sizes = np.bincount(lab, minlength=nc)
    blocks = [np.nonzero(lab == c)[0] for c in range(nc) if sizes[c] >= 2]
    return blocks


def default_c0(g: CSR):
    J = _c(-g.w, np.float64)
    return lib().qo_default_c0(g.n, _p(g.row_ptr), _p(J))


def bsb_init(n, replica_ids, seed, block, it=0):
    rid = _c(replica_ids, np.int32)
    R = rid.shape[0]
    x = np.zeros((R, n))
    y = np.zeros((R, n))
    lib().qo_bsb_init(n, R, _p(rid), seed, block, it, _p(x), _p(y))
    return x, y


# simulated bifurcation variants compared in the paper (standard formulations it cites)
SB_VARIANTS = {"ballistic": 0, "discrete": 1, "adiabatic": 2}


def bsb_run(g: CSR, x, y, t0, t1, steps, dt=1.0, a0=1.0, c0=None, variant="ballistic",
            h=0.0, hdir=None):
    """Advance x, y ([R][n] float64, in place copies returned) by steps t0..t1-1 with J = -w.

    variant: "ballistic" (bSB), "discrete" (dSB: J sgn(x)), "adiabatic" (aSB: cubic
    detuning, no walls).  h, hdir: the deformation field h (1 - t / steps) hdir_i added
    to the force on y (hdir in {-1, +1}^n, None = all +1)."""
    x = np.array(x, dtype=np.float64, order="C")
    y = np.array(y, dtype=np.float64, order="C")
    J = _c(-g.w, np.float64)
    if c0 is None:
        c0 = default_c0(g)
    hd = None if hdir is None else _c(hdir, np.float64)
    lib().qo_sb_run_h(g.n, _p(g.row_ptr), _p(g.col), _p(J), x.shape[0], _p(x), _p(y), t0, t1,
                      steps, dt, a0, c0, SB_VARIANTS[variant], h,
                      _p(hd) if hd is not None else None)
    return x, y


def cut(g: CSR, s):
    s = _c(s, np.int8)
    return lib().qo_cut(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), _p(s))


def ising_energy(g: CSR, s):
    s = _c(s, np.int8)
    J = _c(-g.w, np.float64)
    return lib().qo_ising_energy(g.n, _p(g.row_ptr), _p(g.col), _p(J), _p(s))


def bsb_solve(g: CSR, replica_ids, steps, seed, block=0, it=0, dt=1.0, a0=1.0, c0=0.0,
              variant="ballistic", h=0.0):
    """Multi-replica SB (SB algorithm solution); returns (best_cut, spins, cuts, best_r).
    h > 0: the deformation field along +1 on every vertex."""
    rid = _c(replica_ids, np.int32)
    R = rid.shape[0]
    s = np.zeros(g.n, np.int8)
    cuts = np.zeros(R)
    br = C.c_int32(-1)
    best = lib().qo_sb_solve_h(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), R, _p(rid), steps, dt,
                               a0, c0, seed, block, it, _p(s), _p(cuts), C.byref(br),
                               SB_VARIANTS[variant], h)
    return best, s, cuts, br.value


def bsb_solve_early_stop(g: CSR, replica_ids, steps, seed, check_every, patience, block=0,
                         it=0, dt=1.0, a0=1.0, c0=0.0, variant="ballistic", track_best=False):
    """Multi-replica SB with early stop on a stalled best energy (the paper's maximum
    convergence count, read as a patience over periodic energy checks).  track_best:
    the result is the best cut reached at any check or at the end (the best value
    during the run), ties to the earliest check and lowest replica.  Returns
    (best_cut, spins, cuts, best_r, steps_run); cuts are the final state's."""
    rid = _c(replica_ids, np.int32)
    R = rid.shape[0]
    s = np.zeros(g.n, np.int8)
    cuts = np.zeros(R)
    br = C.c_int32(-1)
    sr = C.c_int32(0)
    best = lib().qo_sb_solve_es(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), R, _p(rid), steps, dt,
                                a0, c0, seed, block, it, check_every, patience, _p(s), _p(cuts),
                                C.byref(br), C.byref(sr), SB_VARIANTS[variant],
                                1 if track_best else 0)
    return best, s, cuts, br.value, sr.value


def refine(g: CSR, replica_ids, steps, seed, block=0, refine_max=15, dt=1.0, a0=1.0, c0=0.0,
           deform_h=0.0, deform_tries=0, stats=None, variant="ballistic"):
    """SNP-based iterative refinement: returns (C counts, accepted partitions, first cut,
    gauged w).  deform_h > 0: re-solve with the deformation field (up to deform_tries
    times, strength deform_h 2^(k-1)) when a solve's cut is <= 0.  stats (a dict, if
    given) receives "solves", the number of bSB solves made.  variant: the SB variant
    of every solve (as in bsb_run)."""
    rid = _c(replica_ids, np.int32)
    w = g.w.copy()
    Cc = np.zeros(g.n, np.int32)
    first = C.c_double(0.0)
    solves = C.c_int32(0)
    it = lib().qo_refine_v(g.n, _p(g.row_ptr), _p(g.col), _p(w), rid.shape[0], _p(rid), steps,
                           dt, a0, c0, seed, block, refine_max, _p(Cc), C.byref(first),
                           deform_h, deform_tries, C.byref(solves), SB_VARIANTS[variant])
    if stats is not None:
        stats["solves"] = solves.value
    return Cc, it, first.value, w


def vote(fr, read_spin, read_block, n_blocks):
    """Read-based consistency processing; returns (hap1, snp_block)."""
    fp, snp, al = _c(fr.frag_ptr, np.int64), _c(fr.snp, np.int32), _c(fr.allele, np.int8)
    rs, rb = _c(read_spin, np.int8), _c(read_block, np.int32)
    hap1 = np.zeros(fr.n_snps, np.int8)
    sb = np.zeros(fr.n_snps, np.int32)
    lib().qo_vote(fr.n_frags, fr.n_snps, _p(fp), _p(snp), _p(al), _p(rs), _p(rb), n_blocks,
                  _p(hap1), _p(sb))
    return hap1, sb


def parity(Ccounts, in_block):
    Cc, ib = _c(Ccounts, np.int32), _c(in_block, np.uint8)
    hap1 = np.zeros(Cc.shape[0], np.int8)
    lib().qo_parity(Cc.shape[0], _p(Cc), _p(ib), _p(hap1))
    return hap1


def phase_read(fr, mode=READ_SIGNED, replica_ids=range(8), steps=1000, seed=1, dt=1.0, a0=1.0,
               c0=0.0):
    """Whole read-based path: graph -> blocks -> bSB -> voting."""
    g = read_graph(fr, mode)
    blocks = blocks_of(g)
    read_spin = np.zeros(fr.n_frags, np.int8)
    read_block = -np.ones(fr.n_frags, np.int32)
    cuts = []
    for b, nodes in enumerate(blocks):
        sub = g.subgraph(nodes)
        best, s, _, _ = bsb_solve(sub, list(replica_ids), steps, seed, b, 0, dt, a0, c0)
        read_spin[nodes] = s
        read_block[nodes] = b
        cuts.append(best)
    hap1, sb = vote(fr, read_spin, read_block, len(blocks))
    return {"graph": g, "blocks": blocks, "cuts": np.array(cuts), "hap1": hap1,
            "snp_block": sb, "read_spin": read_spin}


def phase_snp(fr, replica_ids=range(8), steps=1000, seed=1, refine_max=15, porec_alpha=0.1,
              linkage_k=10, dt=1.0, a0=1.0, c0=0.0, deform_h=0.0, deform_tries=0,
              variant="ballistic"):
    """Whole SNP-based path: graph -> blocks -> refinement (bSB per iteration) -> parity.
    "iters": accepted partitions per block; "solves": bSB solves per block.  variant:
    the SB variant of the solves (bSB is the paper's)."""
    g = snp_graph(fr, porec_alpha, linkage_k)
    blocks = blocks_of(g)
    Ctot = np.zeros(fr.n_snps, np.int32)
    in_block = np.zeros(fr.n_snps, np.uint8)
    snp_block = -np.ones(fr.n_snps, np.int32)
    iters, first_cuts, solves = [], [], []
    for b, nodes in enumerate(blocks):
        sub = g.subgraph(nodes)
        st = {}
        Cc, it, first, _ = refine(sub, list(replica_ids), steps, seed, b, refine_max, dt, a0, c0,
                                  deform_h, deform_tries, st, variant)
        Ctot[nodes] = Cc
        in_block[nodes] = 1
        snp_block[nodes] = b
        iters.append(it)
        solves.append(st["solves"])
        first_cuts.append(first)
    hap1 = parity(Ctot, in_block)
    return {"graph": g, "blocks": blocks, "C": Ctot, "hap1": hap1, "snp_block": snp_block,
            "iters": np.array(iters), "solves": np.array(solves),
            "first_cuts": np.array(first_cuts)}
