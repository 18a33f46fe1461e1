"""Seeded synthetic fragment generators (shared input source for the CUDA path and the oracle).

This module only draws inputs: truth haplotypes, read placements, allele observations,
Phred qualities and Pore-C contacts.  It holds none of the phasing arithmetic (no encoding
rule beyond emitting +1/-1 relative to the initial H1, no graph weights, no solver).

A fragment holds, for one read, the heterozygous sites it covers, the allele seen at
each and its base quality (Methods, input preprocessing). A fragment set is stored as
CSR:

  frag_ptr  int64[m+1]   fragment i owns entries frag_ptr[i] .. frag_ptr[i+1]-1
  snp       int32[nnz]   SNP index, strictly increasing inside a fragment
  allele    int8[nnz]    +1 = allele of the initial H1, -1 = allele of the initial H2
                         (the ternary encoding M of the read-based matrix construction)
  qual      uint8[nnz]   Phred base quality of the observation
  is_porec  uint8[m]     1 for a Pore-C contact fragment

Truth: ``truth[j] = +1`` if the truth haplotype A carries the initial-H1 allele at SNP j,
-1 otherwise; haplotype B is its complement.  Reads are emitted sorted by start
coordinate, like a coordinate-sorted BAM.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Fragments:
    n_snps: int
    frag_ptr: np.ndarray
    snp: np.ndarray
    allele: np.ndarray
    qual: np.ndarray
    is_porec: np.ndarray
    positions: np.ndarray          # int64[n_snps], bp coordinate of each SNP
    truth: np.ndarray              # int8[n_snps], +1/-1
    meta: dict = field(default_factory=dict)

    @property
    def n_frags(self) -> int:
        return int(self.frag_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.frag_ptr[-1])


def _lognormal_params(mean: float, sd: float) -> tuple[float, float]:
    s2 = np.log1p((sd / mean) ** 2)
    return float(np.log(mean) - 0.5 * s2), float(np.sqrt(s2))


def _emit(rng, n_snps, lo, hi, hap_sign, truth, flip_p, miss_p, qual_lo, qual_hi):
    """Turn per-read covered SNP ranges [lo, hi) into CSR observations."""
    counts = (hi - lo).astype(np.int64)
    total = int(counts.sum())
    rid = np.repeat(np.arange(lo.shape[0], dtype=np.int64), counts)
    first = np.repeat(lo.astype(np.int64), counts)
    offs = np.arange(total, dtype=np.int64) - np.repeat(np.cumsum(counts) - counts, counts)
    snp = (first + offs).astype(np.int64)
    keep = rng.random(total) >= miss_p if miss_p > 0 else np.ones(total, bool)
    rid, snp = rid[keep], snp[keep]
    allele = (hap_sign[rid] * truth[snp]).astype(np.int8)
    flips = rng.random(rid.shape[0]) < flip_p
    allele[flips] = -allele[flips]
    qual = rng.integers(qual_lo, qual_hi + 1, size=rid.shape[0]).astype(np.uint8)
    ptr = np.zeros(lo.shape[0] + 1, np.int64)
    np.add.at(ptr, rid + 1, 1)
    return np.cumsum(ptr), snp.astype(np.int32), allele, qual


def reads_on_positions(rng, positions, truth, n_reads, region, len_mean, len_sd,
                       len_max=None, flip_p=0.01, miss_p=0.0, qual=(20, 40), info=None):
    """Long reads with lognormal lengths placed uniformly on [0, region - len].
    info (a dict, if given) receives "hap": each read's haplotype (+1 = truth, -1 = its
    complement), in the returned read order."""
    mu, sig = _lognormal_params(len_mean, len_sd)
    lens = rng.lognormal(mu, sig, size=n_reads)
    if len_max is not None:
        lens = np.minimum(lens, len_max)
    lens = np.maximum(lens, 1.0).astype(np.int64)
    lens = np.minimum(lens, region)
    starts = (rng.random(n_reads) * (region - lens + 1)).astype(np.int64)
    order = np.argsort(starts, kind="stable")
    starts, lens = starts[order], lens[order]
    lo = np.searchsorted(positions, starts, side="left")
    hi = np.searchsorted(positions, starts + lens, side="left")
    hap = np.where(rng.random(n_reads) < 0.5, 1, -1).astype(np.int8)
    ptr, snp, allele, q = _emit(rng, positions.shape[0], lo, hi, hap, truth,
                                flip_p, miss_p, qual[0], qual[1])
    if info is not None:
        info["hap"] = hap
    return ptr, snp, allele, q


def _concat(parts, n_snps):
    ptrs, snps, alls, quals, porec = [], [], [], [], []
    base = 0
    for ptr, snp, allele, q, pc in parts:
        ptrs.append(ptr[1:] + base if ptrs else ptr + base)
        base += int(ptr[-1])
        snps.append(snp)
        alls.append(allele)
        quals.append(q)
        porec.append(np.full(ptr.shape[0] - 1, pc, np.uint8))
    return (np.concatenate(ptrs).astype(np.int64), np.concatenate(snps).astype(np.int32),
            np.concatenate(alls).astype(np.int8), np.concatenate(quals).astype(np.uint8),
            np.concatenate(porec).astype(np.uint8))


def tiny_reads(seed=1001, n_snps=300, n_reads=80, len_lo=10, len_hi=30, flip_p=0.03,
               miss_p=0.0, qual=(30, 30)):
    """Smallest workload: reads covering 10-30 consecutive SNPs at index positions."""
    rng = np.random.Generator(np.random.PCG64(seed))
    truth = np.where(rng.random(n_snps) < 0.5, 1, -1).astype(np.int8)
    lens = rng.integers(len_lo, len_hi + 1, size=n_reads)
    starts = np.array([rng.integers(0, n_snps - L + 1) for L in lens], np.int64)
    order = np.argsort(starts, kind="stable")
    lo = starts[order]
    hi = lo + lens[order]
    hap = np.where(rng.random(n_reads) < 0.5, 1, -1).astype(np.int8)
    ptr, snp, allele, q = _emit(rng, n_snps, lo, hi, hap, truth, flip_p, miss_p, qual[0], qual[1])
    return Fragments(n_snps, ptr, snp, allele, q, np.zeros(n_reads, np.uint8),
                     np.arange(n_snps, dtype=np.int64), truth,
                     {"workload": "tiny-reads", "seed": seed, "n_reads": n_reads,
                      "read_hap": hap})


def region_reads(seed, n_snps=12000, region=4_000_000, n_reads=7200, len_mean=15_000,
                 len_sd=5_000, len_max=None, flip_p=0.01, miss_p=0.02, qual=(20, 40),
                 name="hifi-region"):
    """Regional long-read workload: SNPs uniform over the region, reads sorted by start."""
    rng = np.random.Generator(np.random.PCG64(seed))
    positions = np.sort(rng.choice(region, size=n_snps, replace=False)).astype(np.int64)
    truth = np.where(rng.random(n_snps) < 0.5, 1, -1).astype(np.int8)
    info = {}
    ptr, snp, allele, q = reads_on_positions(rng, positions, truth, n_reads, region, len_mean,
                                             len_sd, len_max, flip_p, miss_p, qual, info)
    return Fragments(n_snps, ptr, snp, allele, q, np.zeros(n_reads, np.uint8), positions,
                     truth, {"workload": name, "seed": seed, "n_reads": n_reads,
                             "region_bp": region, "read_hap": info["hap"]})


def hifi_region(seed=1002, scale=1.0):
    """12,000 het SNPs over 4 Mb, ~7,200 HiFi-like reads (15 kb +- 5 kb, 1% error, 2% missing)."""
    return region_reads(seed, n_snps=int(round(12000 * scale)), region=int(4_000_000 * scale),
                        n_reads=int(round(7200 * scale)), len_mean=15_000, len_sd=5_000,
                        flip_p=0.01, miss_p=0.02, qual=(20, 40), name="hifi-region")


def ont_region(seed=1003, scale=1.0):
    """Same region shape, ~3,600 ONT-like reads (30 kb +- 20 kb, cap 150 kb, 6% error, Q 7-30)."""
    return region_reads(seed, n_snps=int(round(12000 * scale)), region=int(4_000_000 * scale),
                        n_reads=int(round(3600 * scale)), len_mean=30_000, len_sd=20_000,
                        len_max=150_000, flip_p=0.06, miss_p=0.0, qual=(7, 30),
                        name="ont-region")


def batched_blocks(seed=1004, n_blocks=512, n_min=50, n_max=6000, gap=1_000_000,
                   snp_per_kb=3.0):
    """Independent HiFi-like phase blocks of log-uniform read counts, laid end to end.

    Block b holds N_b reads over a region of N_b * 15 kb / 30 (about 30x) with its own
    SNPs; a gap without SNPs separates blocks so no read links two blocks.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=n_blocks))).astype(int)
    parts, positions, truths, haps = [], [], [], []
    snp_base, bp_base = 0, 0
    for b, nb in enumerate(sizes):
        brng = np.random.Generator(np.random.PCG64(40000 + b))
        region = int(nb * 15_000 / 30)
        ns = max(2, int(round(region * snp_per_kb / 1000)))
        pos = np.sort(brng.choice(region, size=ns, replace=False)).astype(np.int64)
        tr = np.where(brng.random(ns) < 0.5, 1, -1).astype(np.int8)
        info = {}
        ptr, snp, allele, q = reads_on_positions(brng, pos, tr, int(nb), region, 15_000, 5_000,
                                                 None, 0.01, 0.02, (20, 40), info)
        haps.append(info["hap"])
        parts.append((ptr, snp + snp_base, allele, q, 0))
        positions.append(pos + bp_base)
        truths.append(tr)
        snp_base += ns
        bp_base += region + gap
    ptr, snp, allele, q, pc = _concat(parts, snp_base)
    return Fragments(snp_base, ptr, snp, allele, q, pc, np.concatenate(positions),
                     np.concatenate(truths), {"workload": "batched-blocks", "seed": seed,
                                              "block_reads": sizes.tolist(),
                                              "read_hap": np.concatenate(haps)})


def porec_contacts(rng, positions, truth, n_contacts, k_lo=2, k_hi=6, d_lo=100_000,
                   d_hi=50_000_000, wrong_hap_p=0.10, qual=(7, 30)):
    """Pore-C multi-way contacts: k SNPs, each next one a log-uniform distance downstream."""
    n = positions.shape[0]
    end = int(positions[-1])
    rows = []
    ks = rng.integers(k_lo, k_hi + 1, size=n_contacts)
    firsts = rng.integers(0, n, size=n_contacts)
    kmax = int(ks.max())
    cur = positions[firsts].astype(np.float64)
    idx = np.full((n_contacts, kmax), -1, np.int64)
    idx[:, 0] = firsts
    alive = np.ones(n_contacts, bool)
    for c in range(1, kmax):
        d = np.exp(rng.uniform(np.log(d_lo), np.log(d_hi), size=n_contacts))
        tgt = cur + d
        alive &= (c < ks) & (tgt <= end)
        j = np.searchsorted(positions, tgt, side="left")
        j = np.clip(j, 0, n - 1)
        jm = np.clip(j - 1, 0, n - 1)
        pick = np.where(np.abs(positions[jm] - tgt) < np.abs(positions[j] - tgt), jm, j)
        prev = idx[:, c - 1]
        pick = np.where(pick <= prev, prev + 1, pick)
        ok = alive & (pick < n)
        idx[ok, c] = pick[ok]
        alive = ok
        cur = np.where(ok, positions[np.clip(pick, 0, n - 1)], cur)
    counts = (idx >= 0).sum(axis=1)
    keep = counts >= 2
    idx, counts = idx[keep], counts[keep]
    m = idx.shape[0]
    flat = idx[idx >= 0]
    rid = np.repeat(np.arange(m), counts)
    hap = np.where(rng.random(m) < 0.5, 1, -1).astype(np.int8)
    allele = (hap[rid] * truth[flat]).astype(np.int8)
    wrong = rng.random(flat.shape[0]) < wrong_hap_p
    allele[wrong] = -allele[wrong]
    q = rng.integers(qual[0], qual[1] + 1, size=flat.shape[0]).astype(np.uint8)
    ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return ptr, flat.astype(np.int32), allele, q


def chromosome_porec(seed=1005, scale=1.0):
    """200,000 het SNPs over 250 Mb, 30x ONT-like reads plus 2M Pore-C contacts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_snps = int(round(200_000 * scale))
    region = int(250_000_000 * scale)
    positions = np.sort(rng.choice(region, size=n_snps, replace=False)).astype(np.int64)
    truth = np.where(rng.random(n_snps) < 0.5, 1, -1).astype(np.int8)
    n_reads = int(round(250_000 * scale))
    p1 = reads_on_positions(rng, positions, truth, n_reads, region, 30_000, 20_000, 150_000,
                            0.06, 0.0, (7, 30))
    p2 = porec_contacts(rng, positions, truth, int(round(2_000_000 * scale)))
    ptr, snp, allele, q, pc = _concat([(*p1, 0), (*p2, 1)], n_snps)
    return Fragments(n_snps, ptr, snp, allele, q, pc, positions, truth,
                     {"workload": "chromosome-porec", "seed": seed, "n_reads": n_reads})


def random_graph(seed, n, p=0.3, w_lo=-5, w_hi=5, integer=True):
    """Symmetric random weighted graph (dense, zero diagonal) for Max-Cut pins."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mask = np.triu(rng.random((n, n)) < p, 1)
    if integer:
        w = rng.integers(w_lo, w_hi + 1, size=(n, n)).astype(np.float64)
    else:
        w = rng.uniform(w_lo, w_hi, size=(n, n))
    w = np.where(mask, w, 0.0)
    return w + w.T
