"""Phasing quality metrics: switch error, Hamming error, N50 (their definitions in Methods).

Evaluation only: these compare phased output with the generator's truth; they are
not part of the GPU path.

hap1[j]  : +1 / -1 = allele of the initial H1 / H2 on phased haplotype 1, 0 unphased
block[j] : phase block of SNP j, -1 if unphased
truth[j] : +1 / -1 on truth haplotype A
"""
from __future__ import annotations

import numpy as np


def switch_hamming(hap1, block, truth, orientation="best"):
    """Switch error rate and Hamming error rate over phased SNPs, per block.

    SE = switches / sum over blocks of (n_b - 1) adjacent phased pairs.
    HE = mismatching alleles / phased SNPs; with orientation="best" each block is
    compared with whichever truth haplotype it matches better, with "fixed" it is
    compared with truth haplotype A as given (the paper's worked example).
    """
    hap1 = np.asarray(hap1)
    block = np.asarray(block)
    truth = np.asarray(truth)
    switches = pairs = ham = phased = 0
    for b in np.unique(block[block >= 0]):
        idx = np.nonzero((block == b) & (hap1 != 0))[0]
        if idx.size == 0:
            continue
        err = (hap1[idx] != truth[idx]).astype(np.int64)
        switches += int(np.count_nonzero(err[1:] != err[:-1]))
        pairs += idx.size - 1
        e = int(err.sum())
        ham += e if orientation == "fixed" else min(e, idx.size - e)
        phased += idx.size
    se = switches / pairs if pairs else 0.0
    he = ham / phased if phased else 0.0
    return se, he


def string_example(inferred: str, reference: str):
    """SE and fixed-orientation HE of two 0/1 strings treated as one block."""
    h = np.array([1 if c == "0" else -1 for c in inferred], np.int8)
    t = np.array([1 if c == "0" else -1 for c in reference], np.int8)
    return switch_hamming(h, np.zeros(h.size, np.int64), t, orientation="fixed")


def block_spans(block, positions):
    """Span (last - first + 1 bp) of each phase block's phased SNPs."""
    block = np.asarray(block)
    positions = np.asarray(positions)
    spans = []
    for b in np.unique(block[block >= 0]):
        p = positions[block == b]
        spans.append(int(p.max() - p.min() + 1))
    return np.array(spans, np.int64)


def n50(spans):
    """Length L such that blocks of span >= L cover at least half of the total span."""
    s = np.sort(np.asarray(spans, np.int64))[::-1]
    if s.size == 0:
        return 0
    c = np.cumsum(s)
    return int(s[np.searchsorted(c, 0.5 * c[-1], side="left")])


def completeness(hap1):
    """Fraction of SNPs that received a phase."""
    hap1 = np.asarray(hap1)
    return float(np.count_nonzero(hap1)) / max(1, hap1.size)


def partition_cut(row_ptr, col, w, spins):
    """Cut sum_{a<b} w_ab [s_a != s_b] of a +-1 partition of a graph given as CSR with both
    directions (evaluation only: e.g. the cut of the generator's true partition)."""
    row_ptr = np.asarray(row_ptr, np.int64)
    s = np.asarray(spins, np.int64)
    rows = np.repeat(np.arange(row_ptr.shape[0] - 1), np.diff(row_ptr))
    cross = s[rows] != s[np.asarray(col, np.int64)]
    return 0.5 * float(np.asarray(w, np.float64)[cross].sum())
