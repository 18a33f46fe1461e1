"""Linkage-depth trade-off of the SNP-based graph (the paper's SNP linkage depth
analysis, its Fig. 4) on the synthetic ONT-like region.

Depth k/10 links each SNP of a read only to its floor(k (N-1) / 10)
nearest downstream SNPs in that read (N SNPs in the read); k = 10 links every pair.
For k = 1..10 this builds the SNP graph on the GPU, solves it with multi-replica bSB
and the iterative refinement, phases it, and reports the edge count, the core
phasing time (graph build + solve + phase, inputs already on the device) and the
switch / Hamming error against the generator's truth.

    python -m paper_2603_25762_gb300.linkage_sweep [--scale 1.0] [--replicas 512]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the 3,600 reads")
    ap.add_argument("--replicas", type=int, default=512)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--refine-max", type=int, default=15)
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--repeats", type=int, default=3)
    args = ap.parse_args(argv)
    import torch

    from . import metrics, qhap, synth
    prec = qhap.PREC_BF16 if args.precision == "bf16" else qhap.PREC_FP32
    fr = synth.ont_region(1003, scale=args.scale)
    dev = torch.device("cuda:0")
    arrays = tuple([fr.n_snps] + [torch.from_numpy(a).to(dev) for a in
                                  (fr.frag_ptr, fr.snp, fr.allele, fr.qual, fr.is_porec)])
    ctx = qhap.Context(0)
    rows = []
    for k in range(1, 11):
        times = []
        for rep in range(args.repeats + 1):  # the first run warms up (and tunes)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = ctx.build_graph(arrays=arrays, on_device=True, mode=qhap.MODE_SNP, linkage_k=k)
            sol = ctx.solve(g, replicas=args.replicas, steps=args.steps, precision=prec, seed=1,
                            refine_max=args.refine_max)
            hap1, _, bid = ctx.phase(g, sol, fr.n_snps)
            torch.cuda.synchronize()
            if rep:
                times.append((time.perf_counter() - t0) * 1e3)
            nnz, nb = g.nnz, g.n_blocks
            sol.free()
            g.free()
        se, he = metrics.switch_hamming(hap1, bid, fr.truth)
        rows.append({"linkage_k": k, "edges": nnz // 2, "blocks": nb,
                     "core_ms": round(float(np.median(times)), 2), "switch_error": se,
                     "hamming_error": he})
        print(json.dumps(rows[-1]), flush=True)
    print("| k/10 | edges | blocks | core ms | SE % | HE % |\n|---|---|---|---|---|---|")
    for r in rows:
        print(f"| {r['linkage_k']} | {r['edges']:,} | {r['blocks']} | {r['core_ms']:.1f} | "
              f"{100 * r['switch_error']:.4f} | {100 * r['hamming_error']:.4f} |")


if __name__ == "__main__":
    main()
