"""Solver quality against the generator's truth on the HiFi-like region: how far the
best cut of multi-replica bSB stays below the cut of the true read partition, and the
phasing errors that follow, as the number of steps, the coupling scale c0 and the time
step dt change.

The paper's read-based runs use 10,000 iterations (its Table 1 setup); the default
schedule here is 1,000.  For every setting this builds the signed read graph on the
GPU, solves it (BF16, 1,024 replicas unless --replicas), phases it, and reports the
summed best cut, its ratio to the truth partition's cut, the switch and Hamming errors
and the device time of the solve.

    python -m paper_2603_25762_gb300.quality_sweep [--steps 1000,2000,4000,10000]
                                                   [--c0-scale 1,0.5,0.25] [--dt 1,0.5]
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", default="1000,2000,4000,10000")
    ap.add_argument("--c0-scale", default="1,0.5,0.25")
    ap.add_argument("--dt", default="1,0.5")
    ap.add_argument("--replicas", type=int, default=1024)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=1)
    args = ap.parse_args(argv)
    from . import build, metrics, qhap, synth
    build.build()
    fr = synth.hifi_region(1002, scale=args.scale)
    ctx = qhap.Context(0)
    g = ctx.build_graph(fr)
    rp, col, w = g.edges()
    truth_cut = metrics.partition_cut(rp, col, w, fr.meta["read_hap"])
    _, _, c0_default = g.layout()
    rows = []
    for steps in [int(v) for v in args.steps.split(",")]:
        for cs in [float(v) for v in args.c0_scale.split(",")]:
            for dt in [float(v) for v in args.dt.split(",")]:
                if len(c0_default) != 1:
                    raise SystemExit("the sweep expects one phase block")
                sol = ctx.solve(g, replicas=args.replicas, steps=steps, precision=qhap.PREC_BF16,
                                seed=args.seed, c0=float(c0_default[0]) * cs, dt=dt)
                h1, _, bid = ctx.phase(g, sol, fr.n_snps)
                se, he = metrics.switch_hamming(h1, bid, fr.truth)
                best = sol.block(0)["best_cut"]
                cuts = sol.cuts()[0]
                t = sol.timing()
                rows.append({"steps": steps, "c0_scale": cs, "dt": dt, "best_cut": best,
                             "median_cut": float(np.median(cuts)),
                             "best_over_truth": best / truth_cut, "switch_error": se,
                             "hamming_error": he, "solve_ms": t["solve_ms"],
                             "kernel": t["kernel"]})
                print(json.dumps(rows[-1]), flush=True)
    print(f"truth partition cut: {truth_cut:.0f}")
    print("| steps | c0 / default | dt | best cut | best / truth | median cut | SE % | HE % | "
          "solve ms |")
    print("|---|---|---|---|---|---|---|---|---|")
    for r in rows:
        print(f"| {r['steps']:,} | {r['c0_scale']} | {r['dt']} | {r['best_cut']:,.0f} | "
              f"{r['best_over_truth']:.4f} | {r['median_cut']:,.0f} | "
              f"{100 * r['switch_error']:.3f} | {100 * r['hamming_error']:.1f} | "
              f"{r['solve_ms']:.1f} |")


if __name__ == "__main__":
    main()
