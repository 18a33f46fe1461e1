"""Ballistic, discrete and adiabatic simulated bifurcation side by side (the paper's
Max-Cut solver comparison, its Figs. 2-3) on the synthetic stand-ins: the
integer-weighted read graph of the HiFi-like region and the real-weighted,
mixed-sign SNP graph of the ONT-like region.

For each variant and step count, several seeds are solved with the same replicas;
the best cut's mean and standard deviation across seeds give convergence (versus
steps) and stability (spread), and the solve time the GPU cost.

    python -m paper_2603_25762_gb300.solver_compare [--replicas 256] [--seeds 5]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

DT = {"ballistic": 1.0, "discrete": 1.0, "adiabatic": 0.1}  # aSB: explicit cubic term


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--replicas", type=int, default=256)
    ap.add_argument("--seeds", type=int, default=5)
    ap.add_argument("--steps", default="100,300,1000,3000")
    args = ap.parse_args(argv)
    import torch

    from . import qhap, synth
    ctx = qhap.Context(0)
    graphs = [("read graph (integer, HiFi-like)", synth.hifi_region(1002), qhap.MODE_READ),
              ("SNP graph (real, mixed sign, ONT-like)", synth.ont_region(1003), qhap.MODE_SNP)]
    rows = []
    for gname, fr, mode in graphs:
        g = ctx.build_graph(fr, mode=mode)
        for variant in ("ballistic", "discrete", "adiabatic"):
            for steps in [int(s) for s in args.steps.split(",")]:
                cuts, ms = [], []
                for seed in range(1, args.seeds + 2):  # the first solve warms up
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    sol = ctx.solve(g, replicas=args.replicas, steps=steps, precision=qhap.PREC_BF16,
                                    seed=seed, dt=DT[variant], variant=variant, refine_max=1)
                    best = sum(sol.block(b)["best_cut"] for b in range(g.n_blocks))
                    sol.free()
                    torch.cuda.synchronize()
                    if seed > 1:
                        cuts.append(best)
                        ms.append((time.perf_counter() - t0) * 1e3)
                row = {"graph": gname, "variant": variant, "steps": steps,
                       "best_cut_mean": float(np.mean(cuts)), "best_cut_std": float(np.std(cuts)),
                       "solve_ms": round(float(np.median(ms)), 2)}
                rows.append(row)
                print(json.dumps(row), flush=True)
        g.free()
    print("| graph | variant | steps | best cut mean | std | solve ms |\n|---|---|---|---|---|---|")
    for r in rows:
        print(f"| {r['graph']} | {r['variant']} | {r['steps']} | {r['best_cut_mean']:.3f} | "
              f"{r['best_cut_std']:.3f} | {r['solve_ms']:.1f} |")


if __name__ == "__main__":
    main()
