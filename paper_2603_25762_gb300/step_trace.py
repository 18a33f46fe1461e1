"""Step timeline of the multi-step bSB kernel: where one step's time goes.

Runs one multi-step launch on a workload with the library's tracing hook
(qh_debug_run_trace), then reads the per-(CTA, step, item) stamps of the pipeline's
hand-off points and prints a summary:

  * the step period (epilogue start of a CTA's first item, step to step) and how much
    of it the epilogue warps are busy;
  * the epilogue side: its duration per item, its idle gap before each item, MMA
    commit to epilogue start;
  * the MMA side: product buffer free to MMAs committed, and whether the operands or
    the buffer gated the MMAs;
  * the producer side: waiting for the item's own previous step to be released, for
    the neighbour row tiles, for a ring slot, and the last operand load to the MMAs;
  * the release: epilogue end to the release of X_hat, and a release (global timer) to
    the moment the waiting producer saw it.

SM-clock stamps give durations inside one SM; global-timer stamps order events of
different SMs.

    python -m paper_2603_25762_gb300.step_trace [--workload hifi-region] [--steps 200]
"""
from __future__ import annotations

import argparse

import numpy as np

EV = ["deps", "loaded", "acc_free", "first_op", "mma_done", "epi_start", "epi_end", "release",
      "prod_start", "own", "slot", "slot1", "slot2", "slot3", "slot4", "slot5"]
E = {n: i for i, n in enumerate(EV)}
N_EV = len(EV)
CLOCK0 = 16  # first SM-clock column of a stamp row


def _q(a):
    a = np.asarray(a, np.float64)
    a = a[np.isfinite(a)]
    if a.size == 0:
        return "-"
    return (f"{np.median(a):8.2f} {np.percentile(a, 10):8.2f} {np.percentile(a, 90):8.2f}"
            f"  ({a.size})")


def clocks(stamps):
    """(global ns, SM cycles) arrays [cta, step, slot, event], NaN where not recorded."""
    g = stamps[..., :N_EV].astype(np.float64)
    c = stamps[..., CLOCK0:CLOCK0 + N_EV].astype(np.float64)
    g[stamps[..., :N_EV] == 0] = np.nan
    c[stamps[..., CLOCK0:CLOCK0 + N_EV] == 0] = np.nan
    return g, c


def analyse(stamps, items, n_kt, ns_per_cycle):
    """Summary rows (name, values in microseconds or fractions)."""
    n_cta, nu, n_slot, _ = stamps.shape
    g, c = clocks(stamps)
    us = ns_per_cycle / 1e3

    def d(a, b):  # duration from event a to event b on each SM's clock
        return (c[..., E[b]] - c[..., E[a]]) * us

    rows = [("step period (CTA, slot 0 to slot 0)",
             np.diff(c[:, :, 0, E["epi_start"]], axis=1) * us)]
    epi = d("epi_start", "epi_end")
    rows.append(("epilogue of one item (warp 2)", epi))
    n_items = (items >= 0).sum(1)
    gaps, busy, pidle = [], [], []
    for cta in range(n_cta):
        k = n_items[cta]
        if k == 0:
            continue
        s = c[cta, :, :k, E["epi_start"]].reshape(-1)
        e = c[cta, :, :k, E["epi_end"]].reshape(-1)
        gaps.append((s[1:] - e[:-1]) * us)
        s0 = c[cta, :, 0, E["epi_start"]]
        busy.append(np.nansum(epi[cta, :-1, :k], axis=1) / (np.diff(s0) * us))
        ps = c[cta, :, :k, E["prod_start"]].reshape(-1)
        pl = c[cta, :, :k, E["loaded"]].reshape(-1)
        pidle.append((ps[1:] - pl[:-1]) * us)
    rows.append(("epilogue idle before an item", np.concatenate(gaps)))
    rows.append(("epilogue busy fraction of a step", np.concatenate(busy)))
    rows.append(("MMA committed -> epilogue start", d("mma_done", "epi_start")))
    rows.append(("product buffer free -> MMA committed", d("acc_free", "mma_done")))
    gate = c[..., E["first_op"]] > c[..., E["acc_free"]]
    rows.append(("share of MMAs waiting on operands (not on the buffer)",
                 gate[np.isfinite(c[..., E["first_op"]])].astype(np.float64)))
    rows.append(("producer: previous item loaded -> reaches this item", np.concatenate(pidle)))
    rows.append(("producer: reaches item -> own previous step released", d("prod_start", "own")))
    rows.append(("producer: own released -> all inputs released", d("own", "deps")))
    rows.append(("producer: reaches item -> first ring slot free", d("prod_start", "slot")))
    rows.append(("producer: all inputs released -> last load issued", d("deps", "loaded")))
    for j in range(1, 6):
        rows.append((f"producer: ring slot of K-slice {j - 1} -> of K-slice {j}",
                     d("slot" if j == 1 else f"slot{j - 1}", f"slot{j}")))
    rows.append(("last load issued -> MMA committed", d("loaded", "mma_done")))
    rows.append(("epilogue end -> X_hat released", d("epi_end", "release")))
    # own release at step u-1 (global timer) -> the producer seeing it at step u
    own = (g[:, 1:, :, E["own"]] - g[:, :-1, :, E["release"]]) / 1e3
    rows.append(("own release -> producer sees it (global timer)", own))
    # a neighbour's release of step u-1 -> the waiter's inputs released at step u
    where = {}
    for cta in range(n_cta):
        for sl in range(n_slot):
            if items[cta, sl] >= 0:
                where[int(items[cta, sl])] = (cta, sl)
    hand = []
    for cta in range(n_cta):
        for sl in range(n_slot):
            it = int(items[cta, sl])
            if it < 0:
                continue
            rt, k = divmod(it, n_kt)
            for nb in (rt - 1, rt + 1):
                src = where.get(nb * n_kt + k)
                if src is None or src[0] == cta:
                    continue
                hand.append((g[cta, 1:, sl, E["deps"]] - g[src[0], :-1, src[1], E["release"]]) / 1e3)
    rows.append(("neighbour release -> waiter's inputs released (global timer)",
                 np.concatenate(hand) if hand else np.zeros(0)))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="hifi-region",
                    choices=["hifi-region", "ont-snp", "batched-blocks"])
    ap.add_argument("--kernel", default="multistep-stream-tile")
    ap.add_argument("--replicas", type=int, default=0)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--u0", type=int, default=100)
    ap.add_argument("--nu", type=int, default=32)
    ap.add_argument("--save", default=None, help="also write the raw stamps (.npz)")
    args = ap.parse_args()
    from . import build, qhap, synth
    build.build()
    gen = {"hifi-region": (synth.hifi_region, 1002, 1024, qhap.MODE_READ),
           "ont-snp": (synth.ont_region, 1003, 512, qhap.MODE_SNP),
           "batched-blocks": (lambda s: synth.batched_blocks(s, n_blocks=24), 1004, 256,
                              qhap.MODE_READ)}[args.workload]
    fr = gen[0](gen[1])
    R = args.replicas or gen[2]
    ctx = qhap.Context(0)
    g = ctx.build_graph(fr, mode=gen[3])
    stamps, items = ctx.debug_run_trace(g, R, args.kernel, args.steps, args.u0, args.nu)
    if args.save:
        np.savez_compressed(args.save, stamps=stamps, items=items, n_kt=R // 128)
    # SM clock to ns: the ratio of the two clocks over each CTA's traced window
    gs, cs = clocks(stamps)
    ratios = []
    for cta in range(stamps.shape[0]):
        m = np.isfinite(gs[cta]) & np.isfinite(cs[cta])
        if m.sum() > 10 and np.ptp(cs[cta][m]) > 0:
            ratios.append(np.ptp(gs[cta][m]) / np.ptp(cs[cta][m]))
    ns_per_cycle = float(np.median(ratios))
    gv = np.unique(gs[np.isfinite(gs)])
    step = np.diff(gv)
    print(f"workload {args.workload}, kernel {args.kernel}, R = {R}, steps {args.steps}, "
          f"traced steps {args.u0}..{args.u0 + args.nu - 1}, {stamps.shape[0]} CTAs, "
          f"items per CTA {np.bincount((items >= 0).sum(1)).tolist()}")
    print(f"SM clock: {1e3 / ns_per_cycle:.0f} MHz (global timer over SM clock); global timer "
          f"resolution: {step[step > 0].min() if step.size else 0:.0f} ns")
    print(f"{'quantity (us)':62s} {'median':>8s} {'p10':>8s} {'p90':>8s}  (samples)")
    for name, vals in analyse(stamps, items, R // 128, ns_per_cycle):
        print(f"{name:62s} {_q(vals)}")


if __name__ == "__main__":
    main()
