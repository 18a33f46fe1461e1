"""Benchmark of the QHap bSB phasing hot path on GB300.

One step = one pass of the whole path on one synthetic input already resident in HBM:
read graph build -> components and J tiles -> batched bSB (all replicas, all steps) ->
exact cut + replica pick -> read voting.  Workload (default): 12,000 het SNPs over 4 Mb,
7,200 HiFi-like reads (15 +- 5 kb, 1% allele error, 2% missing), signed read graph,
1,024 replicas x 1,000 bSB steps.

Metric: bSB spin-updates/s = sum over blocks of N_b * R * steps / step time.
`e2e` repeats the step through the C ABI with host buffers: fragments copied from pinned
host memory and haplotypes + cut copied back inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32]
                       [--impl ours|reference]
Under torchrun each rank runs its own replica range (replica_base = rank * R, weak scaling)
and the per-block best is combined across ranks; --shard blocks splits the phase blocks
by cost instead (strong scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402



def spin_update_work(deg, R, j_bytes):
    """Algorithmic work of one spin update (one vertex, one replica, one step), the
    measurement plan's model whatever a kernel keeps on chip:
      bytes = 16 (x, y FP32 read + write) + 2 (X_hat BF16 write) + deg * j_bytes / R
              (J streamed once per step, amortised over the R replicas)
      flops = 2 deg
    deg = stored J entries per vertex, j_bytes = bytes per stored entry."""
    return 16.0 + 2.0 + deg * j_bytes / R, 2.0 * deg


def kernel_bound(kernel):
    """What binds a step kernel, from its ncu captures: the multi-step and band-tile
    kernels keep the state in L2 / TMEM and wait on latency (hand-offs, gathers), the
    FP32 SIMT step is bound by FP32 arithmetic on the tiles."""
    if kernel == "k_step_f32":
        return "alu"
    return "latency"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device=0):
        self.device = device
        self.proc = None
        self.lines = []  # (arrival time, csv line)
        self.t_start = 0.0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a moment to start: let its first sample arrive before the
            # timed region, then keep only the samples taken inside it
            t_end = time.monotonic() + 3.0
            while not self.lines and time.monotonic() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
        except OSError:
            self.proc = None
        self.t_start = time.monotonic()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [ln for t, ln in self.lines if t >= self.t_start]
        for ln in inside or [ln for _, ln in self.lines[-1:]]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for k, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(k)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


WORKLOADS = {
    # name: (generator, mode, replicas, bsb steps, description)
    "hifi-region": ("hifi_region", "read", 1024, 1000,
                    "hifi-region: 12,000 SNPs / 4 Mb, 7,200 reads, signed read graph"),
    "ont-snp": ("ont_region", "snp", 512, 2000,
                "ont-snp: 12,000 SNPs / 4 Mb, 3,600 ONT-like reads, SNP graph + refinement"),
    "batched-blocks": ("batched_blocks", "read", 256, 1000,
                       "batched-blocks: 512 HiFi-like blocks of 50-6,000 reads, one launch per step"),
    "chromosome-porec": ("chromosome_porec", "snp", 128, 2000,
                         "chromosome-porec: 200,000 SNPs / 250 Mb, 250,000 ONT-like reads + 2M "
                         "Pore-C contacts, SNP graph (CSR storage), 2 refinement iterations"),
}
SEEDS = {"hifi_region": 1002, "ont_region": 1003, "batched_blocks": 1004,
         "chromosome_porec": 1005}
REFINE_DEFAULT = {"ont-snp": 15, "chromosome-porec": 2}
# default timed steps: about a second of timed work (several clock samples) per workload
STEPS_DEFAULT = {"hifi-region": 40, "ont-snp": 10, "batched-blocks": 4, "chromosome-porec": 3}
# timed passes of each workload summarised beside the headline line
OTHER_STEPS = {"hifi-region": 10, "ont-snp": 5, "batched-blocks": 2, "chromosome-porec": 2}

# The paper's own comparison (Results, Performance, Table 1): full-pipeline wall times in
# seconds on the MHC region of GIAB HG002 at 50x, read parsing and preprocessing included.
# Context for a reader of the line, not a target: other data, other hardware, and the
# whole pipeline rather than the synthetic hot path timed here.
PAPER_CONTEXT = {
    "source": "paper, Results (Performance), Table 1: MHC region, HG002 50x, full pipeline",
    "hardware": "QHap: Intel Core i7-14650HX (8 threads) + GeForce RTX 5060 Laptop GPU; "
                "HapCUT2 and WhatsHap: one CPU thread",
    "wall_s": {
        "cycloneseq": {"qhap_read": 63.454, "qhap_snp": 69.634, "hapcut2": 913.032,
                       "whatshap": 304.100},
        "hifi": {"qhap_read": 89.178, "qhap_snp": 45.278, "hapcut2": 858.700,
                 "whatshap": 318.600},
        "ont": {"qhap_read": 115.709, "qhap_snp": 57.059, "hapcut2": 1150.967,
                "whatshap": 493.300},
    },
}


def paper_speedups():
    """The paper's speedups of its faster QHap mode over HapCUT2 and WhatsHap, per dataset."""
    out = {}
    for ds, t in PAPER_CONTEXT["wall_s"].items():
        q = min(t["qhap_read"], t["qhap_snp"])
        out[ds] = {"vs_hapcut2": round(t["hapcut2"] / q, 1), "vs_whatshap": round(t["whatshap"] / q, 1)}
    return out


def _workload(args):
    from paper_2603_25762_gb300 import synth
    gen, mode, R, T, desc = WORKLOADS[args.workload]
    scale = getattr(args, "scale", 1.0)
    if scale != 1.0:  # a reduced case of the same shape, for profiler captures
        if gen == "batched_blocks":
            fr = synth.batched_blocks(SEEDS[gen], n_blocks=max(1, int(round(512 * scale))))
        else:
            fr = getattr(synth, gen)(SEEDS[gen], scale=scale)
        desc = f"{desc} [reduced: scale {scale}]"
    else:
        fr = getattr(synth, gen)(SEEDS[gen])
    R = args.replicas or R
    T = args.bsb_steps or T
    if args.refine_max <= 0:
        args.refine_max = REFINE_DEFAULT.get(args.workload, 15)
    cfg = {"workload": desc, "mode": mode, "n_reads": fr.n_frags, "n_snps": fr.n_snps,
           "replicas": R, "bsb_steps": T, "precision": args.precision,
           "refine_max": REFINE_DEFAULT.get(args.workload, 15) if mode == "snp" else None,
           "sb_variant": getattr(args, "variant", "ballistic"),
           "linkage_k": getattr(args, "linkage_k", 10) if mode == "snp" else None,
           "deform": ({"h": args.deform_h, "tries": args.deform_tries}
                      if mode == "snp" and getattr(args, "deform_h", 0.0) > 0 else None),
           "early_stop": ({"check_every": args.check_every, "patience": args.patience,
                           "checks": ("between launches" if getattr(args, "check_mode", 0) else
                                      "inside the multi-step launch where it applies")}
                          if getattr(args, "check_every", 0) > 0 and getattr(args, "patience", 0) > 0
                          else None),
           "l2": "flushed between timed steps (256 MiB write)"}
    if scale != 1.0:
        cfg["scale"] = scale
    return fr, cfg, mode, R, T


def _cpu_model():
    """The host CPU as /proc/cpuinfo names it (model name, else implementer and part)."""
    import platform
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return platform.machine()
    for line in info:
        if line.lower().startswith("model name"):
            return line.split(":", 1)[1].strip()
    impl = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU implementer")]
    part = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU part")]
    if impl and part:
        return f"{platform.machine()} (implementer {impl[0]}, part {part[0]})"
    return platform.machine()


def cpu_baseline(args, fr, mode, steps, seed=1, reps=None):
    """The FP64 oracle, as it stands, on the host cores: graph, blocks, bSB on a replica
    subset with the full step count, then voting or refinement + parity."""
    from oracle import oracle as o
    from paper_2603_25762_gb300 import synth
    o.build()
    reps = min(reps or args.ref_replicas, args.ref_replicas)
    if args.workload == "hifi-region":
        sample_fr, what = fr, f"full graph ({fr.n_frags} reads)"
    elif args.workload == "chromosome-porec":
        sample_fr = synth.chromosome_porec(1005, scale=0.05)
        what = f"1/20-scale chromosome ({sample_fr.n_frags} fragments, {sample_fr.n_snps} SNPs)"
        reps = min(reps, 16)
    elif args.workload == "ont-snp":
        sample_fr = synth.ont_region(1003, scale=0.25)
        what = f"quarter-size region ({sample_fr.n_frags} reads, {sample_fr.n_snps} SNPs)"
        reps = min(reps, 32)
    else:
        sample_fr = synth.batched_blocks(1004, n_blocks=16)
        what = "first 16 of the 512 blocks"
        reps = min(reps, 64)
    t0 = time.perf_counter()
    if mode == "read":
        res = o.phase_read(sample_fr, o.READ_SIGNED, range(reps), steps, seed=seed)
        units = sum(len(b) for b in res["blocks"]) * reps * steps
    else:
        res = o.phase_snp(sample_fr, range(reps), steps, seed=seed, refine_max=args.refine_max,
                          deform_h=args.deform_h, deform_tries=args.deform_tries)
        units = sum(len(b) * int(k) for b, k in zip(res["blocks"], res["solves"])) * reps * steps
    dt = time.perf_counter() - t0
    return {"value": units / dt, "unit": "spin-updates/s", "cores": os.cpu_count(),
            "cpu_model": _cpu_model(), "kind": "oracle", "replicas": reps,
            "sample": f"{what}, {reps} replicas x {steps} steps, whole path, {dt:.1f} s"}, res


def _profiled(kernel, workload="hifi-region"):
    """DRAM bytes per launch and the utilisation counters from the committed ncu summary
    of the kernel on this workload, or None when there is none or the kernel (its variant
    or its source file) differs from the one that was profiled."""
    import hashlib
    multistep = kernel.startswith("multistep")
    wl = workload.replace("-", "_")
    path = os.path.join(ROOT, "profiles", f"multistep_kernel_{wl}.md" if multistep
                        else f"step_kernel_{wl}.md")
    src = os.path.join(ROOT, "paper_2603_25762_gb300", "csrc",
                       "bsb_run.cu" if multistep else "bsb_tc.cu")
    if not os.path.exists(path):
        return None
    fields = {}
    keys = ("traffic_bytes_per_launch", "kernel", "source_sha256_16", "tensor_pipe_pct",
            "l2_throughput_pct", "dram_throughput_pct", "issue_active_pct")
    for line in open(path):
        if ":" in line and line.split(":")[0] in keys:
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if fields.get("kernel") != kernel or fields.get("source_sha256_16") != sha:
        return None
    out = {"traffic": int(fields["traffic_bytes_per_launch"]),
           "profile": os.path.relpath(path, ROOT)}
    for k in keys[3:]:
        if k in fields:
            out[k] = float(fields[k])
    return out


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    fr, cfg, mode, R, T = _workload(args)
    # size each step's sample so that the whole warm-up + timed run stays near 150 s:
    # one small calibration run, then replicas in proportion to the time left per step
    t0 = time.perf_counter()
    cpu_baseline(args, fr, mode, T, reps=8)
    t_cal = time.perf_counter() - t0
    per_step = max(1.0, (150.0 - t_cal) / (args.warmup + args.steps))
    reps = max(8, int(8 * per_step / max(t_cal, 1e-3)) // 8 * 8)
    runs = []
    for i in range(args.warmup + args.steps):
        cb, _ = cpu_baseline(args, fr, mode, T, reps=reps)
        if i >= args.warmup:
            runs.append(cb)
    value = statistics.median([c["value"] for c in runs])
    line = {"impl": "reference", "metric": "bSB spin-updates/s", "value": value,
            "unit": "spin-updates/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "spin-updates/s", "cores": os.cpu_count(),
                             "cpu_model": _cpu_model(), "kind": "oracle",
                             "sample": runs[-1]["sample"]},
            "e2e": {"value": value, "unit": "spin-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def other_workloads(args):
    """The ONT-like, batched and chromosome + Pore-C workloads, each measured by this
    script in a process of its own (a few timed passes, no CPU baseline), summarised
    beside the headline line."""
    import subprocess
    import sys
    out = {}
    for wl in sorted(WORKLOADS):
        if wl == args.workload:
            continue
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", wl, "--steps",
               str(OTHER_STEPS.get(wl, 2)), "--warmup", "3", "--no-cpu-baseline",
               "--no-other-workloads", "--fp32-steps", "1", "--precision", args.precision]
        r = subprocess.run(cmd, capture_output=True, text=True)
        lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
        if r.returncode != 0 or not lines:
            out[wl] = {"error": (r.stderr.strip().splitlines() or ["no output"])[-1][:300]}
            continue
        d = json.loads(lines[-1])
        rf = d["roofline"]
        q = d["quality"]
        v = d.get("vs_fp32") or {}
        out[wl] = {
            "config": d["config"], "steps": d["steps"], "warmup": d["warmup"],
            "ms_per_step": d["ms_per_step"], "value": d["value"], "unit": d["unit"],
            "e2e": d["e2e"], "breakdown_ms": d["breakdown_ms"],
            "roofline": {k: rf[k] for k in ("bound", "kernel", "achieved", "peak", "unit",
                                            "frac", "traffic", "avg_launch_us",
                                            "launches_per_step", "bytes_per_spin_update",
                                            "tensor", "ncu")},
            "quality": {k: q[k] for k in ("best_cut_sum", "truth_cut", "best_over_truth",
                                          "switch_error", "hamming_error", "n50_bp")},
            "vs_fp32": {k: v.get(k) for k in ("fp32_ms_per_step", "fp32_kernel", "speedup",
                                              "cut_ratio", "fp32_steps")},
            "clocks": d["clocks"], "gpu_launches": d["gpu_launches"]}
    return out


def run_ours(args):
    import torch
    ws, rank = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_2603_25762_gb300 import build, qhap
    build.build()
    fr, cfg, mode, R, T = _workload(args)
    prec = {"bf16": qhap.PREC_BF16, "bf16x2": qhap.PREC_BF16X2, "fp8": qhap.PREC_FP8,
            "fp32": qhap.PREC_FP32}[args.precision]
    gmode = qhap.MODE_READ if mode == "read" else qhap.MODE_SNP
    stream = torch.cuda.Stream()
    ctx = qhap.Context(local, stream=stream.cuda_stream)
    # inputs resident in HBM
    dev = torch.device("cuda", local)
    arrays_dev = (fr.n_snps, torch.from_numpy(fr.frag_ptr).to(dev), torch.from_numpy(fr.snp).to(dev),
                  torch.from_numpy(fr.allele).to(dev), torch.from_numpy(fr.qual).to(dev),
                  torch.from_numpy(fr.is_porec).to(dev))
    outs = (torch.empty(fr.n_snps, dtype=torch.int8, device=dev),
            torch.empty(fr.n_snps, dtype=torch.int8, device=dev),
            torch.empty(fr.n_snps, dtype=torch.int32, device=dev))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    from paper_2603_25762_gb300 import multi
    base, _ = multi.replica_range(rank, ws, R)
    stats = {}

    def one_step(host=False, pinned=None, precision=None, collect=False):
        """One pass of the whole path. collect=True also records the per-block figures
        (block sizes, refinement iterations, best cuts): host loops kept out of the
        timed steps."""
        t0 = time.perf_counter()
        p = prec if precision is None else precision
        if host:
            g = ctx.build_graph(arrays=pinned, on_device=False, mode=gmode, linkage_k=args.linkage_k)
        else:
            g = ctx.build_graph(arrays=arrays_dev, on_device=True, mode=gmode, linkage_k=args.linkage_k)
        stats["build_ms"] = (time.perf_counter() - t0) * 1e3
        kw = dict(replicas=R, steps=T, precision=p, seed=1,
                  step_kernel=args.step_kernel if p == prec else None,
                  refine_max=args.refine_max,
                  variant=args.variant, dt=0.1 if args.variant == "adiabatic" else 1.0,
                  deform_h=args.deform_h, deform_tries=args.deform_tries,
                  check_every=args.check_every, patience=args.patience,
                  check_mode=args.check_mode)
        if ws > 1 and args.shard == "blocks":
            # this rank's share of the blocks by cost, then the per-block exchange
            sol = multi.solve_blocks_sharded(ctx, g, rank, ws, **kw)
        else:
            sol = ctx.solve(g, replica_base=base, **kw)
            if ws > 1:  # replica shards: every block takes the best rank's result
                multi.combine_replica_shards(sol, g)
        if host:
            h = ctx.phase(g, sol, fr.n_snps)
            cut = sol.block(0)["best_cut"] if g.n_blocks else 0.0
        else:
            h = ctx.phase(g, sol, fr.n_snps, out=outs)
            cut = None
        stats["timing"] = sol.timing()
        stats["phase_ms"] = (time.perf_counter() - t0) * 1e3 - stats["build_ms"] - stats["timing"]["solve_ms"]
        stats["blocks"] = g.n_blocks
        stats["units"] = sol.timing()["spin_updates"]
        stats["nnz"] = g.nnz
        if collect:
            from paper_2603_25762_gb300 import metrics
            bs = g.block_sizes()
            info = [sol.block(b) for b in range(g.n_blocks)]
            stats["spins"] = float(sum(bs)) * R  # spin states updated per step
            stats["in_blocks"] = float(sum(bs))
            stats["best_cut_sum"] = float(sum(i["best_cut"] for i in info))
            stats["cuts"] = sol.cuts()  # every replica's cut, per block
            # the cut of the generator's true partition on the same graph (reads: each
            # read's haplotype; SNPs: the true haplotype), for the solver's gap to it
            truth = fr.meta.get("read_hap") if mode == "read" else fr.truth
            if truth is not None and not host:
                rp, col, w = g.edges()
                stats["truth_cut"] = metrics.partition_cut(rp, col, w, truth)
        sol.free()
        g.free()
        return h, cut

    def quality(h):
        """Phasing quality of one pass against the generator's truth (evaluation only)."""
        from paper_2603_25762_gb300 import metrics
        hap1, bid = h[0], h[2]
        if isinstance(hap1, torch.Tensor):
            hap1, bid = hap1.cpu().numpy(), bid.cpu().numpy()
        se, he = metrics.switch_hamming(hap1, bid, fr.truth)
        bid_ph = np.where(hap1 != 0, bid, -1)
        tc = stats.get("truth_cut")
        return {"best_cut_sum": stats["best_cut_sum"], "truth_cut": tc,
                "best_over_truth": stats["best_cut_sum"] / tc if tc else None,
                "switch_error": se, "hamming_error": he,
                "n50_bp": metrics.n50(metrics.block_spans(bid_ph, fr.positions)),
                "phased_fraction": metrics.completeness(hap1)}

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            one_step(collect=i == args.warmup - 1)
        times, step_ms, launches = [], [], []
        parts = {"graph_build": [], "solve": [], "bsb_step_launches": [], "phase_and_host": []}
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        k0 = qhap.kernel_launches()
        with ClockSampler(local) as clk:
            for _ in range(args.steps):
                flush.fill_(1)
                stream.synchronize()
                ev0.record(stream)
                h_last, _ = one_step()
                ev1.record(stream)
                ev1.synchronize()
                times.append(ev0.elapsed_time(ev1))
                step_ms.append(stats["timing"]["step_ms"] / stats["timing"]["n_step_launches"])
                parts["graph_build"].append(stats["build_ms"])
                parts["solve"].append(stats["timing"]["solve_ms"])
                parts["bsb_step_launches"].append(stats["timing"]["step_ms"])
                parts["phase_and_host"].append(stats["phase_ms"])
        torch.cuda.synchronize()
        n_launched = qhap.kernel_launches() - k0
        units = stats["units"]
        # e2e through the C ABI with host buffers (pinned), copies inside the timed region
        pinned = tuple([fr.n_snps] + [torch.from_numpy(a).pin_memory() for a in
                                      (fr.frag_ptr, fr.snp, fr.allele, fr.qual, fr.is_porec)])
        pinned_np = (pinned[0],) + tuple(t.numpy() for t in pinned[1:])
        one_step(host=True, pinned=pinned_np)
        e2e = []
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            one_step(host=True, pinned=pinned_np)
            e2e.append((time.perf_counter() - t0) * 1e3)
        qual = quality(h_last)
        # the same path with the plain FP32 SIMT step on the same GPU: the speedup of the
        # low-precision path at equal best cut
        vs_fp32 = None
        if prec != qhap.PREC_FP32 and not args.no_fp32_leg:
            saved = dict(stats)
            one_step(precision=qhap.PREC_FP32, collect=True)
            t32 = []
            for _ in range(args.fp32_steps):
                flush.fill_(1)
                stream.synchronize()
                ev0.record(stream)
                h32, _ = one_step(precision=qhap.PREC_FP32)
                ev1.record(stream)
                ev1.synchronize()
                t32.append(ev0.elapsed_time(ev1))
            q32 = quality(h32)
            ms32 = statistics.mean(t32)
            vs_fp32 = {"fp32_ms_per_step": ms32, "fp32_kernel": stats["timing"]["kernel"],
                       "fp32_value": stats["units"] * ws / (ms32 / 1e3),
                       "fp32_steps": args.fp32_steps, "fp32_quality": q32}
            stats.clear()
            stats.update(saved)
    ms = statistics.mean(times)
    e2e_ms = statistics.mean(e2e)
    units_all = units * ws
    if ws > 1:  # the job's time is the slowest rank's
        ms = multi.max_over_ranks(ms)
        e2e_ms = multi.max_over_ranks(e2e_ms)
        if args.shard == "blocks":  # each rank ran its own blocks
            units_all = multi.sum_over_ranks(units)
        if vs_fp32 is not None:
            vs_fp32["fp32_ms_per_step"] = multi.max_over_ranks(vs_fp32["fp32_ms_per_step"])
    if rank != 0:
        return
    if vs_fp32 is not None:
        vs_fp32["speedup"] = vs_fp32["fp32_ms_per_step"] / ms
        c32 = vs_fp32["fp32_quality"]["best_cut_sum"]
        vs_fp32["cut_ratio"] = qual["best_cut_sum"] / c32 if c32 else None
    hbm, bf16_tf, src = _peaks()
    # Roofline of the dominant kernel, the step kernel: the measurement plan's work per
    # spin update (spin_update_work) times the spin updates of one launch, over that
    # launch's average duration from the library's CUDA events on the bench's stream.
    kname = stats["timing"]["kernel"]
    n_launch = max(1, stats["timing"]["n_step_launches"])
    launch_us = statistics.mean(step_ms) * 1e3
    deg = stats["nnz"] / max(1.0, stats["in_blocks"])  # stored J entries per vertex
    b_unit, f_unit = spin_update_work(deg, R, 4 if prec == qhap.PREC_FP32 else 2)
    per_launch = units / n_launch  # spin updates of one launch
    achieved = per_launch * b_unit / (launch_us * 1e-6) / 1e9
    achieved_tf = per_launch * f_unit / (launch_us * 1e-6) / 1e12
    prof = _profiled(kname, args.workload)
    h2d = sum(int(a.nbytes) for a in pinned_np[1:])
    d2h = fr.n_snps * (1 + 1 + 4) + 8
    line = {
        "metric": "bSB spin-updates/s", "value": units_all / (ms / 1e3),
        "unit": "spin-updates/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if ws > 1 and args.shard == "blocks" else "weak",
        "vs_baseline": None,
        "dtype": args.precision, "data": "synthetic", "config": cfg,
        "phasing_wall_ms": ms,
        "breakdown_ms": {k: round(statistics.mean(v), 3) for k, v in parts.items()},
        "e2e": {"value": units_all / (e2e_ms / 1e3), "unit": "spin-updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "roofline": {"bound": kernel_bound(kname), "kernel": kname,
                     "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_source": f"{src} HBM copy",
                     "traffic": prof["traffic"] if prof else None,
                     "model": "16 + 2 + deg * b_J / R bytes and 2 deg flops per spin update",
                     "deg": deg, "bytes_per_spin_update": b_unit,
                     "algorithmic_bytes_per_launch": per_launch * b_unit,
                     "avg_launch_us": launch_us, "launches_per_step": n_launch,
                     "tensor": {"achieved": achieved_tf, "peak": bf16_tf, "unit": "TFLOP/s",
                                "frac": achieved_tf / bf16_tf,
                                "peak_source": f"{src} BF16 dense burst"},
                     "ncu": prof},
        "quality": qual,
        "vs_fp32": vs_fp32,
        "gpu_launches": n_launched,
        "clocks": clk.summary(),
        "step_kernel_tuning": ctx.tuning_report(),
        "paper_context": dict(PAPER_CONTEXT, speedups=paper_speedups()),
    }
    if not args.no_cpu_baseline:
        cb, res = cpu_baseline(args, fr, mode, T)
        line["cpu_baseline"] = cb
        if mode == "read" and args.workload == "hifi-region" and "cuts" in stats:
            # cut parity on the oracle's sample: its best over replicas 0 .. r-1 of the
            # full graph against the GPU's best over the same replica indices
            r = cb["replicas"]
            gpu = float(sum(c[:r].max() for c in stats["cuts"]))
            ora = float(sum(res["cuts"]))
            cb["parity"] = {"replicas": r, "oracle_best_cut_sum": ora,
                            "gpu_best_cut_sum_same_replicas": gpu,
                            "gpu_over_oracle": gpu / ora if ora else None}
    if ws == 1 and not args.no_other_workloads:
        line["workloads"] = other_workloads(args)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="0 = the workload's default")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "bf16x2", "fp8", "fp32"])
    ap.add_argument("--workload", default="hifi-region", choices=sorted(WORKLOADS))
    ap.add_argument("--replicas", type=int, default=0, help="0 = the workload's")
    ap.add_argument("--bsb-steps", type=int, default=0, help="0 = the workload's")
    ap.add_argument("--refine-max", type=int, default=0, help="0 = the workload's (SNP graphs)")
    ap.add_argument("--ref-replicas", type=int, default=1024)
    ap.add_argument("--scale", type=float, default=1.0,
                    help="reduced workload of the same shape (profiler captures only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-leg", action="store_true",
                    help="skip timing the same path with the FP32 SIMT step")
    ap.add_argument("--fp32-steps", type=int, default=3)
    ap.add_argument("--shard", default="replicas", choices=["replicas", "blocks"],
                    help="under torchrun: each rank a replica range (weak scaling) or a "
                         "cost-balanced share of the phase blocks (strong scaling)")
    ap.add_argument("--variant", default="ballistic", choices=["ballistic", "discrete", "adiabatic"],
                    help="simulated-bifurcation variant (the paper's solver is ballistic)")
    ap.add_argument("--linkage-k", type=int, default=10, help="SNP graphs: linkage depth k/10")
    ap.add_argument("--deform-h", type=float, default=0.0,
                    help="SNP graphs: deformation field strength of the refinement's re-solves")
    ap.add_argument("--deform-tries", type=int, default=0,
                    help="SNP graphs: deformed re-solves after a failed solve")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="measure the chosen workload only (by default a 1-GPU run also "
                         "summarises the other workloads under 'workloads')")
    ap.add_argument("--check-every", type=int, default=0,
                    help="early stop: energy check period in bSB steps (0 = off)")
    ap.add_argument("--patience", type=int, default=0,
                    help="early stop: checks without a better best cut before a block stops")
    ap.add_argument("--check-mode", type=int, default=0, choices=[0, 1],
                    help="0 = checks inside the multi-step launch where it applies, 1 = between launches")
    ap.add_argument("--step-kernel", default=None,
                    help="pin the BF16 step-kernel variant (default: autotune)")
    args = ap.parse_args()
    if args.steps <= 0:
        args.steps = STEPS_DEFAULT[args.workload]
    args.warmup = max(1, args.warmup)  # the last warm-up pass records the per-block figures
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
