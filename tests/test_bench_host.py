"""Host-side logic of bench.py (no GPU): the clock sampler's parsing and its restriction
to the timed region, the per-workload defaults, and the profiled-traffic lookup that a
changed kernel source must invalidate."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _line(sm, mx, hw="Not Active", pc="Not Active"):
    return f"0, {sm}, {mx}, 900.0, 0x0, {hw}, Not Active, Not Active, {pc}"


def test_clock_summary_keeps_samples_inside_timed_region(bench):
    c = bench.ClockSampler()
    c.lines = [(0.5, _line(345, 2070)), (1.5, _line(2070, 2070)), (1.6, _line(2055, 2070)),
               (1.7, _line(2070, 2070, pc="Active"))]
    c.t_start = 1.0
    s = c.summary()
    assert s["samples"] == 3  # the idle sample before the region is dropped
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_slowdown_and_falls_back_to_last_sample(bench):
    c = bench.ClockSampler()
    c.lines = [(0.1, _line(1500, 2070, hw="Active"))]
    c.t_start = 5.0  # nothing arrived inside: the last sample stands in
    s = c.summary()
    assert s["samples"] == 1 and s["reasons"] == ["hw_slowdown"] and s["sm_mhz"] == 1500.0
    c.lines = [(6.0, "garbage"), (6.1, "0, [N/A], [N/A], 1, 2, 3, 4, 5, 6")]
    assert c.summary()["samples"] == 0


def test_workload_tables_agree(bench):
    assert set(bench.STEPS_DEFAULT) == set(bench.WORKLOADS)
    assert set(bench.OTHER_STEPS) == set(bench.WORKLOADS)
    assert all(k >= 1 for k in bench.STEPS_DEFAULT.values())
    for gen, *_ in bench.WORKLOADS.values():
        assert gen in bench.SEEDS


def test_profiled_traffic_tracks_kernel_source(bench, tmp_path, monkeypatch):
    import hashlib
    prof = tmp_path / "profiles"
    src = tmp_path / "paper_2603_25762_gb300" / "csrc"
    prof.mkdir()
    src.mkdir(parents=True)
    (src / "bsb_run.cu").write_text("// kernel v1\n")
    sha = hashlib.sha256(b"// kernel v1\n").hexdigest()[:16]
    (prof / "multistep_kernel_hifi_region.md").write_text(
        f"kernel: multistep-stream-tile\nsource_sha256_16: {sha}\n"
        "traffic_bytes_per_launch: 1234\ntensor_pipe_pct: 17.5\nl2_throughput_pct: 40.25\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench._profiled("multistep-stream-tile")
    assert got["traffic"] == 1234
    assert got["tensor_pipe_pct"] == 17.5 and got["l2_throughput_pct"] == 40.25
    assert "dram_throughput_pct" not in got
    assert bench._profiled("multistep-jres-group") is None  # another variant
    (src / "bsb_run.cu").write_text("// kernel v2\n")
    assert bench._profiled("multistep-stream-tile") is None  # source changed
    assert bench._profiled("multistep-stream-tile", "ont-snp") is None  # no summary
    (src / "bsb_run.cu").write_text("// kernel v1\n")
    (prof / "multistep_kernel_ont_snp.md").write_text(
        f"kernel: multistep-stream-tile\nsource_sha256_16: {sha}\n"
        "traffic_bytes_per_launch: 99\n")
    assert bench._profiled("multistep-stream-tile", "ont-snp")["traffic"] == 99
    assert bench._profiled("multistep-stream-tile")["traffic"] == 1234


def test_spin_update_work_follows_the_measurement_model(bench):
    # 16 B of x, y, 2 B of X_hat, J once per step over R replicas; 2 flops per entry
    b, f = bench.spin_update_work(52.8, 1024, 2)
    assert b == pytest.approx(18.0 + 52.8 * 2 / 1024) and f == pytest.approx(105.6)
    assert bench.kernel_bound("k_step_f32") == "alu"
    assert bench.kernel_bound("multistep-stream-tile") == "latency"


def test_paper_context_speedups(bench):
    # Table 1's HiFi row: QHap's SNP mode 45.278 s against HapCUT2's 858.700 s
    sp = bench.paper_speedups()
    assert sp["hifi"]["vs_hapcut2"] == 19.0 and sp["ont"]["vs_hapcut2"] == 20.2
    assert sp["cycloneseq"]["vs_whatshap"] == 4.8
