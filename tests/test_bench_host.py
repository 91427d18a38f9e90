"""Host-side logic of bench.py, on the CPU: the reference arm's JSON line
(the FP64 oracle timed on the host cores), the bias estimate of the cache
comparison, and the naming of the traversal kernels in the roofline."""
import json
import os
import subprocess
import sys

import numpy as np
import torch

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "C1", "--steps", "2",
                        "--warmup", "1", "--ref-step-s", "0.2"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"]
    assert isinstance(cpu["sample"], str) and cpu["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"].startswith("C1")


def test_image_stats_separates_bias_from_noise():
    """Batches X_b = (1 + beta) R + noise against a reference with its own
    noise: the noise-corrected bias recovers beta, the raw relative RMSE
    includes the noise."""
    g = torch.Generator().manual_seed(3)
    H, W, nb, beta, sx = 32, 32, 64, 0.02, 0.05
    R = 1.0 + torch.rand((H, W, 3), generator=g, dtype=torch.float64)
    R_batches = R + 0.01 * torch.randn((16, H, W, 3), generator=g, dtype=torch.float64)
    R_mean, R_var = R_batches.mean(0), R_batches.var(0) / 16
    X = (1 + beta) * R + sx * torch.randn((nb, H, W, 3), generator=g, dtype=torch.float64)
    st = bench.image_stats(X, R_mean, R_var)
    true_bias = float(torch.sqrt(((beta * R) ** 2).sum() / (R_mean ** 2).sum()))
    assert abs(st["bias_rel_rmse"] - true_bias) < 0.15 * true_bias, st
    assert st["rel_rmse"] > st["bias_rel_rmse"] and st["noise_rel_rmse"] > 0
    # no bias: the estimate is small and may come out negative (signed)
    st0 = bench.image_stats(R + sx * torch.randn((nb, H, W, 3), generator=g, dtype=torch.float64), R_mean, R_var)
    assert abs(st0["bias_rel_rmse"]) < 0.3 * true_bias, st0


def test_trace_kernel_names_follow_the_schedule():
    class FakePt:
        def __init__(self, sched):
            self.sched = sched

        def last_render_schedule(self, ctx):
            return self.sched

    assert bench.trace_kernels(FakePt("paths"), None, 8) == ("k_paths", 1)
    assert bench.trace_kernels(FakePt("wavefront"), None, 8) == ("k_trace", 8)


def test_traversal_roofline_counts_algorithmic_flops():
    """The traversal roofline divides the tests' algorithmic FLOPs (24 per
    node fetch of two child slabs, 20 per sphere, 10 per quad, 41 per
    triangle) by the kernel time and the measured FMA rate."""
    import bench
    work = {"nodes": 1000, "sphere": 100, "quad": 10, "triangle": 1}
    r = bench.traversal_roofline(work, 1e-3, "k_trace", 8, 50.0, 2070.0, "")
    flop = 24 * 1000 + 20 * 100 + 10 * 10 + 41 * 1
    assert abs(r["achieved"] - flop / 1e-6 / 1e12) < 1e-12
    assert abs(r["frac"] - r["achieved"] / 50.0) < 1e-15
    assert r["unit"] == "TFLOP/s" and r["bound"] == "alu" and r["kernel"] == "k_trace"
    ops = 58 * 1000 + 36 * 100 + 12 * 10 + 46
    assert abs(r["issue_frac"] - ops / 1e-6 / (152 * 128 * 2070e6)) < 1e-12


def test_trace_traffic_follows_the_captured_source(monkeypatch):
    """The traversal's DRAM traffic is reported only while the traversal
    source is the one the ncu capture was taken on."""
    import bench
    monkeypatch.setattr(bench, "TRACE_TRAFFIC",
                        {("C2", "decoded"): {"bytes_per_ray": 40.0, "src": bench.trace_source_hash()}})
    assert bench.trace_traffic("C2", "decoded", 1000) == 40000.0
    assert bench.trace_traffic("C2", "packed", 1000) is None
    assert bench.trace_traffic("C3", "decoded", 1000) is None
    monkeypatch.setattr(bench, "TRACE_TRAFFIC", {("C2", "decoded"): {"bytes_per_ray": 40.0, "src": "0" * 16}})
    assert bench.trace_traffic("C2", "decoded", 1000) is None


def test_recorded_traffic_matches_the_current_traversal_source():
    """Every recorded traversal-traffic figure carries the hash of the source it was captured on; a stale
    entry is reported as null by the bench, so this only checks the format."""
    import bench
    for (wl, form), rec in bench.TRACE_TRAFFIC.items():
        assert wl in ("C1", "C2", "C3", "C4", "C5") and form in bench.NODE_FORMS.values()
        assert rec["bytes_per_ray"] > 0 and len(rec["src"]) == 16


def test_shade_bytes_counts_the_queue_records():
    """Shading traffic per frame: 8 B per camera-ray hit, 56 B read and 48 B written per later ray (32 B more of
    radiance with emitters), 24 B per escape record."""
    import bench
    counts = [100, 50, 20, 5]   # rays at vertices 1..3, then escapes
    assert bench.shade_bytes(counts, 3, False) == 8 * 100 + 104 * 70 + 24 * 5
    assert bench.shade_bytes(counts, 3, True) == 8 * 100 + 136 * 70 + 24 * 5


def test_trace_l2_bytes_follow_the_captured_source(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "TRACE_L2", {("C4", "packed"): {"bytes_per_ray": 10.0, "src": bench.trace_source_hash()}})
    assert bench.trace_l2_bytes("C4", "packed", 100) == 1000.0
    assert bench.trace_l2_bytes("C4", "quant8", 100) is None
    monkeypatch.setattr(bench, "TRACE_L2", {("C4", "packed"): {"bytes_per_ray": 10.0, "src": "0" * 16}})
    assert bench.trace_l2_bytes("C4", "packed", 100) is None
