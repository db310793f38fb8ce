"""Host logic of bench.py that needs no GPU: the device-code hash that keys
the recorded DRAM counters (comment edits keep it, code edits change it),
the lookup that reports null for stale or missing counters, the per-launch
cost model's scaling, the whole-job rate over ranks, and the reference
arm's JSON line (the FP64 oracle on the host cores)."""
import os
import shutil

import pytest

import bench


def _tree(tmp_path, kernel_src):
    d = tmp_path / "paper_2606_06247_gb300" / "csrc"
    d.mkdir(parents=True)
    (d / "k.cu").write_text(kernel_src)
    (d / "api.cpp").write_text("int host_only = 1;\n")
    return str(tmp_path)


def test_source_hash_ignores_comments_and_host_code(tmp_path, monkeypatch):
    a = _tree(tmp_path / "a", "// header\n__global__ void k(float* x) { x[0] = 1.f; /* set */ }\n")
    b = _tree(tmp_path / "b", "/* other\n words */ __global__ void k(float* x) {\n  x[0] = 1.f;  // set\n}\n")
    c = _tree(tmp_path / "c", "__global__ void k(float* x) { x[0] = 2.f; }\n")
    hashes = []
    for root in (a, b, c):
        monkeypatch.setattr(bench, "ROOT", root)
        hashes.append(bench.kernel_sources_sha256())
    assert hashes[0] == hashes[1] != hashes[2]
    # host sources are not part of the key
    (tmp_path / "a" / "paper_2606_06247_gb300" / "csrc" / "api.cpp").write_text("int host_only = 2;\n")
    monkeypatch.setattr(bench, "ROOT", a)
    assert bench.kernel_sources_sha256() == hashes[0]


def test_recorded_traffic_is_reported_only_for_matching_code(monkeypatch):
    key = next(iter(bench.MEASURED_TRAFFIC))
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda: bench.KERNEL_SOURCES_SHA256)
    v, note = bench.measured_traffic(*key)
    assert v == bench.MEASURED_TRAFFIC[key] and "ncu" in note
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda: "0" * 64)
    v, note = bench.measured_traffic(*key)
    assert v is None and "changed" in note
    v, note = bench.measured_traffic("f32x2", "col_mom", 7)
    assert v is None


def test_cost_model_scales_with_the_batch():
    N, C = 256, 25
    hy = (N + C) // 2 + 1
    for kind in bench.PROF_KINDS:
        by1 = bench.kernel_bytes(kind, N, N, hy, 16, 1)
        fl1 = bench.kernel_flops(kind, N, N, N + C, N + C, hy, 2 * (N - 1), 1, False)
        assert bench.kernel_bytes(kind, N, N, hy, 16, 32) == 32 * by1
        assert bench.kernel_flops(kind, N, N, N + C, N + C, hy, 2 * (N - 1), 32, False) == pytest.approx(32 * fl1)
    # FP32 spectra are half the FP32-pair size; FP64 fields are not
    assert bench.kernel_bytes("row_mom", N, N, hy, 8, 1) * 2 == bench.kernel_bytes("row_mom", N, N, hy, 16, 1)


def test_job_rate_counts_every_rank():
    assert bench.job_rate(1000, 4, 2.0) == pytest.approx(4 * 1000 / 2e-3)


def test_hardware_peaks_and_plane_pass_bytes():
    import bench
    assert abs(bench.fp32_peak_tflops(2070.0) - 80.55) < 0.01     # 152 x 128 x 2 x 2.07 GHz
    assert abs(bench.fp64_peak_tflops(2070.0) - 1.2586) < 1e-3    # 152 x 2 x 2 x 2.07 GHz
    assert bench.fp32_lane_inst_rate(2070.0) * 2 / 1e12 == bench.fp32_peak_tflops(2070.0)
    P, n, hy = 256, 1024, 526
    passes = {k: bench.plane_kernel_bytes(k, P, n, n, hy) for k in ("col_fwd", "row_op", "col_out")}
    # every pass moves at least the call's own input or output; together they move
    # more than the call's 16 B per node (the spectra round-trip HBM between passes)
    assert passes["col_fwd"] > P * n * n * 4 and passes["col_out"] > P * n * n * 12
    assert sum(passes.values()) > P * n * n * 16
    assert bench.STEP_BYTES_PER_UPDATE == {"f32": 72, "f32x2": 72, "f64": 112}


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on the host cores
    (one bounded RK3 step here) and prints one JSON line with the keys the
    reference arm carries: the same metric and workload as the GPU arm, a
    cpu_baseline of kind oracle, and an e2e block with no host-device bytes."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("particle-updates/s per ISPH step")
    assert d["unit"] == "particle-updates/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["config"]["batch"] == 32 and d["config"]["nx"] == 256 and d["config"]["ny"] == 256
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
