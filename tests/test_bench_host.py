"""Host-side pieces of bench.py: the algorithmic operation counts behind the
roofline (the figures quoted for the 2048^2 box workload and the 16 x 512^2
Gaussian), the accuracy-job runner of the CPU-baseline leg, and the reference
arm's JSON line (a short run of the oracle on this machine's cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_operation_counts():
    import bench
    # sigma_r = 20: N = 66, 33 nonzero frequencies plus the constant term
    assert bench.box_instr_per_px(33, True) == 1900.0
    # sigma_r = 25: N = 43, 22 nonzero frequencies; Gaussian R = 12
    assert bench.gauss_instr_per_px(22, False, 12) == 22 * (9 + 4 * 50) + 4


def test_accuracy_jobs_run_with_the_oracle_module(oracle):
    import bench
    got = bench.oracle_accuracy([("a", lambda o: {"n": o.n_rule(20.0)}),
                                 ("b", lambda o: 1.5)])
    assert got == {"a": {"n": 66}, "b": 1.5}


def test_reference_arm_line():
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "4"))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "cpu_baseline", "e2e", "config"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    # ms_per_step is the timed step's own (sampled) time; the full step's is extrapolated
    assert 0 < line["px_per_step"] < 3 * 2048 * 2048
    assert 0 < line["ms_per_step"] <= line["ms_per_full_step_extrapolated"]


def test_traffic_is_tied_to_the_kernel_sources(monkeypatch):
    # the ncu DRAM figures are reported only for the build they were captured on
    import bench
    h = bench.kernel_sources_sha256()
    assert h == bench.kernel_sources_sha256() and len(h) == 64
    monkeypatch.setattr(bench, "DRAM_SOURCES_SHA256", h)
    b, note = bench.dram_traffic(32.0)
    assert b == bench.DRAM_BYTES_PER_CALL[32.0] and h[:12] in note
    monkeypatch.setattr(bench, "DRAM_SOURCES_SHA256", "0" * 64)
    b, note = bench.dram_traffic(32.0)
    assert b is None and "not reported" in note


def test_backward_operation_count_and_roofline_object():
    # the adjoint's count for the differentiable workload (Gaussian R = 12,
    # N = 43: 22 nonzero frequencies, no constant term) is ten planes through
    # 2(2R+1) taps plus generation and combine per frequency
    import bench
    assert bench.gauss_bwd_instr_per_px(22, False, 12) == 22 * (35 + 10 * 50)
    r = bench.alu_roofline(4.0e12, 100.0, 40.0e12, "x")
    assert r["bound"] == "alu" and abs(r["achieved"] - 40.0) < 1e-9 and abs(r["frac"] - 1.0) < 1e-12
