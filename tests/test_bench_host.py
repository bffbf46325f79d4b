"""Host-side logic of bench.py that needs no GPU: the DRAM-traffic record is used only
while the apply kernel's sources still hash to the captured version, the whole-job value
divides by every solve of every rank, and the peak falls back when the measured file is
absent."""
import os

import pytest

import bench


def test_traffic_record_scales_and_goes_null_on_a_source_change(monkeypatch):
    t, why = bench.apply_traffic(712_000_000)
    if t is None:
        # a kernel source changed since the capture: the record must say so, not a number
        assert "changed" in why or "unavailable" in why
    else:
        ratio = t / 712_000_000
        assert 1.0 <= ratio < 1.5, ratio
        assert "scaled" in why
    # any other source list hashes differently: the bench then reports no traffic
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES", ("apply.cuh",))
    t2, why2 = bench.apply_traffic(712_000_000)
    assert t2 is None and "changed" in why2


def test_whole_job_value_counts_every_solve_of_every_rank():
    assert bench.whole_job_ms_per_solve(600.0, 10, 1) == pytest.approx(60.0)
    assert bench.whole_job_ms_per_solve(600.0, 10, 4) == pytest.approx(15.0)
    assert bench.replica_seed(3) == 3 and bench.max_over_ranks(2.5, 1) == 2.5


def test_peak_falls_back_without_the_measured_file(monkeypatch):
    real = bench.ROOT
    if os.path.exists(os.path.join(real, "MEASURED_PEAKS.json")):
        peak, kind = bench.read_peaks()
        assert kind == "measured" and peak > 1000.0
    monkeypatch.setattr(bench, "ROOT", os.path.join(real, "no_such_directory"))
    peak, kind = bench.read_peaks()
    assert kind == "fallback" and peak == bench.FALLBACK_HBM_GBS


def test_learned_vs_plain_ratios():
    out = {"box_1157k": {"vn": {"iters_mean": 150.0, "ms_mean": 50.0},
                         "vn_walls": {"iters_mean": 140.0, "ms_mean": 48.0},
                         "learned": {"iters_mean": 120.0, "ms_mean": 45.0}},
           "ensemble_64": {"vn": {"iters_sum": 5000, "ms": 300.0},
                           "learned_highpass": {"iters_sum": 4500, "ms": 290.0}}}
    r = bench.learned_vs_plain(out)
    assert r["box_1157k"]["learned/vn"]["iters"] == pytest.approx(0.8)
    assert r["box_1157k"]["learned/vn_walls"]["ms"] == pytest.approx(45.0 / 48.0)
    assert r["ensemble_64"]["learned_highpass/vn"]["iters"] == pytest.approx(0.9)
    assert "learned_highpass/vn_walls" not in r["ensemble_64"]


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on the host (one full solve of a
    tiny box here) and prints one JSON line with the same metric, the reference marker,
    steps = 1 with the requested count beside it, the workload config of the GPU arm, its
    CPU baseline and an end-to-end object with no host-device traffic."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "20", "--warmup", "5",
                          "--box-side", "12"], cwd=root, capture_output=True, text=True, timeout=600,
                         check=True)
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is False and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["steps_requested"] == 20 and d["warmup_requested"] == 5
    assert d["value"] > 0 and d["ms_per_step"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == dict(value=d["value"], unit=d["unit"], h2d_bytes_per_step=0, d2h_bytes_per_step=0)
    assert d["config"] == bench.workload_config(12, bench._box_count(12))
    assert d["true_rel_res"] <= 1e-6 and len(d["iterations"]) == 3
