"""The benchmark's roofline bookkeeping (host logic, CPU): the top timed kernel with a known
cost is reported against the peak of the arithmetic it runs, the double-float peak follows
from the FP32 issue rate and the 15 instructions of one multiply-add, and per-launch DRAM
traffic is reported only while the kernel's source is the one it was measured on."""

import json
import os

import pytest

import bench
from paper_2010_08581_gb300 import inputs

WL = inputs.WORKLOADS["tr3_500_r10_fp32"]


def test_double_float_factorisation_is_measured_against_the_double_float_peak():
    prof = {"cholesky_leverage": [10.0, 100], "solve_rhs": [5.0, 100]}
    r = bench.roofline(prof, WL, None)
    assert r["kernel"] == "cholesky_leverage" and r["bound"] == "alu"
    per_sm = 128 * 2.07e9 * 2 / 15 / 1e12
    assert r["peak"] == pytest.approx(152 * per_sm, rel=1e-3)
    achieved = (100 ** 3 / 3.0) / (10.0 / 1e3 / 100) / 1e12      # L = 100, 100 us a launch
    assert r["achieved"] == pytest.approx(achieved, rel=1e-3)
    assert r["frac_of_one_sm"] == pytest.approx(achieved / per_sm, rel=1e-3)
    assert r["frac_of_one_sm_fp64"] == pytest.approx(achieved / (1.25 / 152), rel=1e-3)


def test_kernels_without_a_cost_are_skipped_and_kinds_map_to_bounds():
    prof = {"unknown_kernel": [50.0, 1], "gather": [2.0, 100]}
    r = bench.roofline(prof, WL, {"hbm_gbs": 7000.0})
    assert r["kernel"] == "gather" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["peak"] == 7000.0
    r = bench.roofline({"normal_eq_tc": [3.0, 100]}, WL, {"bf16_tflops": 2000.0})
    assert r["bound"] == "tensor" and r["peak"] == pytest.approx(1000.0)
    r = bench.roofline({"cholesky_solve": [4.0, 100]}, WL, None)
    assert r["bound"] == "alu" and "frac_of_one_sm" in r


def test_traffic_is_reported_only_for_the_measured_source(tmp_path, monkeypatch):
    table = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for kernel, entry in table.items():
        assert bench.traffic_for(kernel) in (entry["bytes_per_launch"], None)
        assert bench.algorithmic_cost(kernel, WL) is not None
    fake = tmp_path / "repo"
    (fake / "profiles").mkdir(parents=True)
    (fake / "paper_2010_08581_gb300" / "csrc").mkdir(parents=True)
    src = fake / "paper_2010_08581_gb300" / "csrc" / "k.cuh"
    src.write_text("kernel v1")
    import hashlib
    sha = hashlib.sha256(b"kernel v1").hexdigest()[:16]
    (fake / "profiles" / "traffic.json").write_text(json.dumps(
        {"k": {"source": "k.cuh", "source_sha": sha, "bytes_per_launch": 1234}}))
    monkeypatch.setattr(bench, "ROOT", str(fake))
    assert bench.traffic_for("k") == 1234
    src.write_text("kernel v2")
    assert bench.traffic_for("k") is None
    assert bench.traffic_for("absent") is None


def test_alu_peaks_follow_the_sm_count_and_the_measured_clock():
    sms, ghz = bench.alu_basis({"sm_max_mhz": 1000.0})
    assert ghz == pytest.approx(1.0)
    r = bench.roofline({"cholesky_solve": [4.0, 100]}, WL, {"sm_max_mhz": 1000.0})
    assert r["peak"] == pytest.approx(sms * 128 * 2 * 1.0e9 / 1e12, rel=1e-3)
    assert f"{sms} SMs" in r["peak_source"]
    assert bench.alu_basis(None)[1] == pytest.approx(2.07)
