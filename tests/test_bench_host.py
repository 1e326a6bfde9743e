"""Host logic of bench.py that needs no GPU: the DRAM traffic of the Stage I
kernel is reported only while the kernel's sources are those the committed
ncu counters were taken on, and the roofline arithmetic uses the measured
peaks."""
import json
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _copy_tree(tmp):
    d = json.load(open(os.path.join(ROOT, "profiles", "k_rollout_traffic.json")))
    os.makedirs(os.path.join(tmp, "profiles"))
    shutil.copy(os.path.join(ROOT, "profiles", "k_rollout_traffic.json"), os.path.join(tmp, "profiles"))
    for f in d["source_files"]:
        os.makedirs(os.path.dirname(os.path.join(tmp, f)), exist_ok=True)
        shutil.copy(os.path.join(ROOT, f), os.path.join(tmp, f))
    return d


def test_traffic_is_reported_for_the_captured_sources(tmp_path, monkeypatch):
    d = _copy_tree(str(tmp_path))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    for wl, rec in d["workloads"].items():
        assert bench.rollout_traffic(wl) == rec["bytes_per_launch"]
        assert rec["bytes_per_launch"] == rec["read"] + rec["write"]
    assert bench.rollout_traffic("no such workload") is None


def test_traffic_is_null_once_a_kernel_source_changes(tmp_path, monkeypatch):
    d = _copy_tree(str(tmp_path))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    with open(os.path.join(str(tmp_path), d["source_files"][0]), "a") as f:
        f.write("\n// edited\n")
    for wl in d["workloads"]:
        assert bench.rollout_traffic(wl) is None


def test_traffic_is_null_without_a_record(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.rollout_traffic("ensemble") is None


def test_fp32_peak_is_the_unit_count_times_the_clock():
    assert bench.fp32_peak_tflops(2070.0, 152) == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert bench.fp32_peak_tflops(1000.0, 10) == pytest.approx(10 * 128 * 2 * 1e9 / 1e12)


def _smi(sm, util, reasons=("Not Active",) * 4, mx=2070, power=500.0):
    return ", ".join(["0", str(sm), str(mx), str(power), str(util), "0x0", *reasons])


def test_clock_summary_takes_the_median_under_load_and_every_reason():
    lines = [_smi(2070, 0), _smi(1900, 95), _smi(1800, 99), _smi(1700, 97),
             _smi(2070, 80, ("Not Active", "Not Active", "Not Active", "Active")),
             "garbage line", ""]
    c = bench.clock_summary(lines)
    assert c["samples"] == 5 and c["samples_under_load"] == 4
    assert c["sm_mhz"] == pytest.approx((1800 + 1900) / 2)
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_clock_summary_without_load_uses_every_sample():
    c = bench.clock_summary([_smi(2070, 0), _smi(2000, 10)])
    assert c["samples_under_load"] == 0 and c["sm_mhz"] == pytest.approx(2035.0)
    assert bench.clock_summary([])["sm_mhz"] is None


def test_flop_count_is_the_sum_of_its_terms():
    assert bench.rollout_flops_per_step() == 16 + 12 + 226 + 13 + 69 + 1 + 8
    P = dict(E=2, K=3, T=5, iters=2)
    assert bench.rollout_steps(P) == 2 * 3 * 5 * 2 + 2 * 5
