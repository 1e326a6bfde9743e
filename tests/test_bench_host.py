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
    assert bench.fp32_peak_tflops(2070.0) == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
