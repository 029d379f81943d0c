"""The DRAM traffic that bench.py reports comes from profiles/traffic.json
only while the kernel sources are the ones the counters were taken from:
the table is keyed by a hash of csrc/, and any change to those sources makes
the bench report null instead of stale counters."""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reported_traffic_follows_the_hash():
    import bench
    table = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    current = table["csrc_hash"] == bench.csrc_hash()
    for k, v in table["kernels"].items():
        assert bench.traffic_for(k) == (v if current else None)
        # about one read of the 4096^2 uint16 image (33.5 MB) per launch
        assert 30e6 < v < 40e6, (k, v)


def test_changed_sources_give_null(tmp_path, monkeypatch):
    import bench
    fake = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "paper_1105_3829_gb300", "csrc"), fake / "paper_1105_3829_gb300" / "csrc")
    shutil.copytree(os.path.join(ROOT, "profiles"), fake / "profiles")
    monkeypatch.setattr(bench, "ROOT", str(fake))
    table = json.load(open(fake / "profiles" / "traffic.json"))
    table["csrc_hash"] = bench.csrc_hash()  # as if captured from these sources
    json.dump(table, open(fake / "profiles" / "traffic.json", "w"))
    key = next(iter(table["kernels"]))
    assert bench.traffic_for(key) is not None
    with open(fake / "paper_1105_3829_gb300" / "csrc" / "hist_tile.cuh", "a") as f:
        f.write("\n// edited\n")
    assert bench.traffic_for(key) is None
