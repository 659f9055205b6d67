"""Host-side logic of bench.py, without a GPU: the per-family source hashes
that keep a recorded ncu traffic figure tied to the kernel sources it was
taken on, and the CPU baseline's record."""
import json
import os

import numpy as np
import pytest

import bench
from paper_1412_3655_gb300 import synth


def test_every_recorded_kernel_has_a_family_and_a_profile():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    assert rec
    for key, entry in rec.items():
        assert any(key.startswith(k) for k in bench.KERNEL_SOURCES), key
        assert os.path.exists(os.path.join(bench.ROOT, entry["profile"])), entry["profile"]
        assert entry["dram_bytes_per_launch"] > 0


def test_traffic_is_null_for_unknown_kernels_and_changed_sources(tmp_path, monkeypatch):
    key = "halfsweep_su3_f64_18_tps1_b64_mb1"
    h = bench.source_hash(key)
    assert len(h) == 16
    # families share the base files but not the extra ones
    assert bench.source_hash("heatbath_x") != h and bench.source_hash("mag_halfsweep_x") != h
    fake = tmp_path / "profiles"
    fake.mkdir()
    (fake / "traffic.json").write_text(json.dumps({
        key: {"dram_bytes_per_launch": 123.0, "source_hash": h, "profile": "p"},
        "halfsweep_other": {"dram_bytes_per_launch": 5.0, "source_hash": "0" * 16, "profile": "p"}}))
    csrc = os.path.join(bench.ROOT, "paper_1412_3655_gb300", "csrc")
    os.symlink(os.path.dirname(csrc), tmp_path / "paper_1412_3655_gb300")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic(key) == 123.0
    assert bench.recorded_traffic("halfsweep_other") is None
    assert bench.recorded_traffic("halfsweep_missing") is None


def test_cpu_baseline_record(orc):
    dims = (4, 4, 4, 4)
    U = synth.gauge_config(dims, 3, 0.3, 1)
    r = bench.cpu_baseline(U, dims, 3, 1.7, budget_s=0.2)
    assert r["kind"] == "oracle" and r["unit"] == bench.UNIT
    assert r["value"] > 0 and r["cores"] >= 1 and "sweeps" in r["sample"]
    assert r["one_core"]["value"] > 0
    assert orc.get_threads() == r["cores"]


def test_background_inputs_come_back_by_name():
    """The other workloads' inputs are generated one after another in a
    background thread and handed out by name, whatever order they are asked
    for in."""
    order = []

    def job(name):
        def run():
            order.append(name)
            return name * 2
        return run

    bg = bench.Background([("a", job("a")), ("b", job("b")), ("c", job("c"))])
    assert bg.get("c") == "cc" and bg.get("a") == "aa" and bg.get("b") == "bb"
    bg.close()
    assert order == ["a", "b", "c"]
    assert 1 <= bench.gen_workers() <= 14


def test_gribov_copies_match_the_generator():
    """A copy of the batched Gribov workload is the generator's own copy."""
    dims = (4, 4, 4, 4)
    a = bench._gribov_copy((dims, 3))
    b = synth.gauge_config(dims, 3, 0.3, 4, copy=3)
    assert np.array_equal(a, b.view(np.float64).reshape(-1))
