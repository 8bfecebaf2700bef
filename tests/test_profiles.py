"""The committed ncu counters behind the bench line's roofline.traffic: internally consistent, and
reported only while the kernel source is the one they were taken from."""
import hashlib
import json
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fused_counters_are_consistent():
    with open(os.path.join(ROOT, "profiles", "k_fused3_counters.json")) as fh:
        d = json.load(fh)
    assert d["kernel"] == "k_fused3" and os.path.exists(os.path.join(ROOT, d["source"]))
    full = d["full_launch"]
    assert full["passes"] == 1 and "--clock-control none" in full["command"]
    assert "--clock-control none" in d["command"]
    # the bench launch's bytes are the captured 128-instance bytes scaled by its share of instances
    share = full["site_updates"] / full["captured_site_updates"]
    assert 0.0 < share <= 1.0
    for k in ("dram_bytes_read", "dram_bytes_write"):
        assert abs(full[k] - share * full["captured_" + k]) <= 1e-6 * full["captured_" + k]
    per_su = (full["captured_dram_bytes_read"] + full["captured_dram_bytes_write"]) / full["captured_site_updates"]
    assert abs(per_su - full["dram_bytes_per_site_update"]) <= 1e-9
    # far below the 14 S = 448 B per site-update of a streaming complex64 march
    assert per_su < 1.0


def test_traffic_is_reported_only_for_the_captured_source(tmp_path, monkeypatch):
    import bench
    with open(os.path.join(ROOT, "profiles", "k_fused3_counters.json")) as fh:
        d = json.load(fh)
    src = os.path.join(ROOT, d["source"])
    with open(src, "rb") as fh:
        same = hashlib.sha256(fh.read()).hexdigest() == d["source_sha256"]
    expected = d["full_launch"]["dram_bytes_read"] + d["full_launch"]["dram_bytes_write"]
    got = bench.measured_traffic("k_fused3")
    assert (got == expected) if same else (got is None)
    # a copy of the tree whose kernel source differs by one byte reports no traffic
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", "k_fused3_counters.json"), tmp_path / "profiles")
    os.makedirs(tmp_path / os.path.dirname(d["source"]))
    with open(src, "rb") as fh:
        body = fh.read()
    with open(tmp_path / d["source"], "wb") as fh:
        fh.write(body + b"\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("k_fused3") is None
    assert bench.measured_traffic("no_such_kernel") is None
