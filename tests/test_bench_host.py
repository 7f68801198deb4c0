"""Host logic of bench.py that decides what the JSON line claims (no GPU).

* The roofline's `traffic` comes from profiles/traffic.json only while the sources
  the capture was taken from are unchanged and the workload matches; any edit of
  those sources, or another n, gives null.
* The nominal flop count is the stated convention (4n^3/3 + 2n^3).
"""
import json
import shutil

import bench


def test_committed_traffic_matches_current_sources():
    ent = json.loads((bench.ROOT / "profiles" / "traffic.json").read_text())["kernels"]
    for cat, e in ent.items():
        assert bench.committed_traffic(cat, e["n"]) == e["dram_bytes_per_launch"]
        assert bench.committed_traffic(cat, e["n"] + 1) is None
    assert bench.committed_traffic("no such kernel", 49152) is None


def test_committed_traffic_is_null_after_a_source_change(tmp_path, monkeypatch):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    shutil.copy(bench.ROOT / "profiles" / "traffic.json", root / "profiles" / "traffic.json")
    ent = json.loads((root / "profiles" / "traffic.json").read_text())["kernels"]
    cat, e = next(iter(ent.items()))
    for f in e["sources"]:
        (root / f).parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(bench.ROOT / f, root / f)
    monkeypatch.setattr(bench, "ROOT", root)
    assert bench.committed_traffic(cat, e["n"]) == e["dram_bytes_per_launch"]
    src = root / e["sources"][0]
    src.write_bytes(src.read_bytes() + b"\n// edited\n")
    assert bench.committed_traffic(cat, e["n"]) is None


def test_nominal_flops_convention():
    n = 49152
    assert bench.nominal_flops(n) == 4.0 * n ** 3 / 3.0 + 2.0 * n ** 3
    assert abs(bench.nominal_flops(n) - 3.958e14) / 3.958e14 < 1e-3
