"""Host logic of bench.py that decides what the JSON line claims (no GPU).

* The roofline's `traffic` comes from profiles/traffic.json only while the sources
  the capture was taken from are unchanged and the workload matches (bytes per launch
  for one n, or bytes per tile scaled by the tiles of a launch); any edit of those
  sources, or another n for a per-launch entry, gives null.
* The nominal flop count is the stated convention (4n^3/3 + 2n^3).
"""
import hashlib
import json
import shutil

import bench


def _sources_hash(root, files):
    h = hashlib.sha256()
    for f in files:
        h.update(f.encode())
        h.update((root / f).read_bytes())
    return h.hexdigest()[:16]


def test_committed_traffic_follows_the_sources_hash():
    ent = json.loads((bench.ROOT / "profiles" / "traffic.json").read_text())["kernels"]
    for cat, e in ent.items():
        unchanged = _sources_hash(bench.ROOT, e["sources"]) == e["src_hash"]
        if "dram_bytes_per_tile" in e:
            # per-tile entries hold at any n, scaled by the tiles of one launch
            got = bench.committed_traffic(cat, 49152, tiles_per_launch=1000.0)
            assert got == (e["dram_bytes_per_tile"] * 1000.0 if unchanged else None)
            assert bench.committed_traffic(cat, 49152) is None  # no tile count, no figure
        else:
            got = bench.committed_traffic(cat, e["n"])
            assert got == (e["dram_bytes_per_launch"] if unchanged else None)
            assert bench.committed_traffic(cat, e["n"] + 1) is None
    assert bench.committed_traffic("no such kernel", 49152) is None


def test_committed_traffic_is_null_after_a_source_change(tmp_path, monkeypatch):
    # a consistent entry over copies of the kernel's sources, then one edit
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    srcs = ["paper_2511_16174_gb300/csrc/evd_bcback.cu", "paper_2511_16174_gb300/csrc/tc_common.cuh"]
    for f in srcs:
        (root / f).parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(bench.ROOT / f, root / f)
    entry = {"n": 4096, "dram_bytes_per_launch": 1.5e8, "sources": srcs, "src_hash": _sources_hash(root, srcs)}
    (root / "profiles" / "traffic.json").write_text(json.dumps({"kernels": {"k/tc_split": entry}}))
    monkeypatch.setattr(bench, "ROOT", root)
    assert bench.committed_traffic("k/tc_split", 4096) == 1.5e8
    src = root / srcs[0]
    src.write_bytes(src.read_bytes() + b"\n// edited\n")
    assert bench.committed_traffic("k/tc_split", 4096) is None


def test_nominal_flops_convention():
    n = 49152
    assert bench.nominal_flops(n) == 4.0 * n ** 3 / 3.0 + 2.0 * n ** 3
    assert abs(bench.nominal_flops(n) - 3.958e14) / 3.958e14 < 1e-3
