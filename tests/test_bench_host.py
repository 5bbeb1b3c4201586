"""CPU: bench.py's DRAM-traffic bookkeeping.  A kernel's committed ncu
traffic figure is reported only while the kernel's source is the one it was
measured on; any edit to that kernel makes it null, edits elsewhere do not."""
import json
import os
import shutil

import pytest

pytest.importorskip("torch")
import bench  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1509_06957_gb300", "csrc", "mrpt_query.cu")


def _recorded():
    return json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))


def test_traffic_follows_the_kernel_source(tmp_path):
    rec = _recorded()
    current = {k: e for k, e in rec.items() if e["source_sha"] == bench.kernel_source_sha(k, SRC)}
    assert current, "no kernel's traffic matches its current source"
    name = next(iter(current))
    assert bench.load_traffic(name, SRC) == current[name]["dram_bytes_per_launch"]

    text = open(SRC).read()
    lines = text.split("\n")
    start = next(i for i, ln in enumerate(lines)
                 if "__global__" in ln and (name + "(") in " ".join(lines[i:i + 2]))
    # an edit inside the kernel's body: its traffic is stale
    edited = tmp_path / "edited.cu"
    edited.write_text("\n".join(lines[:start + 2] + ["    // edited"] + lines[start + 2:]))
    assert bench.kernel_source_sha(name, str(edited)) != current[name]["source_sha"]
    assert bench.load_traffic(name, str(edited)) is None
    # an edit outside every kernel: unchanged
    other = tmp_path / "other.cu"
    shutil.copy(SRC, other)
    with open(other, "a") as f:
        f.write("\n// trailing comment\n")
    assert bench.load_traffic(name, str(other)) == current[name]["dram_bytes_per_launch"]


def test_unknown_kernel_has_no_traffic():
    assert bench.load_traffic("k_not_a_kernel", SRC) is None
