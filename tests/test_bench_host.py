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


def test_headline_fits_and_drops_optional_keys_in_order(capsys):
    """The result is read from the last stdout line, so the headline stays
    under HEADLINE_MAX_BYTES: the (T, v) sweep is not part of it, and the
    optional keys go first if a line would still be too long."""
    out = {"metric": "m", "value": 1.0, "unit": "queries/s", "config": {"workload": "w",
           "fp32_best": {"T": 1}, "knobs": {"chunk": 32}}, "stage_ms": {"vote": 0.1},
           "cpu_baseline": {"value": 1.0, "single_thread": {"value": 0.5}}, "pad": "x" * 100}
    line = bench.emit_line(dict(out), limit=4096)
    assert json.loads(line) == out
    small = bench.emit_line(json.loads(json.dumps(out)), limit=190)
    got = json.loads(small)
    assert "stage_ms" not in got and "fp32_best" not in got["config"]
    assert got["value"] == 1.0 and got["metric"] == "m"
    printed = capsys.readouterr().out.strip().splitlines()
    assert printed[-1] == small


@pytest.mark.slow
def test_reference_arm_last_line_parses():
    """`bench.py --impl reference` (the oracle on the benchmark workload, a
    small time budget here) ends stdout with one parseable JSON line under
    the size limit, carrying the keys the result is read from."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                        "--warmup", "3", "--ref-budget-s", "2"], cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    last = r.stdout.strip().splitlines()[-1]
    assert len(last.encode()) <= bench.HEADLINE_MAX_BYTES
    out = json.loads(last)
    assert out["impl"] == "reference" and out["value"] > 0 and out["unit"] == "queries/s"
    assert out["steps"] == 2 and out["warmup"] == 3
    assert out["config"]["workload"] == bench.WORKLOAD["name"]
    for key in ("cpu_baseline", "e2e", "metric", "higher_is_better", "ms_per_step"):
        assert key in out
