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


def test_reduced_copy_emulation_and_distance_error():
    """The host emulation of the reduced copies: bfloat16 keeps integers
    0..255 exactly; e4m3 with the per-row scale max|x| / 448 is within
    2^-4 relative of each value (3 mantissa bits) and keeps each row's
    largest magnitude exactly; the distance error is zero for an exact copy
    and matches a hand computation otherwise."""
    import torch
    g = torch.Generator().manual_seed(0)
    Xi = torch.randint(0, 256, (50, 16), generator=g).float()
    assert torch.equal(bench.lowp_copy(Xi, 1, torch), Xi.double())
    X = torch.rand((50, 16), generator=g) * 3 - 1
    X8 = bench.lowp_copy(X, 2, torch)
    assert torch.all((X8 - X.double()).abs() <= X.double().abs() * 2.0 ** -4 + 1e-6)
    big = X.abs().argmax(1)
    rows = torch.arange(50)
    assert torch.allclose(X8[rows, big].abs(), X.double()[rows, big].abs(), rtol=1e-6)
    Q = torch.rand((3, 16), generator=g)
    ids = torch.tensor([[0, 1], [2, -1], [4, 5]], dtype=torch.int32)
    assert bench.lowp_distance_error(X, X.double(), Q, ids, torch) == (0.0, 0.0)
    emax, emean = bench.lowp_distance_error(X, X8, Q, ids, torch)
    want = []
    for i, row in enumerate(ids.tolist()):
        for j in row:
            if j < 0:
                continue
            d64 = ((X[j].double() - Q[i].double()) ** 2).sum()
            dl = ((X8[j] - Q[i].double()) ** 2).sum()
            want.append(float(abs(dl - d64) / d64))
    assert abs(emax - max(want)) < 1e-12 and abs(emean - sum(want) / len(want)) < 1e-12


def test_search_kernel_name_follows_the_dispatch_rule():
    """bench.py names the search kernel of its roofline by the library's
    dispatch rule; the rule's condition must still read as bench.py assumes."""
    src = open(SRC).read()
    assert "if (nchunk >= 8 && idx->dpad <= 1024) {" in src
    assert "const int nchunk = RK == 2 ? int(row_bytes / 16) - 1 : idx->dpad / vpc;" in src
    assert "idx->row8_bytes = ((idx->dpad + 15) & ~15) + 16;" in src
    cases = {(0, 784): "k_cand_knn_rows", (1, 784): "k_cand_knn_rows", (2, 784): "k_cand_knn_rows",
             (2, 113): "k_cand_knn_rows", (2, 112): "k_cand_knn", (2, 64): "k_cand_knn",
             (2, 1100): "k_cand_knn",
             (0, 1024): "k_cand_knn_rows", (0, 1025): "k_cand_knn", (1, 1100): "k_cand_knn",
             (0, 25): "k_cand_knn_rows", (0, 24): "k_cand_knn", (1, 64): "k_cand_knn_rows",
             (1, 56): "k_cand_knn"}
    for (prec, d), name in cases.items():
        assert bench.search_kernel_name(prec, d) == name, (prec, d)
        assert bench.kernel_source_sha(name, SRC)
