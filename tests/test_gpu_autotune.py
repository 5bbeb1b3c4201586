"""GPU: the autotuner reaches its recall target with the fastest setting it
measured, its recall agrees with an independent brute force, results are
cached, and the kernel-knob sweep returns a valid setting."""
import json

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_06957_gb300 as m
    m.load_library()
    return m


def test_tune_to_target(mr, tmp_path):
    from paper_1509_06957_gb300 import autotune
    X, Q = workloads.mnist_like(6000, 200, seed=11)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    idx = mr.mrpt_build(Xd, 32, 6, 0.0, 1)
    mr.mrpt_add_lowp(idx, mr.MRPT_PREC_BF16)
    cache = str(tmp_path / "tune.json")
    res = autotune.tune(idx, Xd, Qd, 10, target=0.9, v_grid=(1, 2, 4, 8), reps=2,
                        precisions=((0, 0), (1, 0)), cache_path=cache)
    assert res["reached"]
    best = res["best"]
    assert best["recall"] >= 0.9
    assert all(r["ms"] >= best["ms"] for r in res["table"] if r["recall"] >= 0.9)
    # the recall it measured, recomputed against the oracle's brute force
    ids, d = mr.mrpt_query_ex(idx, Qd, 10, best["v"], n_trees=best["n_trees"],
                              precision=best["precision"], margin=best["margin"])
    bi, bd = oracle.brute_knn(X, Q, 10)
    d = d.cpu().numpy()
    ok = (d <= bd[:, -1:] * (1 + 1e-5)) & np.isfinite(d)
    assert abs(ok.mean() - best["recall"]) < 0.02
    # pareto front is monotone
    fr = res["pareto"]
    assert all(a["recall"] < b["recall"] and a["ms"] <= b["ms"] + 1e9 for a, b in zip(fr, fr[1:]))
    # cached
    again = autotune.tune(idx, Xd, Qd, 10, target=0.9, cache_path=cache)
    assert again["best"] == json.load(open(cache))[next(iter(json.load(open(cache))))]["best"]
    kn = autotune.tune_kernels(idx, Qd, 10, best["v"], best["n_trees"], best["precision"],
                               best["margin"], reps=2)
    assert kn["best"]["ms"] == min(r["ms"] for r in kn["table"])
    idx.close()
