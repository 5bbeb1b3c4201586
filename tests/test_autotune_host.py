"""CPU: the autotuner's host-side helpers.  The Pareto front (Sec. IV-B:
the fastest setting at each recall level) against a brute-force
non-domination check, and tie-aware recall@k (Sec. I-A) against a direct
count, padding included."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _autotune():
    from paper_1509_06957_gb300 import autotune
    return autotune


def _dominated(p, pts):
    return any((q["recall"] >= p["recall"] and q["ms"] < p["ms"]) or
               (q["recall"] > p["recall"] and q["ms"] <= p["ms"]) for q in pts)


@pytest.mark.parametrize("seed", range(20))
def test_pareto_front_is_the_non_dominated_set(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    # coarse grids so that equal recalls and equal times occur
    pts = [{"recall": float(rng.integers(0, 12)) / 11, "ms": float(rng.integers(1, 9)), "i": i}
           for i in range(n)]
    front = _autotune().pareto(pts)
    recalls = [p["recall"] for p in front]
    assert recalls == sorted(set(recalls)), "one point per recall level, ascending"
    assert all(a["ms"] < b["ms"] for a, b in zip(front, front[1:])), "time rises with recall"
    assert not any(_dominated(p, pts) for p in front), "a front point is dominated"
    # every non-dominated recall level is on the front
    nd = {p["recall"] for p in pts if not _dominated(p, pts)}
    assert nd == set(recalls)


def test_recall_counts_ties_and_padding():
    at = _autotune()
    true = torch.tensor([[1.0, 2.0, 3.0], [0.5, 0.5, 0.5]])
    got = torch.tensor([[1.0, 3.0, float("inf")],   # padded slot counts nothing
                        [0.5, 0.5, 0.5000001]])     # tie at the k-th, within 1e-5
    assert at.recall(got, true) == pytest.approx(5 / 6)
    far = torch.tensor([[1.0, 2.0, 3.1], [0.5, 0.6, 0.7]])
    assert at.recall(far, true) == pytest.approx(3 / 6)
