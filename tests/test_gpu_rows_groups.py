"""GPU: the candidate search on short rows, where groups of 8 or 16 lanes each
take one row (two slabs of 4 or 2 rows per step), against the oracle.

Rows of 8 to 16 16-byte chunks: float32 of 32 to 64 values, bfloat16 of 64
to 128, e4m3 of 113 to 256.  The cases put several thousand candidates per
query in lists split into several work items (of 37 candidates for k = 10,
so every item ends in a partial step), with k = 10 and k = 100:

* float32 and lossless bfloat16 (integer data): the oracle's rows, distances
  within 1e-5 and ids equal up to ties;
* lossy bfloat16 and e4m3 with the float32 re-rank: ids in S, exact float32
  distances, ascending rows, and recall no more than 0.02 below a float64
  emulation of the same screen.
|S| is compared with the oracle for every query."""
import numpy as np
import pytest

import oracle
import workloads
from _parity import check_lowp_results, check_results, emulated_recall, oracle_sets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_06957_gb300 as m
    m.load_library()
    return m


CASES = [
    # (data, d, precision, margin, lanes per row)
    ("gauss", 32, 0, 0, 8),
    ("gauss", 60, 0, 0, 16),
    ("int", 64, 1, 0, 8),
    ("int", 120, 1, 0, 16),
    ("gauss", 100, 1, 16, 16),
    ("latent", 128, 2, 24, 8),
    ("latent", 250, 2, 24, 16),
]


@pytest.mark.parametrize("k", [10, 100])
@pytest.mark.parametrize("data,d,prec,margin,g", CASES,
                         ids=[f"{c[0]}-d{c[1]}-p{c[2]}-g{c[4]}" for c in CASES])
def test_short_rows_in_lane_groups(mr, data, d, prec, margin, g, k):
    n, m = 6000, 40
    if data == "gauss":
        X, Q = workloads.gaussian_mixture(n, d, m, n_centres=30, seed=d)
    elif data == "int":
        X, Q = workloads.lognormal_int(n, d, m, seed=d)
    else:
        X, Q = workloads.latent_factor(n, d, m, seed=d)
    T, l, v = 24, 4, 2
    dens = float(np.float32(d ** -0.5))
    idx = mr.mrpt_build(torch.from_numpy(X).cuda(), T, l, dens, 3)
    if prec:
        mr.mrpt_add_lowp(idx, prec)
    ncand = torch.empty(m, dtype=torch.int64, device="cuda")
    # k = 10: items of 37 candidates, so every item ends in a partial step
    ids, dd = mr.mrpt_query_ex(idx, torch.from_numpy(Q).cuda(), k, v, precision=prec, margin=margin,
                               chunk=37 if k == 10 else 0, n_cand_out=ncand)
    torch.cuda.synchronize()
    ref = oracle.grow_trees(X, T, l, dens, 3)
    oi, od, _, oleaf, oncand = oracle.query(ref, Q, k, v, want_internals=True)
    assert np.array_equal(ncand.cpu().numpy(), oncand)
    assert oncand.min() > 1000
    sets = oracle_sets(ref, oleaf, v)
    gi, gd = ids.cpu().numpy(), dd.cpu().numpy()
    lossless = prec == 0 or (prec == 1 and data == "int")
    if lossless:
        check_results(X, Q, gi, gd, oi, od, sets)
    else:
        floor = emulated_recall(X, Q, sets, oi, od, k, margin, prec) - 0.02
        check_lowp_results(X, Q, gi, gd, oi, od, sets, floor)
    idx.close()
