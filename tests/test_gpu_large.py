"""GPU parity at the full sizes of the 1M-point workloads (sampled).

Trees are prefix-stable (draws are keyed by tree), so the oracle grows only
the first 4 trees of the full index and the library's queries restricted to
those trees (n_trees = 4) are compared through every internal.  The
full-T queries are checked against what must hold at any size: returned
distances are the exact distances of the returned ids, both query paths
agree, and recall against brute force on a query sample.
"""
import time

import numpy as np
import pytest

import oracle
import workloads
from _parity import REL_TOL, check_results, oracle_sets

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def mr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_06957_gb300 as m
    m.load_library()
    return m


def _prefix_parity(mr, idx, X, Q, T_chk, l, density, seed, k, v, precision=0):
    ref = oracle.grow_trees(X, T_chk, l, density, seed)
    split = mr.mrpt_export(idx, "SPLIT")[:T_chk]
    leaf_ids = mr.mrpt_export(idx, "LEAF_IDS")[:T_chk]
    assert np.array_equal(split.view(np.uint32), ref.split.view(np.uint32)), "split values"
    assert np.array_equal(leaf_ids, ref.leaf_ids), "leaves"
    Qd = torch.from_numpy(Q).cuda()
    ids, d, dbg = mr.mrpt_query_ex(idx, Qd, k, v, n_trees=T_chk, debug=True, precision=precision)
    torch.cuda.synchronize()
    oi, od, oproj, oleaf, oncand = oracle.query(ref, Q, k, v, want_internals=True)
    assert np.array_equal(dbg["proj"].cpu().numpy().view(np.uint32), oproj.view(np.uint32))
    assert np.array_equal(dbg["leaf"].cpu().numpy(), oleaf)
    assert np.array_equal(dbg["n_cand"].cpu().numpy(), oncand)
    sets = oracle_sets(ref, oleaf, v)
    votes = dbg["votes"].cpu().numpy()
    cand = dbg["cand"].cpu().numpy()
    for i in range(len(Q)):
        F, _ = oracle.votes(ref, oleaf[i], v)
        assert np.array_equal(votes[i], F.astype(np.uint8)), f"votes of query {i}"
        assert set(cand[i][: oncand[i]].tolist()) == sets[i], f"S of query {i}"
    check_results(X, Q, ids.cpu().numpy(), d.cpu().numpy(), oi, od, sets)


def _full_checks(mr, idx, X, Q, k, v, precision=0, margin=0):
    Qd = torch.from_numpy(Q).cuda()
    i0, d0 = mr.mrpt_query_ex(idx, Qd, k, v, precision=precision, margin=margin)
    i1, d1 = mr.mrpt_query_ex(idx, Qd, k, v, path=1)
    i0, d0, i1, d1 = (t.cpu().numpy() for t in (i0, d0, i1, d1))
    fin = np.isfinite(d0)
    for i in range(len(Q)):
        got = i0[i][fin[i]]
        ex = np.sqrt(((X[got].astype(np.float64) - Q[i].astype(np.float64)) ** 2).sum(1))
        np.testing.assert_allclose(d0[i][fin[i]], ex, rtol=REL_TOL)
    if precision == 0:
        np.testing.assert_allclose(d0[fin], d1[fin], rtol=REL_TOL)
    bi, bd = oracle.brute_knn(X, Q, k)
    hits = sum(len(set(a[a >= 0].tolist()) & set(b.tolist())) for a, b in zip(i0, bi))
    return hits / bi.size


def test_sift_like_1m_d128_k100(mr):
    """n = 1,000,000, d = 128, integer values 0..255 (heavy-tailed), k = 100,
    T = 100, l = 12: full-size build, chunked vote counters (16 id chunks),
    bfloat16 distances (lossless for these values)."""
    X, Q = workloads.lognormal_int(1_000_000, 128, 24, seed=3)
    dens = float(np.float32(128 ** -0.5))
    t0 = time.perf_counter()
    idx = mr.mrpt_build(torch.from_numpy(X).cuda(), 100, 12, dens, 0)
    print(f"build T=100 l=12 n=1M d=128: {time.perf_counter() - t0:.2f} s")
    mr.mrpt_add_lowp(idx)
    _prefix_parity(mr, idx, X, Q, 4, 12, dens, 0, k=100, v=1)
    _prefix_parity(mr, idx, X, Q[:8], 4, 12, dens, 0, k=100, v=1, precision=1)
    r = _full_checks(mr, idx, X, Q, 100, 2, precision=1, margin=32)
    print(f"recall@100 (T=100, v=2, bf16): {r:.3f}")
    idx.close()


def test_gist_like_1m_d960(mr):
    """n = 1,000,000, d = 960, values in [0, 1] from rank-64 factors, T = 200,
    l = 10, k = 10: full-size build of 200 trees, lossy bfloat16 with the
    float32 re-rank."""
    X, Q = workloads.latent_factor(1_000_000, 960, 16, seed=4)
    dens = float(np.float32(960 ** -0.5))
    t0 = time.perf_counter()
    idx = mr.mrpt_build(torch.from_numpy(X).cuda(), 200, 10, dens, 0)
    print(f"build T=200 l=10 n=1M d=960: {time.perf_counter() - t0:.2f} s")
    mr.mrpt_add_lowp(idx)
    _prefix_parity(mr, idx, X, Q, 4, 10, dens, 0, k=10, v=2)
    r = _full_checks(mr, idx, X, Q, 10, 3, precision=1, margin=32)
    print(f"recall@10 (T=200, v=3, bf16 + re-rank): {r:.3f}")
    idx.close()
