"""Pins for the oracle: each check compares it with something other than
itself -- published generator outputs, a hand-worked example, exact rational
arithmetic, brute force, closed forms and the structural facts the paper
states (Sec. II-III).  CPU only."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads


# ----------------------------------------------------------------- RNG ----

def test_splitmix64_published_outputs(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "splitmix64.json")))
    for vec in g["vectors"]:
        outs = vec.get("outputs") or [int(h, 16) for h in vec["outputs_hex"]]
        for i, want in enumerate(outs):
            assert oracle.splitmix64(vec["seed"], i) == want


def test_random_matrix_statistics():
    """Sec. II-B: components are N(0,1) with probability a, else 0."""
    T, l, d = 40, 8, 784
    a = 1.0 / math.sqrt(d)
    R = oracle.random_matrix(T, l, d, a, seed=7)
    trials = T * l * d
    nnz = len(R.val)
    sd = math.sqrt(trials * a * (1 - a))
    assert abs(nnz - trials * a) < 5 * sd
    # nonzero values are standard normal
    from scipy import stats
    vals = R.val.astype(np.float64)
    assert abs(vals.mean()) < 5 / math.sqrt(nnz)
    assert abs(vals.var() - 1.0) < 5 * math.sqrt(2.0 / nnz)
    assert stats.kstest(vals, "norm").pvalue > 1e-4
    # the Bernoulli draws are spread evenly over dimensions and levels
    counts = np.bincount(R.dim, minlength=d)
    chi2 = ((counts - nnz / d) ** 2 / (nnz / d)).sum()
    assert stats.chi2.sf(chi2, d - 1) > 1e-4
    # each column's dimensions strictly ascend
    for c in range(R.ncols):
        seg = R.dim[R.col_off[c]:R.col_off[c + 1]]
        assert np.all(np.diff(seg) > 0)


def test_random_matrix_density_one_is_dense():
    """a = 1 is the classic dense RP tree (Sec. II-A, Table III 'RP-trees')."""
    R = oracle.random_matrix(3, 4, 50, 1.0, seed=1)
    assert np.all(np.diff(R.col_off) == 50)
    assert np.all(R.val != 0)


def test_random_matrix_prefix_stable_in_T():
    """Reading: draws are keyed by (tree, level, dimension), so the first
    trees of a larger index are the same trees."""
    a = oracle.random_matrix(3, 5, 64, 0.125, seed=11)
    b = oracle.random_matrix(7, 5, 64, 0.125, seed=11)
    n3 = a.col_off[-1]
    assert np.array_equal(a.col_off, b.col_off[:16])
    assert np.array_equal(a.dim, b.dim[:n3])
    assert np.array_equal(a.val, b.val[:n3])
    c = oracle.random_matrix(3, 5, 64, 0.125, seed=12)
    assert not np.array_equal(a.val, c.val[: len(a.val)]) or len(a.val) != len(c.val)


def test_fixed_count_variant_counts():
    """Footnote of Sec. II-D: exactly ceil(a d) nonzeros per vector (at
    least 1, at most d); values worked by hand."""
    for (a, d, k) in [(1.0 / math.sqrt(784), 784, 28), (0.3, 50, 15), (0.01, 50, 1),
                      (1.0, 50, 50), (1.0 / math.sqrt(128), 128, 12), (0.125, 64, 8)]:
        assert oracle.fixed_count(a, d) == k
        R = oracle.random_matrix(5, 3, d, a, seed=2, sparsity=oracle.SPARSITY_FIXED)
        assert np.all(np.diff(R.col_off) == k)
        for c in range(R.ncols):
            seg = R.dim[R.col_off[c]:R.col_off[c + 1]]
            assert np.all(np.diff(seg) > 0) and seg.min() >= 0 and seg.max() < d


def test_fixed_count_variant_nests_with_bernoulli_variant():
    """Both variants take the dimensions with the smallest first draw (the
    Bernoulli variant those below a, the fixed one the k smallest), so per
    column one set contains the other and shared dimensions carry the same
    normal value."""
    d, seed = 200, 5
    for a in (0.03, 0.1, 0.4):
        F = oracle.random_matrix(6, 4, d, a, seed, sparsity=oracle.SPARSITY_FIXED)
        B = oracle.random_matrix(6, 4, d, a, seed)
        for c in range(F.ncols):
            fd = F.dim[F.col_off[c]:F.col_off[c + 1]]
            fv = F.val[F.col_off[c]:F.col_off[c + 1]]
            bd = B.dim[B.col_off[c]:B.col_off[c + 1]]
            bv = B.val[B.col_off[c]:B.col_off[c + 1]]
            sf, sb = set(fd.tolist()), set(bd.tolist())
            assert sf <= sb or sb <= sf
            common = sorted(sf & sb)
            assert np.array_equal(fv[np.searchsorted(fd, common)], bv[np.searchsorted(bd, common)])
    # density 1: both are the dense matrix
    F = oracle.random_matrix(2, 3, 40, 1.0, 9, sparsity=oracle.SPARSITY_FIXED)
    B = oracle.random_matrix(2, 3, 40, 1.0, 9)
    assert np.array_equal(F.col_off, B.col_off) and np.array_equal(F.dim, B.dim)
    assert np.array_equal(F.val, B.val)


def test_fixed_count_variant_statistics_and_nesting():
    """A uniformly random k-subset per vector with N(0,1) values; a larger k
    keeps the smaller k's dimensions; the first trees are prefix-stable."""
    from scipy import stats
    T, l, d = 40, 8, 784
    a = 1.0 / math.sqrt(d)
    R = oracle.random_matrix(T, l, d, a, 7, sparsity=oracle.SPARSITY_FIXED)
    nnz = len(R.val)
    assert nnz == T * l * 28
    vals = R.val.astype(np.float64)
    assert abs(vals.mean()) < 5 / math.sqrt(nnz)
    assert abs(vals.var() - 1.0) < 5 * math.sqrt(2.0 / nnz)
    assert stats.kstest(vals, "norm").pvalue > 1e-4
    counts = np.bincount(R.dim, minlength=d)
    chi2 = ((counts - nnz / d) ** 2 / (nnz / d)).sum()
    assert stats.chi2.sf(chi2, d - 1) > 1e-4
    big = oracle.random_matrix(T, l, d, 2 * a, 7, sparsity=oracle.SPARSITY_FIXED)
    for c in range(0, R.ncols, 7):
        small = set(R.dim[R.col_off[c]:R.col_off[c + 1]].tolist())
        assert small <= set(big.dim[big.col_off[c]:big.col_off[c + 1]].tolist())
    few = oracle.random_matrix(3, l, d, a, 7, sparsity=oracle.SPARSITY_FIXED)
    assert np.array_equal(few.dim, R.dim[:len(few.dim)])
    assert np.array_equal(few.val, R.val[:len(few.val)])


# ---------------------------------------------------------- projection ----

def _round_to_f32(x: Fraction) -> np.float32:
    """Round an exact rational to the nearest float32, ties to even."""
    if x == 0:
        return np.float32(0.0)
    guess = np.float32(float(x))
    cands = [guess, np.nextafter(guess, np.float32(np.inf)),
             np.nextafter(guess, np.float32(-np.inf))]
    best = None
    for c in cands:
        if not np.isfinite(c):
            continue
        err = abs(Fraction(float(c)) - x)
        key = (err, int(np.array(c, dtype=np.float32).view(np.uint32)) & 1)
        if best is None or key < best[0]:
            best = (key, c)
    return np.float32(best[1])


def test_projection_is_correctly_rounded_fma_chain():
    """P = XR (Algorithm 1) as a chain of single-rounding fused
    multiply-adds over ascending dimension from +0 -- recomputed here in
    exact rational arithmetic with one rounding per step."""
    g = np.random.default_rng(3)
    n, d = 6, 37
    X = (g.standard_normal((n, d)) * g.choice([1e-3, 1.0, 300.0], size=(n, 1))).astype(np.float32)
    X[1, ::3] = 0.0
    R = oracle.random_matrix(2, 3, d, 0.3, seed=5)
    P = oracle.project(X, R)
    for x in range(n):
        for c in range(R.ncols):
            acc = np.float32(0.0)
            for e in range(R.col_off[c], R.col_off[c + 1]):
                exact = (Fraction(float(X[x, R.dim[e]])) * Fraction(float(R.val[e]))
                         + Fraction(float(acc)))
                acc = _round_to_f32(exact)
            assert np.float32(P[x, c]).tobytes() == acc.tobytes(), (x, c)


def test_projection_matches_dense_product():
    """Same values as a float64 dense X @ R within the chain's error bound,
    which pins the operand layout (row of X against column of R)."""
    g = np.random.default_rng(4)
    X = g.standard_normal((50, 64)).astype(np.float32)
    R = oracle.random_matrix(4, 6, 64, 0.25, seed=9)
    P = oracle.project(X, R)
    exact = X.astype(np.float64) @ R.dense().astype(np.float64)
    bound = (np.abs(X).astype(np.float64) @ np.abs(R.dense()).astype(np.float64)) * 64 * 2**-23
    assert np.all(np.abs(P - exact) <= bound + 1e-30)


# --------------------------------------------------------- hand example ----

def _hand_index(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "hand_8points.json")))
    X = np.array(g["X"], dtype=np.float32)
    cols = g["R_columns"]
    col_off = [0]
    dims, vals = [], []
    for c in cols:
        dims += c["dim"]
        vals += c["val"]
        col_off.append(len(dims))
    R = oracle.RandomMatrix(np.array(col_off, np.int32), np.array(dims, np.int32),
                            np.array(vals, np.float32), X.shape[1])
    idx = oracle.grow_trees(X, T=2, l=g["l"], density=1.0, seed=0, R=R)
    return g, idx


def test_hand_example_tree_growth(golden_dir):
    g, idx = _hand_index(golden_dir)
    assert np.array_equal(idx.split, np.array(g["split"], np.float32))
    assert np.array_equal(idx.leaf_off, np.array(g["leaf_off"], np.int32))
    assert np.array_equal(idx.leaf_ids, np.array(g["leaf_ids"], np.int32))


def _f(x):
    return math.inf if x == "inf" else float(x)


def test_hand_example_queries(golden_dir):
    g, idx = _hand_index(golden_dir)
    for qcase in g["queries"]:
        q = np.array([qcase["q"]], dtype=np.float32)
        for case in qcase["cases"]:
            k, v = case["k"], case["v"]
            ids, dists, proj, leaf, ncand = oracle.query(idx, q, k, v, want_internals=True)
            assert leaf[0].tolist() == qcase["leaf"]
            F, S = oracle.votes(idx, leaf[0], v)
            nz = {str(i): int(F[i]) for i in np.nonzero(F)[0]}
            assert nz == qcase["votes_nonzero"]
            assert sorted(S.tolist()) == case["S"]
            assert int(ncand[0]) == len(case["S"])
            assert ids[0].tolist() == case["ids"]
            np.testing.assert_allclose(dists[0], [_f(x) for x in case["dists"]], rtol=1e-7)
            for mode in (0, 1):
                i2, d2 = oracle.query(idx, q, k, v, mode=mode)
                assert i2[0].tolist() == case["ids"]


# ------------------------------------------------ special cases / brute ----

def _numpy_knn(X, q, S, k):
    """Independent exact k-NN on the index set S, ordered by (dist, id)."""
    S = np.asarray(S, dtype=np.int64)
    dd = ((X[S].astype(np.float64) - q.astype(np.float64)) ** 2).sum(1)
    order = np.lexsort((S, dd))[:k]
    ids = np.full(k, -1, np.int64)
    dist = np.full(k, np.inf)
    ids[: len(order)] = S[order]
    dist[: len(order)] = np.sqrt(dd[order])
    return ids, dist


def test_single_leaf_reduces_to_exact_knn():
    """T = 1, l = 0, v = 1: the one leaf holds every point, so S = X and
    Algorithm 4 returns exact k-NN (Sec. I-A)."""
    X, Q = workloads.gaussian_mixture(300, 16, 20, n_centres=5, seed=2)
    idx = oracle.grow_trees(X, T=1, l=0, density=0.25, seed=0)
    ids, dists = oracle.query(idx, Q, k=7, v=1)
    bids, bdists = oracle.brute_knn(X, Q, k=7)
    for i, q in enumerate(Q):
        eids, edist = _numpy_knn(X, q, np.arange(len(X)), 7)
        assert ids[i].tolist() == eids.tolist()
        assert bids[i].tolist() == eids.tolist()
        np.testing.assert_allclose(dists[i], edist, rtol=1e-6)
        np.testing.assert_allclose(bdists[i], edist, rtol=1e-6)


def test_knn_pads_and_breaks_ties_by_id():
    X = np.array([[0, 0], [1, 0], [0, 1], [5, 5]], np.float32)
    q = np.array([0, 0], np.float32)
    ids, d = oracle.knn(X, q, np.array([3, 2, 1]), 5)
    assert ids.tolist() == [1, 2, 3, -1, -1]
    assert np.isinf(d[3:]).all() and d[0] == 1.0 and d[1] == 1.0
    ids, d = oracle.knn(X, q, np.array([], np.int32), 2)
    assert ids.tolist() == [-1, -1]


def test_d1_dense_leaves_are_rank_blocks():
    """d = 1, a = 1: every level projects onto a multiple of x, so each leaf
    is a contiguous block of points in rank order of r*x (ties by id), and
    blocks have ceil/floor(n/2^l) points (Sec. III-A)."""
    g = np.random.default_rng(8)
    n, l = 101, 3
    X = g.integers(-20, 20, size=(n, 1)).astype(np.float32)  # many ties
    R = oracle.random_matrix(1, l, 1, 1.0, seed=3)
    r = R.val
    # this check needs every level's vector to have the same sign
    assert np.all(r > 0) or np.all(r < 0)
    idx = oracle.grow_trees(X, T=1, l=l, density=1.0, seed=3, R=R)
    key = X[:, 0] * r[0]
    order = np.lexsort((np.arange(n), key))
    off = idx.leaf_off[0]
    sizes = np.diff(off)
    assert set(sizes.tolist()) <= {n // 8, -(-n // 8)}
    for b in range(8):
        assert idx.leaf_ids[0, off[b]:off[b + 1]].tolist() == sorted(order[off[b]:off[b + 1]].tolist())


# ----------------------------------------------------------- invariants ----

@pytest.fixture(scope="module")
def small_index():
    X, Q = workloads.gaussian_mixture(3000, 32, 40, n_centres=20, sigma=0.4, seed=5)
    idx = oracle.grow_trees(X, T=12, l=5, density=32 ** -0.5, seed=1)
    return X, Q, idx


def _leaf_of_points(idx):
    """leaf_of[t, x]: the leaf holding point x in tree t."""
    lo = np.full((idx.T, idx.n), -1, np.int64)
    for t in range(idx.T):
        off = idx.leaf_off[t]
        for b in range(idx.L):
            lo[t, idx.leaf_ids[t, off[b]:off[b + 1]]] = b
    return lo


def test_each_point_in_exactly_one_leaf(small_index):
    X, Q, idx = small_index
    n, L = idx.n, idx.L
    for t in range(idx.T):
        assert np.array_equal(np.sort(idx.leaf_ids[t]), np.arange(n))
        sizes = np.diff(idx.leaf_off[t])
        assert set(sizes.tolist()) <= {n // L, -(-n // L)}
        for b in range(L):
            seg = idx.leaf_ids[t, idx.leaf_off[t, b]:idx.leaf_off[t, b + 1]]
            assert np.all(np.diff(seg) > 0)


def test_splits_are_medians(small_index):
    """Every inner node's split is the largest left-side projection, no
    right-side point projects below it (Sec. II-A, Algorithm 2)."""
    X, Q, idx = small_index
    l, L = idx.l, idx.L
    for t in range(idx.T):
        off = idx.leaf_off[t]
        for j in range(l):
            span = L >> j  # leaves under a node at level j
            for b in range(1 << j):
                node = (1 << j) - 1 + b
                lo, mid, hi = b * span, b * span + span // 2, (b + 1) * span
                left = idx.leaf_ids[t, off[lo]:off[mid]]
                right = idx.leaf_ids[t, off[mid]:off[hi]]
                kl = idx.P[left, t * l + j]
                kr = idx.P[right, t * l + j]
                assert len(left) == -(-(len(left) + len(right)) // 2)
                assert kl.max() == idx.split[t, node]
                assert kr.min() >= idx.split[t, node]


def test_points_route_to_their_own_leaf(small_index):
    """With continuous data (no ties), routing a data point as a query
    (Algorithm 3) lands in the leaf that Algorithm 2 put it in."""
    X, Q, idx = small_index
    lo = _leaf_of_points(idx)
    _, _, _, leaf, _ = oracle.query(idx, X[:300], k=1, v=1, want_internals=True)
    assert np.array_equal(leaf, lo[:, :300].T)


def test_votes_match_definition(small_index):
    """F(x; q) = sum_t 1{x and q share a leaf in tree t} (Sec. III-A),
    computed from leaf membership, equals Algorithm 4's counters; S(v) =
    {x : F >= v}; v = 1 gives the union of the leaves (defeatist search);
    |S| <= T ceil(n/2^l) (Sec. III-B); and the totals agree."""
    X, Q, idx = small_index
    lo = _leaf_of_points(idx)
    _, _, _, leaf, ncand = oracle.query(idx, Q, k=5, v=3, want_internals=True)
    for i in range(len(Q)):
        Fdef = (lo == leaf[i][:, None]).sum(0)
        union = set()
        for t in range(idx.T):
            union |= set(np.nonzero(lo[t] == leaf[i, t])[0].tolist())
        for v in (1, 2, 3, 5, 12):
            F, S = oracle.votes(idx, leaf[i], v)
            assert np.array_equal(F, Fdef)
            assert sorted(S.tolist()) == np.nonzero(Fdef >= v)[0].tolist()
            assert len(S) <= idx.T * -(-idx.n // idx.L)
            if v == 1:
                assert set(S.tolist()) == union
        assert F.sum() == sum(np.diff(idx.leaf_off[t])[leaf[i, t]] for t in range(idx.T))
        assert ncand[i] == (Fdef >= 3).sum()


def test_exact_search_on_candidates(small_index):
    """knn(q, k, S) returns the k nearest members of S (Sec. I-A metric)."""
    X, Q, idx = small_index
    ids, dists, _, leaf, _ = oracle.query(idx, Q, k=10, v=2, want_internals=True)
    for i, q in enumerate(Q):
        _, S = oracle.votes(idx, leaf[i], 2)
        eids, ed = _numpy_knn(X, q, S, 10)
        assert ids[i].tolist() == eids.tolist()
        np.testing.assert_allclose(dists[i], ed, rtol=1e-6)


def test_monotone_in_trees_and_threshold(small_index):
    """With prefix-stable trees, S grows with T and shrinks with v, so
    recall is non-decreasing in T and non-increasing in v (Sec. III-A)."""
    X, Q, idx = small_index
    truth, _ = oracle.brute_knn(X, Q, 10)
    prev = -1.0
    for T in (1, 3, 6, 12):
        ids, _ = oracle.query(idx, Q, 10, 1, T=T)
        r = oracle.recall(ids, truth)
        assert r >= prev
        prev = r
    prev = 2.0
    for v in (1, 2, 3, 4, 6):
        ids, _ = oracle.query(idx, Q, 10, v)
        r = oracle.recall(ids, truth)
        assert r <= prev
        prev = r
    _, _, _, leaf, _ = oracle.query(idx, Q, 10, 1, want_internals=True)
    for i in range(5):
        for v in (1, 2, 4):
            _, S6 = oracle.votes(idx, leaf[i], v, T=6)
            _, S12 = oracle.votes(idx, leaf[i], v, T=12)
            _, S12b = oracle.votes(idx, leaf[i], v + 1, T=12)
            assert set(S6.tolist()) <= set(S12.tolist())
            assert set(S12b.tolist()) <= set(S12.tolist())


def test_fp32_mode_close_to_fp64(small_index):
    X, Q, idx = small_index
    i64, d64 = oracle.query(idx, Q, 10, 2, mode=0)
    i32, d32 = oracle.query(idx, Q, 10, 2, mode=1)
    fin = np.isfinite(d64)
    np.testing.assert_allclose(d32[fin], d64[fin], rtol=1e-5)


def test_integer_data_fp32_distances_exact():
    """Integer data with squared distances below 2^24 gives exact float
    distances in any order, so both modes agree bit for bit."""
    X, Q = workloads.lognormal_int(400, 16, 10, seed=3)
    idx = oracle.grow_trees(X, T=4, l=3, density=0.25, seed=2)
    a = oracle.query(idx, Q, 10, 1, mode=0)
    b = oracle.query(idx, Q, 10, 1, mode=1)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1] ** 2, b[1] ** 2) or np.allclose(a[1], b[1], rtol=1e-7)


def test_rejects_too_deep_trees():
    P = np.zeros((5, 3), np.float32)
    with pytest.raises(ValueError):
        oracle.grow_tree(P, 0, 3)
