"""GPU parity: the CUDA library (through the C ABI) against the oracle on
the same seeded inputs.  Bit-exact: random matrix, split values, leaves,
query projections, leaf of every query, vote counts and candidate sets.
Distances within 1e-5 relative of the oracle's float64; ids equal except at
ties."""
import numpy as np
import pytest

import oracle
import workloads
from _parity import REL_TOL, check_index_parity, check_results, oracle_sets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_06957_gb300 as m
    m.load_library()
    return m


def _dens(d):
    return float(np.float32(1.0 / np.sqrt(d)))


def _run(mr, X, Q, T, l, k, v, density, seed, n_trees=0, host=False, path=0, vote_table=0):
    dev = torch.device("cuda:0")
    if host:
        idx = mr.mrpt_build(X, T, l, density, seed)
        ids, dists, dbg = mr.mrpt_query_ex(idx, Q, k, v, n_trees=n_trees, debug=True, path=path,
                                           vote_table=vote_table)
        return idx, ids, dists, dbg
    idx = mr.mrpt_build(torch.from_numpy(X).to(dev), T, l, density, seed)
    ids, dists, dbg = mr.mrpt_query_ex(idx, torch.from_numpy(Q).to(dev), k, v, n_trees=n_trees,
                                       debug=True, path=path, vote_table=vote_table)
    torch.cuda.synchronize()
    return idx, ids.cpu().numpy(), dists.cpu().numpy(), {kk: vv.cpu().numpy() for kk, vv in dbg.items()}


def _full_check(mr, X, Q, T, l, k, v, density, seed, n_trees=0, host=False, path=0, vote_table=0):
    idx, gi, gd, dbg = _run(mr, X, Q, T, l, k, v, density, seed, n_trees, host, path, vote_table)
    ref = oracle.grow_trees(X, T, l, density, seed)
    check_index_parity(idx, mr, ref)
    Tq = n_trees or T
    oi, od, oproj, oleaf, oncand = oracle.query(ref, Q, k, v, T=Tq, want_internals=True)
    assert np.array_equal(dbg["proj"].view(np.uint32), oproj.view(np.uint32)), "projections"
    assert np.array_equal(dbg["leaf"], oleaf), "leaf of query"
    assert np.array_equal(dbg["n_cand"], oncand), "|S|"
    sets = oracle_sets(ref, oleaf, v, T=Tq)
    for i in range(len(Q)):
        F, _ = oracle.votes(ref, oleaf[i], v, T=Tq)
        assert np.array_equal(dbg["votes"][i], F.astype(np.uint8)), f"votes of query {i}"
        got = set(dbg["cand"][i][: dbg["n_cand"][i]].tolist())
        assert got == sets[i], f"candidate set of query {i}"
    check_results(X, Q, gi, gd, oi, od, sets)
    idx.close()
    return gi, gd


PATHS = [0, 1]  # vote/emit + candidate search, one fused kernel


@pytest.mark.parametrize("path", PATHS)
def test_tiny_gaussian_mixture(mr, path):
    """n=10,000, d=128, 100 clusters, T=10, l=6, v=3, k=10, seed 0."""
    X, Q = workloads.gaussian_mixture(10000, 128, 100, seed=0)
    _full_check(mr, X, Q, 10, 6, 10, 3, _dens(128), 0, path=path)


@pytest.mark.parametrize("path", PATHS)
def test_mnist_like_small_with_ties(mr, path):
    """Sparse integer images: many projections tie exactly (often at 0), so
    the (projection, id) median order is exercised."""
    X, Q = workloads.mnist_like(4000, 40, seed=1)
    _full_check(mr, X, Q, 16, 5, 10, 2, _dens(784), 3, path=path)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("k", [1, 33, 100, 256])
def test_k_values_and_padding(mr, k, path):
    X, Q = workloads.gaussian_mixture(1500, 24, 30, n_centres=8, seed=4)
    _full_check(mr, X, Q, 5, 3, k, 2, 0.3, 5, path=path)


@pytest.mark.parametrize("path", PATHS)
def test_candidate_sets_of_thousands(mr, path):
    """v = 1 on two-leaf trees: |S| of several thousand per query, all in
    the candidate lists (sized T ceil(n / 2^l) / v) and work items."""
    X, Q = workloads.gaussian_mixture(6000, 12, 20, n_centres=3, seed=12)
    _full_check(mr, X, Q, 6, 1, 10, 1, 0.5, 3, path=path)


def test_ragged_dimension_and_host_buffers(mr):
    """d not a multiple of 4 or 8, n odd, numpy (host) inputs and outputs."""
    X, Q = workloads.gaussian_mixture(1001, 37, 17, n_centres=6, seed=6)
    _full_check(mr, X, Q, 7, 4, 10, 2, 0.2, 9, host=True)


@pytest.mark.parametrize("d,T,l,density", [
    (100, 37, 5, 0.1),   # 64-query tiles, 32 warps per block
    (100, 37, 1, 0.02),  # depth 1; many empty columns
    (800, 21, 4, 0.05),  # 64-query tiles, 16 warps per block
    (800, 5, 3, 1.0),    # dense vectors: columns span many ring chunks
    (900, 19, 4, 0.05),  # tile too large: one query per lane
])
def test_routing_kernels(mr, d, T, l, density):
    """Projections and leaves of every query, bit-exact, for each routing
    kernel: 150 queries (two full 64-query tiles and a ragged one), tree
    counts that are not multiples of the warps per block."""
    X, Q = workloads.gaussian_mixture(3000, d, 150, n_centres=12, seed=d + l)
    dev = torch.device("cuda:0")
    idx = mr.mrpt_build(torch.from_numpy(X).to(dev), T, l, density, 21)
    _, _, dbg = mr.mrpt_query_ex(idx, torch.from_numpy(Q).to(dev), 5, 1, debug=True)
    torch.cuda.synchronize()
    ref = oracle.grow_trees(X, T, l, density, 21)
    _, _, oproj, oleaf, _ = oracle.query(ref, Q, 5, 1, want_internals=True)
    assert np.array_equal(dbg["proj"].cpu().numpy().view(np.uint32), oproj.view(np.uint32)), "projections"
    assert np.array_equal(dbg["leaf"].cpu().numpy(), oleaf), "leaf of query"
    idx.close()


def test_single_leaf_is_exact_knn(mr):
    """T = 1, l = 0, v = 1: S = X, so the result is exact k-NN (Sec. I-A)."""
    X, Q = workloads.gaussian_mixture(700, 19, 20, n_centres=4, seed=8)
    gi, gd = _full_check(mr, X, Q, 1, 0, 12, 1, 0.5, 1)
    bi, bd = oracle.brute_knn(X, Q, 12)
    check_results(X, Q, gi, gd, bi, bd)


def test_vote_threshold_equal_to_T_and_subset_of_trees(mr):
    X, Q = workloads.gaussian_mixture(2500, 32, 25, n_centres=10, seed=9)
    _full_check(mr, X, Q, 8, 4, 10, 8, _dens(32), 2)
    _full_check(mr, X, Q, 8, 4, 10, 3, _dens(32), 2, n_trees=5)


# (path, vote table): the fused kernel's own id chunks, then path 0 with
# counters over id chunks and with the hash table
VOTE_MODES = [(1, 0), (0, 1), (0, 2)]


@pytest.mark.parametrize("path,vote_table", VOTE_MODES, ids=["fused", "counters", "hash"])
@pytest.mark.parametrize("l", [9, 12])
def test_counter_chunks_beyond_shared_memory(mr, path, vote_table, l):
    """n > 65,536 ids.  Counters: votes in id chunks (per-tree cursors); depth
    9 (leaves of 274, about 91 per chunk) takes per-tree windows, depth 12
    (leaves of 35, about 12 per chunk) windows over the chunk's segments laid
    end to end.  Hash: one table of (id, count) words for the query's 6
    leaves.  Votes, |S|, S and rows equal the oracle's."""
    X, Q = workloads.gaussian_mixture(140000, 8, 12, n_centres=30, seed=10)
    _full_check(mr, X, Q, 6, l, 10, 2, 0.5, 4, path=path, vote_table=vote_table)


@pytest.mark.parametrize("v", [1, 3])
def test_hashed_votes_full_table_load(mr, v):
    """The hash table at its capacity: 96 trees of depth 9 over n = 131,072
    hold 96 * 256 = 24,576 entries per query (3/4 of the table's slots), the
    most it takes.  Votes, |S|, S and rows equal the oracle's at v = 1 and
    3."""
    X, Q = workloads.gaussian_mixture(131072, 8, 6, n_centres=30, seed=12)
    _full_check(mr, X, Q, 96, 9, 10, v, 0.5, 6, vote_table=2)


def test_hashed_votes_refused_beyond_capacity(mr):
    """vote_table = 2 with more than 24,576 leaf entries per query is
    refused before any work."""
    X, Q = workloads.gaussian_mixture(131072, 8, 2, n_centres=30, seed=12)
    idx = mr.mrpt_build(torch.from_numpy(X).cuda(), 97, 9, 0.5, 6)
    with pytest.raises(mr.MRPTError) as e:
        mr.mrpt_query_ex(idx, torch.from_numpy(Q).cuda(), 10, 2, vote_table=2)
    assert e.value.code == mr.MRPT_ERR_INVALID_ARG
    ids, _ = mr.mrpt_query_ex(idx, torch.from_numpy(Q).cuda(), 10, 2, n_trees=96, vote_table=2)
    torch.cuda.synchronize()
    assert ids.shape == (2, 10)
    idx.close()


def test_degenerate_all_equal_points(mr):
    """Every projection ties: splits are decided by id alone."""
    X = np.ones((300, 5), np.float32)
    Q = np.ones((4, 5), np.float32)
    _full_check(mr, X, Q, 3, 3, 5, 1, 1.0, 0)


def test_empty_batch(mr):
    X, Q = workloads.gaussian_mixture(200, 8, 1, seed=1)
    idx = mr.mrpt_build(torch.from_numpy(X).cuda(), 2, 2, 0.5, 0)
    ids, dists = mr.mrpt_query(idx, torch.empty((0, 8), device="cuda"), 5, 1)
    assert ids.shape == (0, 5)
    idx.close()


def test_prefix_stable_trees(mr):
    """The first trees of a larger index are the same trees."""
    X, _ = workloads.gaussian_mixture(3000, 16, 1, seed=2)
    a = mr.mrpt_build(X, 4, 5, 0.25, 77)
    b = mr.mrpt_build(X, 9, 5, 0.25, 77)
    assert np.array_equal(mr.mrpt_export(a, "SPLIT"), mr.mrpt_export(b, "SPLIT")[:4])
    assert np.array_equal(mr.mrpt_export(a, "LEAF_IDS"), mr.mrpt_export(b, "LEAF_IDS")[:4])
    a.close()
    b.close()


@pytest.mark.slow
def test_mnist_like_full_size_sampled(mr):
    """n=60,000, d=784, l=8 (the benchmark's shape) at T=50: full index
    parity, and a sample of 64 queries through every internal."""
    X, Q = workloads.mnist_like(60000, 64, seed=0)
    _full_check(mr, X, Q, 50, 8, 10, 4, _dens(784), 0)


# ---------------------------------------------------------------- errors --

def test_invalid_arguments(mr):
    X = np.zeros((16, 4), np.float32)
    for args in [(X, 0, 1), (X, 256, 1), (X, 2, 5), (X, 2, -1)]:
        with pytest.raises(mr.MRPTError) as e:
            mr.mrpt_build(*args)
        assert e.value.code == mr.MRPT_ERR_INVALID_ARG
    idx = mr.mrpt_build(X + np.arange(16, dtype=np.float32)[:, None], 2, 2, 1.0, 0)
    q = np.zeros((2, 4), np.float32)
    for k, v in [(0, 1), (257, 1), (3, 0), (3, 3)]:
        with pytest.raises(mr.MRPTError) as e:
            mr.mrpt_query(idx, q, k, v)
        assert e.value.code == mr.MRPT_ERR_INVALID_ARG
    idx.close()


def test_nonfinite_inputs(mr):
    X = np.random.default_rng(0).standard_normal((64, 6)).astype(np.float32)
    bad = X.copy()
    bad[5, 2] = np.nan
    with pytest.raises(mr.MRPTError) as e:
        mr.mrpt_build(bad, 2, 2, 0.5, 0)
    assert e.value.code == mr.MRPT_ERR_NONFINITE_INPUT
    idx = mr.mrpt_build(torch.from_numpy(X).cuda(), 2, 2, 0.5, 0)
    q = torch.zeros((3, 6), device="cuda")
    q[1, 3] = float("inf")
    mr.mrpt_query(idx, q, 4, 1)  # device buffers: latched, reported by sync
    with pytest.raises(mr.MRPTError) as e:
        mr.mrpt_sync(idx)
    assert e.value.code == mr.MRPT_ERR_NONFINITE_INPUT
    mr.mrpt_sync(idx)  # cleared
    with pytest.raises(mr.MRPTError) as e:  # host buffers: reported by the call
        mr.mrpt_query(idx, q.cpu().numpy(), 4, 1)
    assert e.value.code == mr.MRPT_ERR_NONFINITE_INPUT
    idx.close()


def test_injected_allocation_failure(mr):
    X = np.random.default_rng(1).standard_normal((128, 8)).astype(np.float32)
    for after in range(0, 6):
        mr.mrpt_debug_fail_alloc_after(after)
        try:
            idx = mr.mrpt_build(X, 3, 3, 0.5, 0)
            idx.close()
        except mr.MRPTError as e:
            assert e.code == mr.MRPT_ERR_OOM
        finally:
            mr.mrpt_debug_fail_alloc_after(-1)
    idx = mr.mrpt_build(X, 3, 3, 0.5, 0)  # the library is still usable
    ids, _ = mr.mrpt_query(idx, X[:4], 3, 1)
    assert ids[:, 0].tolist() == [0, 1, 2, 3]
    idx.close()


def test_batch_beyond_the_candidate_scratch_budget(mr):
    """v = 1 on two trees of depth 1 over 60,000 points: the list capacity
    is n = 60,000 per query, so 9,000 queries need more candidate scratch
    than one launch may use (2 GiB) and run as consecutive sub-batches.
    Every row equals the oracle's; stage times are the sum over them."""
    X, Q = workloads.gaussian_mixture(60000, 8, 9000, n_centres=40, seed=31)
    idx = mr.mrpt_build(torch.from_numpy(X).cuda(), 2, 1, 0.5, 8)
    stage = np.zeros(4, np.float32)
    ids, dists = mr.mrpt_query_ex(idx, torch.from_numpy(Q).cuda(), 10, 1, stage_ms=stage)
    torch.cuda.synchronize()
    assert stage[3] > 0 and stage[1] > 0 and stage[2] > 0
    ref = oracle.grow_trees(X, 2, 1, 0.5, 8)
    check_index_parity(idx, mr, ref)
    oi, od, _, oleaf, oncand = oracle.query(ref, Q, 10, 1, want_internals=True)
    assert oncand.min() > 30000
    gi, gd = ids.cpu().numpy(), dists.cpu().numpy()
    diff = np.nonzero((gi != oi).any(1))[0]
    sets = dict(zip(diff.tolist(), oracle_sets(ref, oleaf[diff], 1)))
    check_results(X, Q, gi, gd, oi, od, [sets.get(i, set()) for i in range(len(Q))])
    idx.close()
