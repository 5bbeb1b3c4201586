"""CPU: the comparison that the GPU parity tests use (tests/_parity.py) is
not vacuous.  The oracle's own answer passes it; the same answer with one
planted error (a wrong id, a distance off by more than the tolerance,
padding in the wrong place, a duplicate, an id outside S, an id beyond the
k-th neighbour) fails it; a swap of two ids at an exact tie passes."""
import numpy as np
import pytest

import oracle
import workloads
from _parity import REL_TOL, check_results, oracle_sets


@pytest.fixture(scope="module")
def case():
    X, Q = workloads.lognormal_int(3000, 16, 24, seed=9)  # integer data: exact ties occur
    ref = oracle.grow_trees(X, 6, 4, 0.5, 3)
    ids, dists, _, leaf, _ = oracle.query(ref, Q, 10, 2, want_internals=True)
    return X, Q, ids, dists, oracle_sets(ref, leaf, 2)


def test_oracle_answer_passes(case):
    X, Q, ids, dists, sets = case
    check_results(X, Q, ids.copy(), dists.copy(), ids, dists, sets)


def _row_with_full_result(dists):
    return int(np.flatnonzero(np.isfinite(dists).all(axis=1))[0])


def test_wrong_id_fails(case):
    X, Q, ids, dists, sets = case
    i = _row_with_full_result(dists)
    gi = ids.copy()
    outside = next(x for x in range(len(X)) if x not in sets[i])
    gi[i, 0] = outside
    with pytest.raises(AssertionError):
        check_results(X, Q, gi, dists.copy(), ids, dists, sets)


def test_distance_beyond_tolerance_fails(case):
    X, Q, ids, dists, sets = case
    i = _row_with_full_result(dists)
    gd = dists.copy()
    gd[i, 3] *= 1 + 10 * REL_TOL
    with pytest.raises(AssertionError):
        check_results(X, Q, ids.copy(), gd, ids, dists, sets)


def test_padding_mismatch_fails(case):
    X, Q, ids, dists, sets = case
    i = _row_with_full_result(dists)
    gi, gd = ids.copy(), dists.copy()
    gi[i, -1], gd[i, -1] = -1, np.inf
    with pytest.raises(AssertionError):
        check_results(X, Q, gi, gd, ids, dists, sets)


def test_duplicate_id_fails(case):
    X, Q, ids, dists, sets = case
    i = _row_with_full_result(dists)
    gi, gd = ids.copy(), dists.copy()
    gi[i, 1], gd[i, 1] = gi[i, 0], gd[i, 0]
    with pytest.raises(AssertionError):
        check_results(X, Q, gi, gd, ids, dists, sets)


def test_id_beyond_the_kth_neighbour_fails(case):
    """A member of S farther than the k-th neighbour in the last slot, with
    the oracle's distance reported there: the returned id is not at the
    distance reported."""
    X, Q, ids, dists, sets = case
    for i in range(len(Q)):
        if not np.isfinite(dists[i]).all():
            continue
        d_all = np.sqrt(((X.astype(np.float64) - Q[i].astype(np.float64)) ** 2).sum(1))
        far = [x for x in sets[i] if d_all[x] > dists[i, -1] * (1 + 1e-3)]
        if far:
            gi, gd = ids.copy(), dists.copy()
            gi[i, -1] = far[0]
            with pytest.raises(AssertionError):
                check_results(X, Q, gi, gd, ids, dists, sets)
            return
    pytest.skip("no query with a farther member of S")


def test_swap_at_an_exact_tie_passes(case):
    X, Q, ids, dists, sets = case
    for i in range(len(Q)):
        for j in range(ids.shape[1] - 1):
            if np.isfinite(dists[i, j]) and dists[i, j] == dists[i, j + 1]:
                gi = ids.copy()
                gi[i, j], gi[i, j + 1] = gi[i, j + 1], gi[i, j]
                check_results(X, Q, gi, dists.copy(), ids, dists, sets)
                return
    pytest.skip("no exact tie in this sample")


# ---- the reduced-precision comparison (ids in S, exact distances, recall)

def test_lowp_oracle_answer_passes(case):
    from _parity import check_lowp_results
    X, Q, ids, dists, sets = case
    assert check_lowp_results(X, Q, ids.copy(), dists.copy(), ids, dists, sets, 1.0) == 1.0


def test_lowp_missing_neighbour_lowers_recall(case):
    """A true neighbour replaced by the next member of S (its exact
    distance reported, the row re-sorted) passes the exactness checks and
    lowers the recall: the bound decides."""
    from _parity import check_lowp_results
    X, Q, ids, dists, sets = case
    i = _row_with_full_result(dists)
    S = np.array(sorted(sets[i]))
    ex = np.sqrt(((X[S].astype(np.float64) - Q[i].astype(np.float64)) ** 2).sum(1))
    order = np.lexsort((S, ex))
    k = ids.shape[1]
    if len(S) <= k:
        pytest.skip("S too small")
    pick = np.concatenate([order[1:k], order[k:k + 1]])      # drop the nearest, take the (k+1)-th
    if ex[order[k]] <= dists[i, -1] * (1 + REL_TOL):
        pytest.skip("the (k+1)-th ties the k-th")
    gi, gd = ids.copy(), dists.copy()
    gi[i], gd[i] = S[pick], ex[pick].astype(np.float32)
    rec = check_lowp_results(X, Q, gi, gd, ids, dists, sets, 0.0)
    assert rec < 1.0
    with pytest.raises(AssertionError):
        check_lowp_results(X, Q, gi, gd, ids, dists, sets, 1.0)


@pytest.mark.parametrize("mistake", ["outside", "distance", "order", "duplicate", "padding"])
def test_lowp_planted_errors_fail(case, mistake):
    from _parity import check_lowp_results
    X, Q, ids, dists, sets = case
    i = _row_with_full_result(dists)
    gi, gd = ids.copy(), dists.copy()
    if mistake == "outside":
        gi[i, 0] = next(x for x in range(len(X)) if x not in sets[i])
    elif mistake == "distance":
        gd[i, 3] *= 1 + 10 * REL_TOL
    elif mistake == "order":
        gi[i, [2, 7]], gd[i, [2, 7]] = gi[i, [7, 2]], gd[i, [7, 2]]
        if gd[i, 2] == gd[i, 7]:
            pytest.skip("tie")
    elif mistake == "duplicate":
        gi[i, 1], gd[i, 1] = gi[i, 0], gd[i, 0]
    else:
        gi[i, -1], gd[i, -1] = -1, np.inf
    with pytest.raises(AssertionError):
        check_lowp_results(X, Q, gi, gd, ids, dists, sets, 0.0)
