"""Helpers shared by the GPU parity tests: run the library and the oracle on
the same seeded inputs and compare."""
import numpy as np

import oracle

REL_TOL = 1e-5  # float32 distances vs the oracle's float64 (relative)


def check_index_parity(idx, mr, ref):
    """Bit-exact random matrix, split values and leaves."""
    assert np.array_equal(mr.mrpt_export(idx, "R_COL_OFF"), ref.R.col_off)
    assert np.array_equal(mr.mrpt_export(idx, "R_DIM"), ref.R.dim)
    assert np.array_equal(mr.mrpt_export(idx, "R_VAL").view(np.uint32), ref.R.val.view(np.uint32))
    assert np.array_equal(mr.mrpt_export(idx, "SPLIT").view(np.uint32),
                          ref.split.view(np.uint32))
    assert np.array_equal(mr.mrpt_export(idx, "LEAF_OFF"), ref.leaf_off)
    assert np.array_equal(mr.mrpt_export(idx, "LEAF_IDS"), ref.leaf_ids)


def check_results(X, Q, gi, gd, oi, od, cand_sets=None):
    """The library's k-NN rows against the oracle's:

    * padding (-1, +inf) in the same places;
    * distances position by position within REL_TOL of the oracle's;
    * ids equal, except where the oracle's distances tie within REL_TOL --
      there every returned id must be a member of S, unique, at the
      distance reported, and no farther than the oracle's k-th neighbour.
    """
    m, k = oi.shape
    fin = np.isfinite(od)
    assert np.array_equal(np.isfinite(gd), fin), "padding differs"
    assert np.array_equal(gi == -1, ~fin), "padding ids differ"
    if fin.any():
        np.testing.assert_allclose(gd[fin], od[fin], rtol=REL_TOL, atol=1e-30)
    for i in range(m):
        got = gi[i][fin[i]]
        want = oi[i][fin[i]]
        if np.array_equal(got, want):
            continue
        assert len(set(got.tolist())) == len(got), f"query {i}: duplicate ids"
        if cand_sets is not None:
            assert set(got.tolist()) <= cand_sets[i], f"query {i}: id outside S"
        ex = np.sqrt(((X[got].astype(np.float64) - Q[i].astype(np.float64)) ** 2).sum(1))
        np.testing.assert_allclose(ex, gd[i][fin[i]], rtol=REL_TOL, atol=1e-30)
        kth = od[i][fin[i]][-1]
        assert np.all(ex <= kth * (1 + REL_TOL) + 1e-30), f"query {i}: id beyond the k-th"


def oracle_sets(ref, leaf, v, T=None):
    out = []
    for row in leaf:
        _, S = oracle.votes(ref, row, v, T=T)
        out.append(set(S.tolist()))
    return out


def check_lowp_results(X, Q, gi, gd, oi, od, cand_sets, min_recall):
    """Rows from reduced-precision candidate distances with a float32
    re-rank, against the oracle's exact rows.  The re-rank restores exact
    order only among the survivors, so a true neighbour may be missing;
    everything else is exact:

    * padding (-1, +inf) in the oracle's places (min(k, |S|) neighbours);
    * every returned id is a member of S and unique in its row;
    * every distance is the exact distance of its id within REL_TOL;
    * rows ascend by distance;
    * tie-aware recall against the oracle's k-th distance >= min_recall.
    Returns that recall."""
    m, k = oi.shape
    fin = np.isfinite(od)
    assert np.array_equal(np.isfinite(gd), fin), "padding differs"
    assert np.array_equal(gi == -1, ~fin), "padding ids differ"
    hit = total = 0
    for i in range(m):
        got = gi[i][fin[i]]
        if len(got) == 0:
            continue
        assert len(set(got.tolist())) == len(got), f"query {i}: duplicate ids"
        assert set(got.tolist()) <= cand_sets[i], f"query {i}: id outside S"
        ex = np.sqrt(((X[got].astype(np.float64) - Q[i].astype(np.float64)) ** 2).sum(1))
        np.testing.assert_allclose(ex, gd[i][fin[i]], rtol=REL_TOL, atol=1e-30)
        assert np.all(np.diff(gd[i][fin[i]]) >= 0), f"query {i}: not ascending"
        kth = od[i][fin[i]][-1]
        hit += int(np.sum(ex <= kth * (1 + REL_TOL) + 1e-30))
        total += len(got)
    rec = hit / max(total, 1)
    assert rec >= min_recall, f"tie-aware recall {rec:.4f} below {min_recall}"
    return rec


def emulated_recall(X, Q, sets, oi, od, k, margin, prec):
    """Tie-aware recall of a float64 emulation of a reduced-precision screen
    (prec 1 bfloat16, 2 e4m3 with the per-row scale): the k + margin members
    of S nearest by the reduced copy's distances, re-ranked exactly, the k
    nearest kept."""
    import torch
    import bench
    Xl = bench.lowp_copy(torch.from_numpy(X), prec, torch).numpy()
    hit = total = 0
    for i, s in enumerate(sets):
        ids = np.array(sorted(s), dtype=np.int64)
        q = Q[i].astype(np.float64)
        screen = ((Xl[ids] - q) ** 2).sum(1)
        keep = ids[np.lexsort((ids, screen))[:k + margin]]
        exact = ((X[keep].astype(np.float64) - q) ** 2).sum(1)
        best = keep[np.lexsort((keep, exact))[:k]]
        fin = np.isfinite(od[i])
        if not fin.any():
            continue
        kth = od[i][fin][-1]
        dist = np.sqrt(((X[best].astype(np.float64) - q) ** 2).sum(1))
        hit += min(int((dist <= kth * (1 + 1e-6)).sum()), int(fin.sum()))
        total += int(fin.sum())
    return hit / total
