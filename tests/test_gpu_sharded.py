"""GPU: tree-sharded voting (Sec. I-C) through the C ABI, on one GPU.

Shards are indexes built with a tree offset.  Checked against the oracle:
- a shard's random matrix, splits and leaves are the full index's trees
  t0 .. t0+c-1 (trees are keyed by their index);
- mrpt_vote_counts gives, per query, exactly the ids with a vote among the
  shard's trees and their counts (the oracle's counts over the first t0 + c
  trees minus those over the first t0), ids ascending;
- mrpt_query_from_counts on the shards' lists concatenated per query gives
  the oracle's rows of the full T-tree index, in float32 and bfloat16;
- a saved and loaded shard keeps its tree offset.
The exchange between processes is covered on CPU ranks
(tests/test_sharded_cpu.py)."""
import numpy as np
import pytest

import oracle
import workloads
from _parity import check_results, oracle_sets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T, L, V, K, SEED = 12, 5, 3, 10, 17


@pytest.fixture(scope="module")
def mr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_06957_gb300 as m
    m.load_library()
    return m


@pytest.fixture(scope="module")
def case(mr):
    from paper_1509_06957_gb300 import sharded
    X, Q = workloads.gaussian_mixture(6000, 40, 300, n_centres=20, seed=23)
    dens = float(np.float32(40 ** -0.5))
    ref = oracle.grow_trees(X, T, L, dens, SEED)
    oi, od, _, oleaf, _ = oracle.query(ref, Q, K, V, want_internals=True)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    shards = [sharded.build_shard(Xd, T, L, dens, SEED, rank=r, world=3) for r in range(3)]
    yield dict(X=X, Q=Q, Qd=Qd, ref=ref, oi=oi, od=od, oleaf=oleaf, shards=shards, sharded=sharded)
    for s in shards:
        s.close()


def test_shards_hold_the_full_index_trees(mr, case):
    ref = case["ref"]
    for r, idx in enumerate(case["shards"]):
        t0, c = case["sharded"].shard_trees(T, r, 3)
        assert idx.tree_offset == t0 and idx.T == c
        col = ref.R.col_off
        lo, hi = col[t0 * L], col[(t0 + c) * L]
        assert np.array_equal(mr.mrpt_export(idx, "R_COL_OFF"), col[t0 * L:(t0 + c) * L + 1] - lo)
        assert np.array_equal(mr.mrpt_export(idx, "R_DIM"), ref.R.dim[lo:hi])
        assert np.array_equal(mr.mrpt_export(idx, "R_VAL").view(np.uint32), ref.R.val[lo:hi].view(np.uint32))
        assert np.array_equal(mr.mrpt_export(idx, "SPLIT").view(np.uint32),
                              ref.split[t0:t0 + c].view(np.uint32))
        assert np.array_equal(mr.mrpt_export(idx, "LEAF_IDS"), ref.leaf_ids[t0:t0 + c])


def _shard_counts(ref, leaf_row, t0, c):
    F_hi = oracle.votes(ref, leaf_row, 1, T=t0 + c)[0].astype(np.int64)
    F_lo = oracle.votes(ref, leaf_row, 1, T=t0)[0].astype(np.int64) if t0 > 0 else 0
    return F_hi - F_lo


def test_vote_counts_are_the_shards_votes(mr, case):
    for r, idx in enumerate(case["shards"]):
        t0, c = case["sharded"].shard_trees(T, r, 3)
        nnz, ids, counts = mr.mrpt_vote_counts(idx, case["Qd"])
        torch.cuda.synchronize()
        nnz, ids, counts = nnz.cpu().numpy(), ids.cpu().numpy(), counts.cpu().numpy()
        for i in range(0, len(case["Q"]), 7):
            F = _shard_counts(case["ref"], case["oleaf"][i], t0, c)
            want = np.nonzero(F)[0]
            got = ids[i, :nnz[i]]
            assert np.array_equal(got, want), f"shard {r}, query {i}: ids"
            assert np.array_equal(counts[i, :nnz[i]], F[want].astype(np.uint8)), f"shard {r}, query {i}"


@pytest.mark.parametrize("opts", [dict(), dict(precision=1, margin=8)], ids=["fp32", "bf16"])
def test_query_from_summed_counts_is_the_full_index(mr, case, opts):
    lists = [mr.mrpt_vote_counts(idx, case["Qd"]) for idx in case["shards"]]
    torch.cuda.synchronize()
    m = len(case["Q"])
    per_q_ids, per_q_cnt, off = [], [], [0]
    host = [(a.cpu().numpy(), b.cpu().numpy(), c.cpu().numpy()) for a, b, c in lists]
    for i in range(m):
        for nnz, ids, cnt in host:
            per_q_ids.append(ids[i, :nnz[i]])
            per_q_cnt.append(cnt[i, :nnz[i]])
        off.append(off[-1] + sum(int(h[0][i]) for h in host))
    dev = case["Qd"].device
    off_t = torch.tensor(off, dtype=torch.int64, device=dev)
    ids_t = torch.from_numpy(np.concatenate(per_q_ids).astype(np.int32)).to(dev)
    cnt_t = torch.from_numpy(np.concatenate(per_q_cnt).astype(np.uint8)).to(dev)
    owner = case["shards"][1]              # any shard holds the data for the search
    if opts:
        mr.mrpt_add_lowp(owner)
    gi, gd = mr.mrpt_query_from_counts(owner, case["Qd"], K, V, off_t, ids_t, cnt_t, **opts)
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    if opts:
        from _parity import check_lowp_results
        check_lowp_results(case["X"], case["Q"], gi, gd, case["oi"], case["od"],
                           oracle_sets(case["ref"], case["oleaf"], V), min_recall=0.99)
    else:
        check_results(case["X"], case["Q"], gi, gd, case["oi"], case["od"],
                      oracle_sets(case["ref"], case["oleaf"], V))


def test_empty_lists_pad_every_row(mr, case):
    dev = case["Qd"].device
    off = torch.zeros(5, dtype=torch.int64, device=dev)
    e_i = torch.empty(0, dtype=torch.int32, device=dev)
    e_c = torch.empty(0, dtype=torch.uint8, device=dev)
    gi, gd = mr.mrpt_query_from_counts(case["shards"][0], case["Qd"][:4], K, 1, off, e_i, e_c)
    torch.cuda.synchronize()
    assert (gi.cpu().numpy() == -1).all() and np.isinf(gd.cpu().numpy()).all()


def test_vote_count_capacity_is_checked(mr, case):
    import ctypes
    idx = case["shards"][0]
    lib = mr.load_library()
    Qd = case["Qd"][:2]
    need = mr.vote_count_capacity(idx)
    buf = torch.empty((2, need), dtype=torch.int32, device=Qd.device)
    cnt = torch.empty((2, need), dtype=torch.uint8, device=Qd.device)
    nnz = torch.empty(2, dtype=torch.int32, device=Qd.device)
    rc = lib.mrpt_vote_counts(idx.handle, ctypes.c_void_p(Qd.data_ptr()), 2, 0, need - 1,
                              ctypes.c_void_p(nnz.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                              ctypes.c_void_p(cnt.data_ptr()))
    assert rc == mr.MRPT_ERR_INVALID_ARG and str(need) in mr.mrpt_last_error()


def test_shard_save_load_keeps_the_offset(mr, case, tmp_path):
    idx = case["shards"][2]
    path = str(tmp_path / "shard.mrpt")
    mr.mrpt_save(idx, path)
    back = mr.mrpt_load(path)
    assert back.tree_offset == idx.tree_offset and back.T == idx.T
    assert np.array_equal(mr.mrpt_export(back, "SPLIT"), mr.mrpt_export(idx, "SPLIT"))
    a = [t.cpu().numpy() for t in mr.mrpt_vote_counts(idx, case["Qd"][:16])]
    b = [t.cpu().numpy() for t in mr.mrpt_vote_counts(back, case["Qd"][:16])]
    assert np.array_equal(a[0], b[0])
    for i in range(16):
        n_i = a[0][i]
        assert np.array_equal(a[1][i, :n_i], b[1][i, :n_i]) and np.array_equal(a[2][i, :n_i], b[2][i, :n_i])
    back.close()
