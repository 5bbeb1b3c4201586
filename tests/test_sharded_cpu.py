"""Tree-sharded voting (Sec. I-C) on CPU ranks: the host side of the exchange.

Each gloo rank holds a contiguous share of the T trees.  Its per-query vote
counts come from the oracle here (the counts of trees [t0, t0 + c) are the
oracle's counts over the first t0 + c trees minus those over the first t0,
which is exact because trees are keyed by their index); the exchange must
deliver to every query's owner the lists of all ranks, so that their sum is
the oracle's F(x;q) over all T trees and S = {x : F >= v} is the oracle's
candidate set.  World sizes 2 and 3, ragged query splits."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1509_06957_gb300 import sharded  # noqa: E402


def test_tree_and_query_splits():
    for T, world in [(8, 2), (10, 3), (255, 4), (5, 5)]:
        parts = [sharded.shard_trees(T, r, world) for r in range(world)]
        assert parts[0][0] == 0
        for (a, c), (b, _) in zip(parts, parts[1:]):
            assert a + c == b
        assert sum(c for _, c in parts) == T
        assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    with pytest.raises(ValueError):
        sharded.shard_trees(2, 0, 3)
    for m, world in [(40, 2), (41, 3), (2, 4), (0, 2)]:
        own = sharded.query_owners(m, world)
        assert own[0][0] == 0 and own[-1][1] == m
        assert all(a[1] == b[0] for a, b in zip(own, own[1:]))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _shard_lists(ref, leaf, t0, c, v_unused=None):
    """Oracle counts of trees [t0, t0 + c) for every query, as padded lists."""
    import oracle
    m = leaf.shape[0]
    rows = []
    for i in range(m):
        F_hi, _ = oracle.votes(ref, leaf[i], 1, T=t0 + c)
        F_lo = oracle.votes(ref, leaf[i], 1, T=t0)[0] if t0 > 0 else np.zeros_like(F_hi)
        F = F_hi.astype(np.int64) - F_lo.astype(np.int64)
        ids = np.nonzero(F)[0]
        rows.append((ids.astype(np.int32), F[ids].astype(np.uint8)))
    cap = max(1, max(len(r[0]) for r in rows))
    nnz = np.array([len(r[0]) for r in rows], np.int32)
    ids = np.zeros((m, cap), np.int32)
    cnt = np.zeros((m, cap), np.uint8)
    for i, (a, b) in enumerate(rows):
        ids[i, :len(a)] = a
        cnt[i, :len(b)] = b
    return nnz, ids, cnt


def _rank_main(rank, world, port, q, T, v):
    import torch.distributed as dist

    import oracle
    import workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, Q = workloads.gaussian_mixture(3000, 16, 41, n_centres=9, seed=5)
        ref = oracle.grow_trees(X, T, 4, 0.25, 7)
        _, _, _, leaf, _ = oracle.query(ref, Q, 5, 1, want_internals=True)
        t0, c = sharded.shard_trees(T, rank, world)
        nnz, ids, cnt = _shard_lists(ref, leaf, t0, c)
        off, rid, rcnt = sharded.exchange_lists(torch.from_numpy(nnz), torch.from_numpy(ids),
                                                torch.from_numpy(cnt), world, rank)
        q0, q1 = sharded.query_owners(len(Q), world)[rank]
        off, rid, rcnt = off.numpy(), rid.numpy(), rcnt.numpy()
        assert len(off) == q1 - q0 + 1 and off[0] == 0 and off[-1] == len(rid) == len(rcnt)
        for j, qi in enumerate(range(q0, q1)):
            F = np.zeros(len(X), np.int64)
            np.add.at(F, rid[off[j]:off[j + 1]], rcnt[off[j]:off[j + 1]].astype(np.int64))
            F_all, S_all = oracle.votes(ref, leaf[qi], v)
            assert np.array_equal(F, F_all.astype(np.int64)), f"summed counts of query {qi}"
            assert set(np.nonzero(F >= v)[0].tolist()) == set(S_all.tolist()), f"S of query {qi}"
            # every shard sent one entry per id it voted for
            assert off[j + 1] - off[j] == sum(
                int(np.count_nonzero(_ref_counts(ref, leaf[qi], *sharded.shard_trees(T, r, world))))
                for r in range(world))
        q.put((rank, q1 - q0, "ok"))
    except Exception as e:  # reported to the parent
        q.put((rank, -1, repr(e)))
        raise
    finally:
        dist.destroy_process_group()


def _ref_counts(ref, leaf_row, t0, c):
    import oracle
    F_hi = oracle.votes(ref, leaf_row, 1, T=t0 + c)[0].astype(np.int64)
    F_lo = oracle.votes(ref, leaf_row, 1, T=t0)[0].astype(np.int64) if t0 > 0 else 0
    return F_hi - F_lo


@pytest.mark.parametrize("world,T,v", [(2, 8, 2), (3, 10, 3)])
def test_exchange_sums_to_the_oracles_votes(world, T, v):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q, T, v)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, n_own, msg in res:
        assert msg == "ok", f"rank {rank}: {msg}"
    assert sum(n for _, n, _ in res) == 41
    for p in procs:
        assert p.exitcode == 0
