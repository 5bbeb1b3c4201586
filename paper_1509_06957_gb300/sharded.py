"""Tree-sharded voting over processes (Sec. I-C: the trees are independent
and can be spread over machines).

Rank g of G builds the trees [t_g, t_g + T_g) of one seed (a contiguous
split of T; ``mrpt_build(..., tree_offset=t_g)``), so the shards together
hold exactly the trees of one T-tree index.  A query batch is answered in
three steps:

1. every rank counts the votes of its own trees for every query
   (``mrpt_vote_counts``: a sparse (id, count) list per query);
2. one exchange sends each query's lists to the rank that owns the query
   (queries are split into G contiguous ranges) -- an all-to-all of the
   per-query list lengths, then of the ids and of the counts;
3. the owner adds the lists up to F(x;q), keeps S = {x : F >= v} and runs
   the exact search on S (``mrpt_query_from_counts``).

The rows equal those of one index holding all T trees.  The exchange is
plain torch.distributed (NCCL between GPUs, gloo on CPUs); the library
computes the counts and the search.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import mrpt_build, mrpt_query_from_counts, mrpt_vote_counts


def shard_trees(T: int, rank: int, world: int) -> tuple[int, int]:
    """(first tree, trees) of rank's shard: a contiguous split of T trees,
    the first T mod world ranks one tree larger."""
    if not 0 <= rank < world or T < world:
        raise ValueError(f"need 0 <= rank < world <= T, got rank={rank} world={world} T={T}")
    base, extra = divmod(T, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def query_owners(m: int, world: int) -> list[tuple[int, int]]:
    """The query range [q0, q1) that each rank owns (contiguous, as even as
    possible)."""
    base, extra = divmod(m, world)
    out, q0 = [], 0
    for r in range(world):
        q1 = q0 + base + (1 if r < extra else 0)
        out.append((q0, q1))
        q0 = q1
    return out


def build_shard(data, T: int, l: int, density: float = 0.0, seed: int = 0, rank: int = 0,
                world: int = 1, **kw):
    """This rank's shard of a T-tree index: trees shard_trees(T, rank, world)."""
    first, count = shard_trees(T, rank, world)
    return mrpt_build(data, count, l, density, seed=seed, tree_offset=first, **kw)


def exchange_lists(nnz, ids, counts, world: int, rank: int, group=None):
    """Send every query's (id, count) list to the rank that owns the query.

    nnz [m] (int32), ids [m, cap] (int32) and counts [m, cap] (uint8) are
    this rank's lists for all m queries (row i's first nnz[i] entries), on
    the device that the group's backend reads (CUDA for NCCL, CPU for gloo).
    Returns (off [m_own + 1] int64, ids int32, counts uint8) for this rank's
    own queries: the lists of all ranks, query by query (rank order within a
    query), off[i]..off[i+1] being query i's entries."""
    dev = ids.device
    m = nnz.shape[0]
    owners = query_owners(m, world)
    nnz64 = nnz.to(torch.int64)
    # per destination: the lengths of its queries' lists, then the entries
    keep = torch.arange(ids.shape[1], device=dev)[None, :] < nnz64[:, None]
    flat_ids = ids[keep]          # row-major: query by query, so destination by destination
    flat_counts = counts[keep]
    send_items = [int(nnz64[q0:q1].sum()) for q0, q1 in owners]
    own_q0, own_q1 = owners[rank]
    m_own = own_q1 - own_q0
    # 1. lengths: rank r receives, from every source, the lengths of r's queries
    len_out = nnz64.clone()
    len_in = torch.empty(world * m_own, dtype=torch.int64, device=dev)
    dist.all_to_all_single(len_in, len_out, output_split_sizes=[m_own] * world,
                           input_split_sizes=[q1 - q0 for q0, q1 in owners], group=group)
    lens = len_in.view(world, m_own)                          # [source, own query]
    recv_items = [int(x) for x in lens.sum(1).tolist()]
    # 2. entries
    ids_in = torch.empty(sum(recv_items), dtype=torch.int32, device=dev)
    counts_in = torch.empty(sum(recv_items), dtype=torch.uint8, device=dev)
    dist.all_to_all_single(ids_in, flat_ids.contiguous(), output_split_sizes=recv_items,
                           input_split_sizes=send_items, group=group)
    dist.all_to_all_single(counts_in, flat_counts.contiguous(), output_split_sizes=recv_items,
                           input_split_sizes=send_items, group=group)
    # 3. reorder source-major -> query-major
    per_query = lens.sum(0)                                   # [own query]
    off = torch.zeros(m_own + 1, dtype=torch.int64, device=dev)
    off[1:] = torch.cumsum(per_query, 0)
    src_start = torch.zeros(world * m_own, dtype=torch.int64, device=dev)
    src_start[1:] = torch.cumsum(len_in, 0)[:-1]              # start of (source, query) in the received order
    before = torch.cumsum(lens, 0) - lens                     # entries of earlier sources of the same query
    dst_start = (off[:-1][None, :] + before).reshape(-1)      # start of (source, query) in query order
    total = int(off[-1])
    seg = torch.repeat_interleave(torch.arange(world * m_own, device=dev), len_in)
    pos_in_seg = torch.arange(total, device=dev) - src_start[seg]
    dst = dst_start[seg] + pos_in_seg
    out_ids = torch.empty(total, dtype=torch.int32, device=dev)
    out_counts = torch.empty(total, dtype=torch.uint8, device=dev)
    out_ids[dst] = ids_in
    out_counts[dst] = counts_in
    return off, out_ids, out_counts


def sharded_query(index, Q, k: int, v: int, world: int, rank: int, group=None, **opts):
    """Answer the batch Q (every rank passes the same Q, a CUDA tensor) with
    the trees of all shards.  Returns (q0, ids, dists): this rank's own
    query range [q0, q0 + len(ids)) and its k-NN rows."""
    nnz, ids, counts = mrpt_vote_counts(index, Q)
    off, cand_ids, cand_counts = exchange_lists(nnz, ids, counts, world, rank, group)
    q0, q1 = query_owners(Q.shape[0], world)[rank]
    out_ids, out_dists = mrpt_query_from_counts(index, Q[q0:q1].contiguous(), k, v, off, cand_ids,
                                                cand_counts, **opts)
    return q0, out_ids, out_dists
