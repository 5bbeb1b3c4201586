"""mrpt_query_noalloc: the query for callers that may not allocate device
memory (a serving loop with a latency budget, where cudaMalloc/cudaFree can
synchronise the device, or a process whose device memory belongs to another
framework's pool).  On consecutive calls that reuse its one fixed scratch
array it must give the oracle's rows (Algorithms 3-4) -- the rows mrpt_query
gives -- while every device allocation of the library is made to fail, and it
must refuse batches larger than that array.  Collected last on purpose (file
name), so that a run stopping at the first failure has already run every
other test."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from _parity import check_results, oracle_sets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_06957_gb300 as m
    m.load_library()
    return m


def _noalloc(mr, idx, Q, k, v, n_trees=0):
    """Call the entry point through the C ABI with device buffers."""
    lib = mr.load_library()
    m = Q.shape[0]
    ids = torch.full((m, k), -7, dtype=torch.int32, device=Q.device)
    dists = torch.full((m, k), float("nan"), dtype=torch.float32, device=Q.device)
    lib.mrpt_set_stream(idx.handle, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    rc = lib.mrpt_query_noalloc(idx.handle, ctypes.c_void_p(Q.data_ptr()), m, k, v, n_trees,
                                ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dists.data_ptr()))
    torch.cuda.synchronize()
    return rc, ids.cpu().numpy(), dists.cpu().numpy()


def test_noalloc_matches_the_oracle_on_consecutive_calls(mr):
    X, Q = workloads.mnist_like(5000, 300, seed=5)
    dev = torch.device("cuda:0")
    # a fresh index: none of its query scratch has been allocated yet
    idx = mr.mrpt_build(torch.from_numpy(X).to(dev), 24, 5, 0.0, seed=2)
    ref = oracle.grow_trees(X, 24, 5, float(np.float32(1 / np.sqrt(784))), 2)
    Qd = torch.from_numpy(Q).to(dev)
    for k, v, n_trees in [(10, 3, 0), (100, 2, 16)]:
        oi, od, _, oleaf, _ = oracle.query(ref, Q, k, v, T=n_trees or 24, want_internals=True)
        sets = oracle_sets(ref, oleaf, v, T=n_trees or 24)
        for call in range(2):
            # the next device allocation of the library fails: the calls
            # below succeed only because they make none
            mr.mrpt_debug_fail_alloc_after(0)
            try:
                rc, ids, dists = _noalloc(mr, idx, Qd, k, v, n_trees)
            finally:
                mr.mrpt_debug_fail_alloc_after(-1)
            assert rc == 0, mr.mrpt_last_error()
            check_results(X, Q, ids, dists, oi, od, sets)
        # the allocating entry point gives the same rows
        ref_ids, ref_d = mr.mrpt_query(idx, Qd, k, v, n_trees=n_trees)
        check_results(X, Q, ref_ids.cpu().numpy(), ref_d.cpu().numpy(), oi, od, sets)
    # allocation works again afterwards
    mr.mrpt_query(idx, Qd[:4], 5, 1)
    idx.close()


def test_noalloc_rejects_batches_beyond_its_scratch(mr):
    X, _ = workloads.gaussian_mixture(2000, 16, 1, seed=1)
    dev = torch.device("cuda:0")
    idx = mr.mrpt_build(torch.from_numpy(X).to(dev), 8, 4, 0.0, seed=1)
    m = mr.MRPT_NOALLOC_MAX_LEAF_ENTRIES // 8 + 1
    Q = torch.zeros((m, 16), dtype=torch.float32, device=dev)
    rc, _, _ = _noalloc(mr, idx, Q, 5, 2)
    assert rc == mr.MRPT_ERR_INVALID_ARG
    assert "exceeds" in mr.mrpt_last_error()
    # the largest batch that fits is accepted
    rc, ids, _ = _noalloc(mr, idx, Q[: m - 1], 5, 2)
    assert rc == 0, mr.mrpt_last_error()
    # host buffers are refused (staging them would allocate)
    lib = mr.load_library()
    qh = np.zeros((4, 16), np.float32)
    oi = np.zeros((4, 5), np.int32)
    od = np.zeros((4, 5), np.float32)
    rc = lib.mrpt_query_noalloc(idx.handle, ctypes.c_void_p(qh.ctypes.data), 4, 5, 2, 0,
                                ctypes.c_void_p(oi.ctypes.data), ctypes.c_void_p(od.ctypes.data))
    assert rc == mr.MRPT_ERR_INVALID_ARG
    idx.close()
