"""mrpt_query_noalloc: the query for callers that may not allocate device
memory (a serving loop with a latency budget, where cudaMalloc/cudaFree can
synchronise the device, or a process whose device memory belongs to another
framework's pool).  It must give what mrpt_query gives, on consecutive
calls that reuse its one fixed scratch array, and refuse batches larger
than that array.  Collected last on purpose (file name), so that a run
stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import workloads
from _parity import REL_TOL

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


def test_noalloc_matches_mrpt_query_on_consecutive_calls(mr):
    X, Q = workloads.mnist_like(5000, 300, seed=5)
    dev = torch.device("cuda:0")
    idx = mr.mrpt_build(torch.from_numpy(X).to(dev), 24, 5, 0.0, seed=2)
    Qd = torch.from_numpy(Q).to(dev)
    for k, v, n_trees in [(10, 3, 0), (100, 2, 16)]:
        ref_ids, ref_d = mr.mrpt_query(idx, Qd, k, v, n_trees=n_trees)
        ref_ids, ref_d = ref_ids.cpu().numpy(), ref_d.cpu().numpy()
        for call in range(2):
            rc, ids, dists = _noalloc(mr, idx, Qd, k, v, n_trees)
            assert rc == 0, mr.mrpt_last_error()
            fin = np.isfinite(ref_d)
            assert np.array_equal(np.isfinite(dists), fin)
            np.testing.assert_allclose(dists[fin], ref_d[fin], rtol=REL_TOL, atol=1e-30)
            same = (ids == ref_ids) | ~fin
            # ids may differ only between equal distances
            if not same.all():
                np.testing.assert_allclose(dists[~same], ref_d[~same], rtol=REL_TOL)
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
