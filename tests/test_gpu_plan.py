"""GPU: query plans (the whole query captured in a CUDA graph, replayed per
batch with the batch read from a device record) give the same rows as
mrpt_query_ex, for any batch size up to the plan's maximum."""
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


@pytest.fixture(scope="module")
def setup(mr):
    X, Q = workloads.mnist_like(8000, 600, seed=9)
    idx = mr.mrpt_build(torch.from_numpy(X).cuda(), 24, 6, 0.0, 3)
    mr.mrpt_add_lowp(idx)
    yield idx, torch.from_numpy(Q).cuda()
    idx.close()


def _same(a_ids, a_d, b_ids, b_d):
    a_ids, a_d, b_ids, b_d = (t.cpu().numpy() if hasattr(t, "cpu") else t for t in (a_ids, a_d, b_ids, b_d))
    fin = np.isfinite(b_d)
    assert np.array_equal(np.isfinite(a_d), fin)
    np.testing.assert_allclose(a_d[fin], b_d[fin], rtol=REL_TOL)
    diff = (a_ids != b_ids) & fin
    if diff.any():  # only between equal distances
        np.testing.assert_allclose(a_d[diff], b_d[diff], rtol=REL_TOL)


@pytest.mark.parametrize("opts", [dict(), dict(path=1), dict(precision=1, margin=8),
                                  dict(n_trees=12, chunk=64, ring=3)])
def test_plan_matches_query_for_any_batch(mr, setup, opts):
    idx, Q = setup
    k, v = 10, 3
    plan = mr.Plan(idx, 512, k, v, **opts)
    for m in (1, 37, 256, 512, 5):
        ids, d = plan.run(Q[:m])
        rids, rd = mr.mrpt_query_ex(idx, Q[:m], k, v, **opts)
        torch.cuda.synchronize()
        _same(ids, d, rids, rd)
    plan.close()


def test_plan_host_buffers_and_limits(mr, setup):
    idx, Q = setup
    plan = mr.Plan(idx, 64, 5, 2)
    qh = Q[:50].cpu().numpy()
    ids, d = plan.run(qh)
    rids, rd = mr.mrpt_query_ex(idx, qh, 5, 2)
    _same(ids, d, rids, rd)
    with pytest.raises(mr.MRPTError) as e:
        plan.run(Q[:65])
    assert e.value.code == mr.MRPT_ERR_INVALID_ARG
    plan.close()
    with pytest.raises(mr.MRPTError):
        mr.Plan(idx, 0, 5, 2)
