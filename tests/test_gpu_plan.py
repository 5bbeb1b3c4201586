"""GPU: query plans (the whole query captured in a CUDA graph, replayed per
batch with the batch read from a device record) give the oracle's rows
(Algorithms 3-4), for any batch size up to the plan's maximum, in every
option set a plan can fix."""
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


@pytest.fixture(scope="module")
def setup(mr):
    X, Q = workloads.mnist_like(8000, 600, seed=9)
    idx = mr.mrpt_build(torch.from_numpy(X).cuda(), 24, 6, 0.0, 3)
    mr.mrpt_add_lowp(idx)
    ref = oracle.grow_trees(X, 24, 6, float(np.float32(1 / np.sqrt(784))), 3)
    yield idx, X, Q, torch.from_numpy(Q).cuda(), ref
    idx.close()


def _oracle_rows(ref, Q, k, v, T):
    oi, od, _, oleaf, _ = oracle.query(ref, Q, k, v, T=T, want_internals=True)
    return oi, od, oracle_sets(ref, oleaf, v, T=T)


def _np(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else t


@pytest.mark.parametrize("opts", [dict(), dict(path=1), dict(precision=1, margin=8),
                                  dict(n_trees=12, chunk=64, ring=3)])
def test_plan_matches_the_oracle_for_any_batch(mr, setup, opts):
    idx, X, Q, Qd, ref = setup
    k, v = 10, 3
    oi, od, sets = _oracle_rows(ref, Q, k, v, opts.get("n_trees") or 24)
    plan = mr.Plan(idx, 512, k, v, **opts)
    for m in (1, 37, 256, 512, 5):
        ids, d = plan.run(Qd[:m])
        torch.cuda.synchronize()
        check_results(X, Q[:m], _np(ids), _np(d), oi[:m], od[:m], sets[:m])
    plan.close()


def test_plan_host_buffers_and_limits(mr, setup):
    idx, X, Q, Qd, ref = setup
    oi, od, sets = _oracle_rows(ref, Q[:50], 5, 2, 24)
    plan = mr.Plan(idx, 64, 5, 2)
    ids, d = plan.run(Q[:50].copy())
    check_results(X, Q[:50], _np(ids), _np(d), oi, od, sets)
    with pytest.raises(mr.MRPTError) as e:
        plan.run(Qd[:65])
    assert e.value.code == mr.MRPT_ERR_INVALID_ARG
    plan.close()
    with pytest.raises(mr.MRPTError):
        mr.Plan(idx, 0, 5, 2)
