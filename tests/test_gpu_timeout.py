"""GPU: the bounded device waits report a timeout instead of hanging.

The only spin-waits of the library are the waits for a staged row in the
candidate search that copies whole rows with bulk copies (an mbarrier phase
completed by the copy): e4m3 rows of few values, and rows longer than 1,024
values (the other rows are copied per lane with cp.async and waited for per
thread, which always completes).  A testing aid,
mrpt_debug_row_wait_tries, lets those waits give up after a given number of
tries; with 0 tries every wait of the distance loop gives up at once, before
its copy has landed.  The warp must then record MRPT_ERR_TIMEOUT in the
index's status, wait with the full bound for its own copies in flight, and
exit -- no GPU fault, no hang -- and the next query must be correct."""
import numpy as np
import pytest

import oracle
import workloads
from _parity import check_lowp_results, check_results, oracle_sets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_06957_gb300 as m
    m.load_library()
    return m


@pytest.mark.parametrize("d,opts", [(64, dict(precision=2, margin=8)), (1100, dict()),
                                    (1100, dict(precision=1, margin=8))],
                         ids=["fp8-d64", "fp32-d1100", "bf16-d1100"])
def test_row_wait_that_runs_out_reports_timeout(mr, d, opts):
    X, Q = workloads.gaussian_mixture(4000, d, 200, n_centres=12, seed=17)
    T, l, v, k = 8, 4, 2, 10
    idx = mr.mrpt_build(torch.from_numpy(X).cuda(), T, l, 0.0, 6)
    mr.mrpt_add_lowp(idx, mr.MRPT_PREC_BF16)
    mr.mrpt_add_lowp(idx, mr.MRPT_PREC_FP8)
    Qd = torch.from_numpy(Q).cuda()
    ref = oracle.grow_trees(X, T, l, float(np.float32(d ** -0.5)), 6)
    oi, od, _, oleaf, _ = oracle.query(ref, Q, k, v, want_internals=True)
    sets = oracle_sets(ref, oleaf, v)

    mr.mrpt_debug_row_wait_tries(0)
    try:
        # device buffers: the call returns; the status is latched
        mr.mrpt_query_ex(idx, Qd, k, v, **opts)
        with pytest.raises(mr.MRPTError) as e:
            mr.mrpt_sync(idx)
        assert e.value.code == mr.MRPT_ERR_TIMEOUT
        # host buffers: the call itself synchronises and reports it
        with pytest.raises(mr.MRPTError) as e:
            mr.mrpt_query_ex(idx, Q, k, v, **opts)
        assert e.value.code == mr.MRPT_ERR_TIMEOUT
    finally:
        mr.mrpt_debug_row_wait_tries(-1)
    mr.mrpt_sync(idx)  # cleared

    # the context and the index are still good: the next query is the oracle's
    ids, dists = mr.mrpt_query_ex(idx, Qd, k, v, **opts)
    mr.mrpt_sync(idx)
    if opts:  # reduced-precision rows, re-ranked: exact distances, ids in S
        check_lowp_results(X, Q, ids.cpu().numpy(), dists.cpu().numpy(), oi, od, sets, min_recall=0.95)
    else:
        check_results(X, Q, ids.cpu().numpy(), dists.cpu().numpy(), oi, od, sets)
    idx.close()
