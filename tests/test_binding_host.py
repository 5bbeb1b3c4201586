"""CPU: the Python binding rejects buffers the C ABI would misread.

The C entry points take bare pointers and trust the sizes passed with them,
so the binding checks every matrix it hands over: queries must be m x d for
an index of dimension d, output buffers m x k of the right type, everything
contiguous.  These checks run before any library call, so they are tested
here with a stand-in index that carries only its sizes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_1509_06957_gb300 as mr  # noqa: E402


class _Calls:
    """Stands in for the loaded library: any call is a test failure."""

    def __getattr__(self, name):
        raise AssertionError(f"{name} was called with invalid arguments")


@pytest.fixture
def index(monkeypatch):
    monkeypatch.setattr(mr, "load_library", lambda build_if_missing=True: _Calls())
    idx = object.__new__(mr.Index)
    idx._h = None
    idx.n, idx.d, idx.T, idx.l = 100, 8, 4, 3
    return idx


@pytest.mark.parametrize("Q", [
    np.zeros((5, 7), np.float32),            # wrong dimension
    np.zeros(8, np.float32),                 # one query as a vector
    np.zeros((2, 5, 8), np.float32),         # not a matrix
    torch.zeros((5, 9)),                     # wrong dimension, torch
])
def test_queries_must_be_m_by_d(index, Q):
    with pytest.raises(ValueError, match="queries"):
        mr.mrpt_query_ex(index, Q, 3, 1)


@pytest.mark.parametrize("name,ids,dists", [
    ("out_ids", np.zeros((5, 2), np.int32), np.zeros((5, 3), np.float32)),
    ("out_ids", np.zeros((5, 3), np.int64), np.zeros((5, 3), np.float32)),
    ("out_ids", np.zeros((3, 5), np.int32).T, np.zeros((5, 3), np.float32)),
    ("out_dists", np.zeros((5, 3), np.int32), np.zeros((4, 3), np.float32)),
    ("out_dists", np.zeros((5, 3), np.int32), np.zeros((5, 3), np.float64)),
    ("out_dists", torch.zeros((5, 3), dtype=torch.int32), torch.zeros((3, 5)).t()),
])
def test_output_buffers_must_be_m_by_k(index, name, ids, dists):
    Q = np.zeros((5, 8), np.float32)
    with pytest.raises(ValueError, match=name):
        mr.mrpt_query_ex(index, Q, 3, 1, out_ids=ids, out_dists=dists)


@pytest.mark.parametrize("ncand", [
    np.zeros(4, np.int64),                    # too short
    np.zeros(5, np.int32),                    # wrong type
    np.zeros((5, 1), np.int64),               # not a vector
    np.zeros(10, np.int64)[::2],              # not contiguous
])
def test_n_cand_out_must_be_m_int64(index, ncand):
    Q = np.zeros((5, 8), np.float32)
    with pytest.raises(ValueError, match="n_cand_out"):
        mr.mrpt_query_ex(index, Q, 3, 1, n_cand_out=ncand)


def test_noalloc_checks_its_buffers(index):
    Q = torch.zeros((5, 8))
    ok_i, ok_d = torch.zeros((5, 3), dtype=torch.int32), torch.zeros((5, 3))
    with pytest.raises(ValueError, match="queries"):
        mr.mrpt_query_noalloc(index, torch.zeros((5, 8), dtype=torch.float64), 3, 1, ok_i, ok_d)
    with pytest.raises(ValueError, match="queries"):
        mr.mrpt_query_noalloc(index, torch.zeros((5, 6)), 3, 1, ok_i, ok_d)
    with pytest.raises(ValueError, match="out_ids"):
        mr.mrpt_query_noalloc(index, Q, 4, 1, ok_i, ok_d)


def test_plan_run_checks_its_buffers(index):
    plan = object.__new__(mr.Plan)
    plan.index, plan.k, plan._lib, plan._h = index, 3, _Calls(), None
    with pytest.raises(ValueError, match="queries"):
        plan.run(np.zeros((5, 9), np.float32))
    with pytest.raises(ValueError, match="out_dists"):
        plan.run(np.zeros((5, 8), np.float32), np.zeros((5, 3), np.int32), np.zeros((5, 2), np.float32))


def test_build_data_must_be_a_matrix(monkeypatch):
    monkeypatch.setattr(mr, "load_library", lambda build_if_missing=True: _Calls())
    with pytest.raises(ValueError, match="data"):
        mr.mrpt_build(np.zeros(16, np.float32), 2, 1)


def test_non_contiguous_pointer_is_refused():
    with pytest.raises(ValueError, match="contiguous"):
        mr._ptr(np.zeros((4, 6), np.float32)[:, ::2])
    with pytest.raises(ValueError, match="contiguous"):
        mr._ptr(torch.zeros((4, 6))[:, ::2])
