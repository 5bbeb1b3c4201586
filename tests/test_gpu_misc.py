"""GPU: index save/load, the paper's fully specified "Random" workload
(unit-length N(0, I) vectors, d = 4096, Sec. IV-A), the dense (a = 1,
classic RP tree) ablation and the fixed-count sparse vectors of the
Sec. II-D footnote, each against the oracle."""
import os

import numpy as np
import pytest

import oracle
import workloads
from _parity import check_index_parity, check_results, oracle_sets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1509_06957_gb300 as m
    m.load_library()
    return m


def _check(mr, X, Q, T, l, k, v, density, seed, idx=None, sparsity=0):
    own = idx is None
    if own:
        idx = mr.mrpt_build(torch.from_numpy(X).cuda(), T, l, density, seed, sparsity=sparsity)
    ref = oracle.grow_trees(X, T, l, density, seed, sparsity=sparsity)
    check_index_parity(idx, mr, ref)
    gi, gd = mr.mrpt_query_ex(idx, torch.from_numpy(Q).cuda(), k, v)
    torch.cuda.synchronize()
    oi, od, _, oleaf, _ = oracle.query(ref, Q, k, v, want_internals=True)
    check_results(X, Q, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, oracle_sets(ref, oleaf, v))
    if own:
        idx.close()


def test_save_load_roundtrip(mr, tmp_path):
    X, Q = workloads.gaussian_mixture(3000, 20, 30, n_centres=9, seed=3)
    idx = mr.mrpt_build(X, 7, 5, 0.3, 12)
    path = str(tmp_path / "index.mrpt")
    mr.mrpt_save(idx, path)
    idx2 = mr.mrpt_load(path)
    for what in ("R_COL_OFF", "R_DIM", "R_VAL", "SPLIT", "LEAF_OFF", "LEAF_IDS", "DATA"):
        assert np.array_equal(mr.mrpt_export(idx, what), mr.mrpt_export(idx2, what)), what
    a = mr.mrpt_query(idx, Q, 10, 2)
    b = mr.mrpt_query(idx2, Q, 10, 2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    _check(mr, X, Q, 7, 5, 10, 2, 0.3, 12, idx=idx2)
    # damaged files are refused
    blob = open(path, "rb").read()
    open(path, "wb").write(blob[: len(blob) // 2])
    with pytest.raises(mr.MRPTError) as e:
        mr.mrpt_load(path)
    assert e.value.code == mr.MRPT_ERR_INVALID_ARG
    open(path, "wb").write(b"NOTANIDX" + blob[8:])
    with pytest.raises(mr.MRPTError):
        mr.mrpt_load(path)
    idx.close()
    idx2.close()


def test_random_unit_vectors_d4096(mr):
    """The paper's "Random" set shape: unit-length N(0, I) vectors, d = 4096."""
    X, Q = workloads.unit_gaussian(4000, 4096, 12, seed=5)
    _check(mr, X, Q, 6, 5, 10, 2, float(np.float32(4096 ** -0.5)), 1)


def test_dense_classic_rp_trees(mr):
    """a = 1: classic dense RP trees with one vector per level."""
    X, Q = workloads.gaussian_mixture(2000, 48, 20, n_centres=10, seed=6)
    _check(mr, X, Q, 5, 4, 10, 2, 1.0, 4)


@pytest.mark.parametrize("d,density", [(784, 0.0), (128, 0.0), (37, 0.3)])
def test_fixed_count_sparse_vectors(mr, d, density):
    """Exactly ceil(a d) nonzeros per vector (mrpt_build_ex, sparsity
    FIXED): random matrix, splits, leaves and answers equal the oracle's."""
    if d == 784:
        X, Q = workloads.mnist_like(3000, 40, seed=4)
    else:
        X, Q = workloads.gaussian_mixture(2500, d, 40, n_centres=12, seed=4)
    a = density if density > 0 else float(np.float32(1.0 / np.sqrt(d)))
    idx = mr.mrpt_build(torch.from_numpy(X).cuda(), 12, 6, a, 21, sparsity=mr.MRPT_SPARSITY_FIXED)
    k_nz = oracle.fixed_count(a, d)
    assert np.all(np.diff(mr.mrpt_export(idx, "R_COL_OFF")) == k_nz)
    _check(mr, X, Q, 12, 6, 10, 3, a, 21, idx=idx, sparsity=oracle.SPARSITY_FIXED)
    idx.close()


def test_unknown_sparsity_is_rejected(mr):
    X = np.random.default_rng(0).standard_normal((64, 6)).astype(np.float32)
    with pytest.raises(mr.MRPTError) as e:
        mr.mrpt_build(X, 2, 2, 0.5, 0, sparsity=7)
    assert e.value.code == mr.MRPT_ERR_INVALID_ARG


def test_host_buffers_large_batch_chunked_upload(mr):
    """Host queries in a batch of at least 8,192 are copied in chunks, each
    routed as soon as it arrives; the rows equal the oracle's, as do those
    of the same batch in device buffers."""
    X, Q = workloads.mnist_like(6000, 9000, seed=6)
    idx = mr.mrpt_build(torch.from_numpy(X).cuda(), 16, 5, 0.0, 3)
    ref = oracle.grow_trees(X, 16, 5, float(np.float32(1 / np.sqrt(784))), 3)
    check_index_parity(idx, mr, ref)
    oi, od, _, oleaf, _ = oracle.query(ref, Q, 10, 3, want_internals=True)
    sets = oracle_sets(ref, oleaf, 3)
    ids_d, dists_d = mr.mrpt_query(idx, torch.from_numpy(Q).cuda(), 10, 3)
    ids_h, dists_h = mr.mrpt_query(idx, Q, 10, 3)
    assert isinstance(ids_h, np.ndarray)
    check_results(X, Q, ids_h, dists_h, oi, od, sets)
    check_results(X, Q, ids_d.cpu().numpy(), dists_d.cpu().numpy(), oi, od, sets)
    mr.mrpt_add_lowp(idx, mr.MRPT_PREC_BF16)
    a = mr.mrpt_query_ex(idx, torch.from_numpy(Q).cuda(), 10, 3, precision=mr.MRPT_PREC_BF16, margin=8)
    b = mr.mrpt_query_ex(idx, Q, 10, 3, precision=mr.MRPT_PREC_BF16, margin=8)
    check_results(X, Q, b[0], b[1], oi, od, sets)
    check_results(X, Q, a[0].cpu().numpy(), a[1].cpu().numpy(), oi, od, sets)
    idx.close()


@pytest.mark.parametrize("host", [False, True], ids=["device", "host"])
def test_n_cand_out_alone_is_the_oracle_count(mr, host):
    """|S| of every query through n_cand_out alone (no m x n debug buffers),
    device and host buffers, equals the oracle's count, and the rows are the
    oracle's."""
    X, Q = workloads.gaussian_mixture(5000, 40, 300, n_centres=10, seed=21)
    T, l, v, k = 12, 5, 3, 8
    dens = float(np.float32(40 ** -0.5))
    idx = mr.mrpt_build(torch.from_numpy(X).cuda(), T, l, dens, 4)
    ref = oracle.grow_trees(X, T, l, dens, 4)
    oi, od, _, oleaf, oncand = oracle.query(ref, Q, k, v, want_internals=True)
    if host:
        ncand = np.full(len(Q), -7, np.int64)
        gi, gd = mr.mrpt_query_ex(idx, Q, k, v, n_cand_out=ncand)
    else:
        ncand_d = torch.full((len(Q),), -7, dtype=torch.int64, device="cuda")
        gi, gd = mr.mrpt_query_ex(idx, torch.from_numpy(Q).cuda(), k, v, n_cand_out=ncand_d)
        torch.cuda.synchronize()
        ncand, gi, gd = ncand_d.cpu().numpy(), gi.cpu().numpy(), gd.cpu().numpy()
    assert np.array_equal(ncand, oncand)
    check_results(X, Q, gi, gd, oi, od, oracle_sets(ref, oleaf, v))
    idx.close()
