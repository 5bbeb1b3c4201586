"""MRPT oracle -- TEST INFRASTRUCTURE ONLY.

A plain CPU restatement of the multiple random projection tree method with
voting (arXiv:1509.06957), written in C (``mrpt_oracle.c``) and driven from
numpy through ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library in
``paper_1509_06957_gb300``; neither imports the other.

Functions and the passages they follow:

* :func:`random_matrix` -- Algorithm 1 inner loops, Sec. II-B, Sec. II-C.
* :func:`project`       -- P = XR of Algorithm 1 / p = q^T R of Algorithm 3.
* :func:`grow_tree`, :func:`grow_trees` -- Algorithm 2 with the order-based
  median of Sec. II-A.
* :func:`route`         -- Algorithm 3.
* :func:`votes`         -- Algorithm 4 vote loop; F and S of Sec. III-A.
* :func:`knn`           -- knn(q, k, S) of Algorithm 4 (Sec. I-A metric).
* :func:`query`         -- Algorithm 4 for a batch of queries.
* :func:`brute_knn`     -- exact k-NN of Sec. I-A.

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force, hand-worked fixtures under
``tests/golden/`` and invariants stated in Sec. II-III; none is unpinned.
``tests/test_oracle_mutations.py`` checks that the pins are strong enough: it
compiles copies of ``mrpt_oracle.c`` with one planted mistake each and runs
the pins against them through ``MRPT_ORACLE_LIB`` (the path of an oracle
library to load instead of building this one).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrpt_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle_mrpt.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction of a*b+c, so only the
    explicit fmaf calls fuse).  Returns the shared-library path."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f32p = ctypes.POINTER(ctypes.c_float)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(os.environ.get("MRPT_ORACLE_LIB") or build())
            lib.orc_splitmix64.restype = ctypes.c_uint64
            lib.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.orc_random_matrix.restype = ctypes.c_int64
            lib.orc_random_matrix.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_float, ctypes.c_uint64, _i32p, _i32p, _f32p]
            lib.orc_random_matrix_fixed.restype = ctypes.c_int64
            lib.orc_random_matrix_fixed.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                    ctypes.c_float, ctypes.c_uint64, _i32p, _i32p,
                                                    _f32p]
            lib.orc_fixed_count.restype = ctypes.c_int32
            lib.orc_fixed_count.argtypes = [ctypes.c_float, ctypes.c_int32]
            lib.orc_project.restype = None
            lib.orc_project.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                        _i32p, _i32p, _f32p, _f32p]
            lib.orc_grow_tree.restype = ctypes.c_int32
            lib.orc_grow_tree.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, _f32p, _i32p, _i32p]
            lib.orc_route.restype = ctypes.c_int32
            lib.orc_route.argtypes = [_f32p, _f32p, ctypes.c_int32]
            lib.orc_votes.restype = ctypes.c_int64
            lib.orc_votes.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _i32p, _i32p,
                                      _i32p, ctypes.c_int32, _i32p, _i32p]
            lib.orc_knn.restype = ctypes.c_int32
            lib.orc_knn.argtypes = [_f32p, ctypes.c_int32, _f32p, _i32p, ctypes.c_int64,
                                    ctypes.c_int32, ctypes.c_int32, _i32p, _f32p]
            lib.orc_query.restype = ctypes.c_int32
            lib.orc_query.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, _i32p, _i32p, _f32p, _f32p, _i32p, _i32p,
                                      _f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, _i32p, _f32p, _f32p, _i32p,
                                      _i64p]
            lib.orc_brute_knn.restype = ctypes.c_int32
            lib.orc_brute_knn.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, _f32p,
                                          ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _i32p,
                                          _f32p]
            lib.orc_max_threads.restype = ctypes.c_int32
            lib.orc_max_threads.argtypes = []
            _lib = lib
    return _lib


def _p(a: np.ndarray | None, ptype):
    if a is None:
        return ctypes.cast(None, ptype)
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ptype)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def max_threads() -> int:
    return int(_load().orc_max_threads())


def splitmix64(seed: int, i: int) -> int:
    """The i-th output (0-based) of SplitMix64 started at state ``seed``."""
    return int(_load().orc_splitmix64(seed & (2**64 - 1), i))


@dataclass
class RandomMatrix:
    """Compressed-column sparse R with T*l columns (column t*l + j = tree t,
    level j), nonzeros in ascending dimension."""
    col_off: np.ndarray  # int32 [T*l + 1]
    dim: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float32 [nnz]
    d: int

    @property
    def ncols(self) -> int:
        return len(self.col_off) - 1

    def dense(self) -> np.ndarray:
        """Dense d x ncols copy (float32)."""
        R = np.zeros((self.d, self.ncols), dtype=np.float32)
        for c in range(self.ncols):
            s, e = self.col_off[c], self.col_off[c + 1]
            R[self.dim[s:e], c] = self.val[s:e]
        return R


SPARSITY_BERNOULLI = 0  # each component nonzero with probability a (Sec. II-B)
SPARSITY_FIXED = 1      # exactly ceil(a d) nonzeros per vector (Sec. II-D footnote)


def fixed_count(density: float, d: int) -> int:
    """Nonzeros per vector of the fixed-count variant: ceil(a d) in [1, d]."""
    return int(_load().orc_fixed_count(ctypes.c_float(density).value, d))


def random_matrix(T: int, l: int, d: int, density: float, seed: int,
                  sparsity: int = SPARSITY_BERNOULLI) -> RandomMatrix:
    """Sparse random vectors of Algorithm 1 (Sec. II-B, II-C); with
    sparsity=SPARSITY_FIXED, the variant in the footnote of Sec. II-D."""
    lib = _load()
    fn = lib.orc_random_matrix_fixed if sparsity == SPARSITY_FIXED else lib.orc_random_matrix
    col_off = np.zeros(T * l + 1, dtype=np.int32)
    dens = ctypes.c_float(density).value
    nnz = fn(T, l, d, dens, seed, _p(col_off, _i32p), None, None)
    dim = np.zeros(max(nnz, 1), dtype=np.int32)
    val = np.zeros(max(nnz, 1), dtype=np.float32)
    fn(T, l, d, dens, seed, _p(col_off, _i32p), _p(dim, _i32p), _p(val, _f32p))
    return RandomMatrix(col_off, dim[:nnz].copy(), val[:nnz].copy(), d)


def project(X: np.ndarray, R: RandomMatrix) -> np.ndarray:
    """P = X R with the fixed ascending-dimension fmaf chain; n x ncols."""
    X = _f32(X)
    n, d = X.shape
    assert d == R.d
    P = np.zeros((n, R.ncols), dtype=np.float32)
    dim = R.dim if len(R.dim) else np.zeros(1, np.int32)
    val = R.val if len(R.val) else np.zeros(1, np.float32)
    _load().orc_project(_p(X, _f32p), n, d, R.ncols, _p(R.col_off, _i32p), _p(dim, _i32p),
                        _p(val, _f32p), _p(P, _f32p))
    return P


def grow_tree(P: np.ndarray, col0: int, l: int):
    """Algorithm 2 on columns col0..col0+l-1 of P.  Returns
    (split[2^l - 1], leaf_off[2^l + 1], leaf_ids[n])."""
    P = _f32(P)
    n, ncols = P.shape
    L = 1 << l
    split = np.zeros(max(L - 1, 1), dtype=np.float32)
    leaf_off = np.zeros(L + 1, dtype=np.int32)
    leaf_ids = np.zeros(n, dtype=np.int32)
    rc = _load().orc_grow_tree(_p(P, _f32p), n, ncols, col0, l, _p(split, _f32p),
                               _p(leaf_off, _i32p), _p(leaf_ids, _i32p))
    if rc != 0:
        raise ValueError(f"orc_grow_tree failed ({rc}): need 1 <= 2^l <= n")
    return split[:L - 1].copy(), leaf_off, leaf_ids


@dataclass
class Index:
    """Everything Algorithm 1 returns, in flat arrays."""
    X: np.ndarray          # float32 n x d
    T: int
    l: int
    R: RandomMatrix
    P: np.ndarray          # float32 n x (T*l)
    split: np.ndarray      # float32 T x (L-1)
    leaf_off: np.ndarray   # int32 T x (L+1)
    leaf_ids: np.ndarray   # int32 T x n

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]

    @property
    def L(self) -> int:
        return 1 << self.l


def grow_trees(X: np.ndarray, T: int, l: int, density: float, seed: int,
               R: RandomMatrix | None = None, sparsity: int = SPARSITY_BERNOULLI) -> Index:
    """Algorithm 1: random matrix, projection, then one tree per t."""
    X = _f32(X)
    n, d = X.shape
    if R is None:
        R = random_matrix(T, l, d, density, seed, sparsity)
    P = project(X, R)
    L = 1 << l
    split = np.zeros((T, max(L - 1, 0)), dtype=np.float32)
    leaf_off = np.zeros((T, L + 1), dtype=np.int32)
    leaf_ids = np.zeros((T, n), dtype=np.int32)
    for t in range(T):
        s, o, i = grow_tree(P, t * l, l)
        split[t] = s
        leaf_off[t] = o
        leaf_ids[t] = i
    return Index(X, T, l, R, P, split, leaf_off, leaf_ids)


def route(p: np.ndarray, split: np.ndarray, l: int) -> int:
    """Algorithm 3 for one tree: p holds its l projections."""
    p = _f32(p)
    s = _f32(split) if len(split) else np.zeros(1, np.float32)
    return int(_load().orc_route(_p(p, _f32p), _p(s, _f32p), l))


def votes(index: Index, leaf_of_q: np.ndarray, v: int, T: int | None = None):
    """Algorithm 4's vote loop over the first T trees.  Returns
    (F[n] int32, S in emission order int32)."""
    T = index.T if T is None else T
    lq = _i32(leaf_of_q[:T])
    F = np.zeros(index.n, dtype=np.int32)
    S = np.zeros(index.n, dtype=np.int32)
    s = _load().orc_votes(T, index.n, index.L, _p(lq, _i32p),
                          _p(_i32(index.leaf_off[:T]), _i32p),
                          _p(_i32(index.leaf_ids[:T]), _i32p), v, _p(F, _i32p), _p(S, _i32p))
    return F, S[:s].copy()


def knn(X: np.ndarray, q: np.ndarray, S: np.ndarray, k: int, mode: int = 0):
    """knn(q, k, S): k nearest in S by (distance, id); (-1, inf) padding."""
    X = _f32(X)
    q = _f32(q)
    s = len(S)
    S = _i32(S) if s else np.zeros(1, np.int32)
    ids = np.zeros(k, dtype=np.int32)
    dists = np.zeros(k, dtype=np.float32)
    _load().orc_knn(_p(X, _f32p), X.shape[1], _p(q, _f32p), _p(S, _i32p), s, k, mode,
                    _p(ids, _i32p), _p(dists, _f32p))
    return ids, dists


def query(index: Index, Q: np.ndarray, k: int, v: int, mode: int = 0, nthreads: int = 0,
          T: int | None = None, want_internals: bool = False):
    """Algorithm 4 for every row of Q using the first T trees.  Returns
    (ids m x k, dists m x k) and, with want_internals, also
    (proj m x (T*l), leaf m x T, ncand m)."""
    T = index.T if T is None else T
    Q = _f32(Q)
    m = Q.shape[0]
    l = index.l
    ids = np.zeros((m, k), dtype=np.int32)
    dists = np.zeros((m, k), dtype=np.float32)
    proj = np.zeros((m, T * l), dtype=np.float32) if want_internals else None
    leaf = np.zeros((m, T), dtype=np.int32) if want_internals else None
    ncand = np.zeros(m, dtype=np.int64) if want_internals else None
    R = index.R
    ncols_used = T * l
    col_off = _i32(R.col_off[:ncols_used + 1])
    dim = R.dim if len(R.dim) else np.zeros(1, np.int32)
    val = R.val if len(R.val) else np.zeros(1, np.float32)
    split = _f32(index.split[:T]) if index.split.size else np.zeros(1, np.float32)
    rc = _load().orc_query(_p(index.X, _f32p), index.n, index.d, T, l, _p(col_off, _i32p),
                           _p(dim, _i32p), _p(val, _f32p), _p(split, _f32p),
                           _p(_i32(index.leaf_off[:T]), _i32p),
                           _p(_i32(index.leaf_ids[:T]), _i32p), _p(Q, _f32p), m, k, v, mode,
                           nthreads, _p(ids, _i32p), _p(dists, _f32p), _p(proj, _f32p),
                           _p(leaf, _i32p), _p(ncand, _i64p))
    if rc != 0:
        raise MemoryError("orc_query: allocation failed")
    if want_internals:
        return ids, dists, proj, leaf, ncand
    return ids, dists


def brute_knn(X: np.ndarray, Q: np.ndarray, k: int, nthreads: int = 0):
    """Exact k-NN over all points (Sec. I-A), double precision."""
    X = _f32(X)
    Q = _f32(Q)
    n, d = X.shape
    m = Q.shape[0]
    ids = np.zeros((m, k), dtype=np.int32)
    dists = np.zeros((m, k), dtype=np.float32)
    rc = _load().orc_brute_knn(_p(X, _f32p), n, d, _p(Q, _f32p), m, k, nthreads,
                               _p(ids, _i32p), _p(dists, _f32p))
    if rc != 0:
        raise MemoryError("orc_brute_knn: allocation failed")
    return ids, dists


def recall(found: np.ndarray, truth: np.ndarray) -> float:
    """Recall = |A n K| / k averaged over queries (Sec. I-A)."""
    m, k = truth.shape
    hits = 0
    for a, t in zip(found, truth):
        hits += len(set(a[a >= 0].tolist()) & set(t.tolist()))
    return hits / float(m * k)
