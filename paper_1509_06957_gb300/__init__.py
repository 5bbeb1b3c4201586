"""GB300 (sm_103a) multiple random projection trees with voting.

Thin Python binding of the C ABI in ``include/mrpt.h`` (library
``_build/libmrpt.so``, built from ``csrc/`` by :mod:`.build`).  Every step
of index construction and of the query runs in the library's CUDA kernels;
this module only marshals arguments: it passes raw pointers of torch tensors
(device memory, current stream) or numpy arrays (host memory) and turns
error codes into exceptions.  There is no CPU fallback: if the library is
missing or a call fails, an exception is raised.

Names follow the C ABI: :func:`mrpt_build`, :func:`mrpt_query`,
:func:`mrpt_query_ex`, :func:`mrpt_free`, :func:`mrpt_last_error`,
:func:`mrpt_set_stream`, :func:`mrpt_sync`, :func:`mrpt_info`,
:func:`mrpt_export`, plus the :class:`Index` handle.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

MRPT_OK = 0
MRPT_ERR_INVALID_ARG = -1
MRPT_ERR_NONFINITE_INPUT = -2
MRPT_ERR_OOM = -3
MRPT_ERR_CUDA = -4
MRPT_ERR_TIMEOUT = -5
MRPT_ERR_UNSUPPORTED = -6

MRPT_MAX_TREES = 255
MRPT_MAX_DEPTH = 24
MRPT_MAX_K = 256
MRPT_MAX_DIM = 32768

EXPORT = {
    "R_COL_OFF": (0, np.int32),
    "R_DIM": (1, np.int32),
    "R_VAL": (2, np.float32),
    "SPLIT": (3, np.float32),
    "LEAF_OFF": (4, np.int32),
    "LEAF_IDS": (5, np.int32),
    "DATA": (6, np.float32),
}

#: every symbol include/mrpt.h declares
ABI_SYMBOLS = (
    "mrpt_build", "mrpt_query", "mrpt_query_ex", "mrpt_free", "mrpt_last_error",
    "mrpt_set_stream", "mrpt_sync", "mrpt_info", "mrpt_export_size", "mrpt_export",
    "mrpt_debug_fail_alloc_after", "mrpt_query_noalloc", "mrpt_add_lowp",
    "mrpt_plan_create", "mrpt_plan_run", "mrpt_plan_free", "mrpt_save", "mrpt_load",
    "mrpt_build_ex", "mrpt_debug_row_wait_tries", "mrpt_vote_counts", "mrpt_query_from_counts",
)
MRPT_SPARSITY_BERNOULLI = 0
MRPT_SPARSITY_FIXED = 1
MRPT_PREC_FP32 = 0
MRPT_PREC_BF16 = 1
MRPT_PREC_FP8 = 2
MRPT_VOTE_COUNTERS = 1
MRPT_VOTE_HASH = 2
MRPT_VOTE_HASH_ENTRIES = 24576
MRPT_NOALLOC_MAX_LEAF_ENTRIES = 1048512


class MRPTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class BuildOpts(ctypes.Structure):
    _fields_ = [("sparsity", ctypes.c_int32), ("tree_offset", ctypes.c_int32)]


class QueryOpts(ctypes.Structure):
    _fields_ = [
        ("n_trees", ctypes.c_int32),
        ("path", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("margin", ctypes.c_int32),
        ("chunk", ctypes.c_int32),
        ("ring", ctypes.c_int32),
        ("proj", ctypes.c_void_p),
        ("leaf", ctypes.c_void_p),
        ("votes", ctypes.c_void_p),
        ("n_cand", ctypes.c_void_p),
        ("cand", ctypes.c_void_p),
        ("cand_cap", ctypes.c_int64),
        ("stage_ms", ctypes.POINTER(ctypes.c_float)),
        ("vote_table", ctypes.c_int32),
    ]


class IndexInfo(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("d", ctypes.c_int32),
        ("T", ctypes.c_int32),
        ("l", ctypes.c_int32),
        ("density", ctypes.c_float),
        ("seed", ctypes.c_uint64),
        ("nnz", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64),
        ("tree_offset", ctypes.c_int32),
    ]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libmrpt.so (building it first when it is missing or stale and
    nvcc is available).  Raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build_library()
        if not os.path.exists(path):
            raise RuntimeError(f"libmrpt.so not found at {path}; run paper_1509_06957_gb300.build")
        lib = ctypes.CDLL(path)
        vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        lib.mrpt_build.restype = ctypes.c_int
        lib.mrpt_build.argtypes = [vp, i64, i32, i32, i32, f32, ctypes.c_uint64,
                                   ctypes.POINTER(vp)]
        lib.mrpt_build_ex.restype = ctypes.c_int
        lib.mrpt_build_ex.argtypes = [vp, i64, i32, i32, i32, f32, ctypes.c_uint64,
                                      ctypes.POINTER(BuildOpts), ctypes.POINTER(vp)]
        lib.mrpt_query.restype = ctypes.c_int
        lib.mrpt_query.argtypes = [vp, vp, i64, i32, i32, vp, vp]
        lib.mrpt_query_ex.restype = ctypes.c_int
        lib.mrpt_query_ex.argtypes = [vp, vp, i64, i32, i32, ctypes.POINTER(QueryOpts), vp, vp]
        lib.mrpt_free.restype = ctypes.c_int
        lib.mrpt_free.argtypes = [vp]
        lib.mrpt_last_error.restype = ctypes.c_char_p
        lib.mrpt_last_error.argtypes = []
        lib.mrpt_set_stream.restype = ctypes.c_int
        lib.mrpt_set_stream.argtypes = [vp, vp]
        lib.mrpt_sync.restype = ctypes.c_int
        lib.mrpt_sync.argtypes = [vp]
        lib.mrpt_info.restype = ctypes.c_int
        lib.mrpt_info.argtypes = [vp, ctypes.POINTER(IndexInfo)]
        lib.mrpt_export_size.restype = ctypes.c_int64
        lib.mrpt_export_size.argtypes = [vp, i32]
        lib.mrpt_export.restype = ctypes.c_int
        lib.mrpt_export.argtypes = [vp, i32, vp, i64]
        lib.mrpt_debug_fail_alloc_after.restype = ctypes.c_int
        lib.mrpt_debug_fail_alloc_after.argtypes = [i32]
        lib.mrpt_debug_row_wait_tries.restype = ctypes.c_int
        lib.mrpt_debug_row_wait_tries.argtypes = [i32]
        lib.mrpt_vote_counts.restype = ctypes.c_int
        lib.mrpt_vote_counts.argtypes = [vp, vp, i64, i32, i64, vp, vp, vp]
        lib.mrpt_query_from_counts.restype = ctypes.c_int
        lib.mrpt_query_from_counts.argtypes = [vp, vp, i64, i32, i32, vp, vp, vp, ctypes.POINTER(QueryOpts),
                                               vp, vp]
        lib.mrpt_plan_create.restype = ctypes.c_int
        lib.mrpt_plan_create.argtypes = [vp, i64, i32, i32, ctypes.POINTER(QueryOpts),
                                         ctypes.POINTER(vp)]
        lib.mrpt_plan_run.restype = ctypes.c_int
        lib.mrpt_plan_run.argtypes = [vp, vp, i64, vp, vp]
        lib.mrpt_plan_free.restype = ctypes.c_int
        lib.mrpt_plan_free.argtypes = [vp]
        lib.mrpt_save.restype = ctypes.c_int
        lib.mrpt_save.argtypes = [vp, ctypes.c_char_p]
        lib.mrpt_load.restype = ctypes.c_int
        lib.mrpt_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(vp)]
        lib.mrpt_add_lowp.restype = ctypes.c_int
        lib.mrpt_add_lowp.argtypes = [vp, i32]
        lib.mrpt_query_noalloc.restype = ctypes.c_int
        lib.mrpt_query_noalloc.argtypes = [vp, vp, i64, i32, i32, i32, vp, vp]
        _lib = lib
        return lib


def mrpt_last_error() -> str:
    return load_library().mrpt_last_error().decode(errors="replace")


def _check(rc: int) -> None:
    if rc != MRPT_OK:
        raise MRPTError(rc, mrpt_last_error())


# ------------------------------------------------------------ marshalling --

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """Raw pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous (row-major, tightly packed)")
        return ctypes.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous (row-major, tightly packed)")
    return ctypes.c_void_p(x.ctypes.data)


_DTYPE_NAMES = {np.float32: "float32", np.int32: "int32"}


def _check_matrix(name: str, x, rows: int, cols: int, dtype) -> None:
    """The C ABI takes a bare pointer and trusts the sizes it is given, so a
    buffer of another shape or type would be read or written out of bounds:
    x must be a contiguous rows x cols matrix of `dtype`."""
    shape = tuple(x.shape)
    if _is_torch(x):
        import torch
        ok_type = x.dtype == {np.float32: torch.float32, np.int32: torch.int32}[dtype]
        contiguous = x.is_contiguous()
    else:
        ok_type = np.dtype(x.dtype) == np.dtype(dtype)
        contiguous = bool(x.flags["C_CONTIGUOUS"])
    if shape != (rows, cols):
        raise ValueError(f"{name} must have shape ({rows}, {cols}), got {shape}")
    if not ok_type:
        raise ValueError(f"{name} must be {_DTYPE_NAMES[dtype]}, got {x.dtype}")
    if not contiguous:
        raise ValueError(f"{name} must be contiguous (row-major, tightly packed)")


def _check_vector(name: str, x, size: int, dtype) -> None:
    """x must be a contiguous vector of `size` elements of `dtype` (the C ABI
    writes that many)."""
    if _is_torch(x):
        import torch
        ok_type = x.dtype == {np.int64: torch.int64, np.int32: torch.int32}[dtype]
        contiguous = x.is_contiguous()
    else:
        ok_type = np.dtype(x.dtype) == np.dtype(dtype)
        contiguous = bool(x.flags["C_CONTIGUOUS"])
    if tuple(x.shape) != (size,):
        raise ValueError(f"{name} must have shape ({size},), got {tuple(x.shape)}")
    if not ok_type:
        raise ValueError(f"{name} must be {np.dtype(dtype).name}, got {x.dtype}")
    if not contiguous:
        raise ValueError(f"{name} must be contiguous")


def _check_queries(Q, index) -> int:
    """Q must be an m x d matrix for an index of dimension d; returns m."""
    if len(Q.shape) != 2:
        raise ValueError(f"queries must be a 2-D (m, d) matrix, got shape {tuple(Q.shape)}")
    _check_matrix("queries", Q, Q.shape[0], index.d, np.float32)
    return int(Q.shape[0])


def _current_stream(x):
    if _is_torch(x) and x.is_cuda:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    return None


def _as_f32(x):
    if _is_torch(x):
        import torch
        return x.to(torch.float32).contiguous()
    return np.ascontiguousarray(x, dtype=np.float32)


def _empty_like_input(x, shape, dtype):
    """Output buffer on the same side (device/host) as the input `x`."""
    if _is_torch(x):
        import torch
        tdt = {np.int32: torch.int32, np.float32: torch.float32, np.uint8: torch.uint8,
               np.int64: torch.int64}[dtype]
        return torch.empty(shape, dtype=tdt, device=x.device)
    return np.empty(shape, dtype=dtype)


class Index:
    """Handle of an index built by :func:`mrpt_build`; freed on close()."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        self._lib = load_library()
        info = IndexInfo()
        _check(self._lib.mrpt_info(self._h, ctypes.byref(info)))
        self.n, self.d, self.T, self.l = info.n, info.d, info.T, info.l
        self.density, self.seed, self.nnz = info.density, info.seed, info.nnz
        self.tree_offset = info.tree_offset

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("index is closed")
        return self._h

    def info(self) -> IndexInfo:
        return mrpt_info(self)

    def query(self, Q, k: int, v: int, **kw):
        return mrpt_query(self, Q, k, v, **kw)

    def export(self, what: str):
        return mrpt_export(self, what)

    def close(self):
        if self._h is not None:
            _check(self._lib.mrpt_free(self._h))
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mrpt_build(data, T: int, l: int, density: float = 0.0, seed: int = 0,
               sparsity: int = MRPT_SPARSITY_BERNOULLI, tree_offset: int = 0) -> Index:
    """Algorithm 1: grow T trees of depth l over the rows of ``data`` (torch
    tensor on the GPU or the host, or a numpy array).  sparsity selects the
    random vectors' nonzeros (mrpt_build_ex): MRPT_SPARSITY_BERNOULLI or
    MRPT_SPARSITY_FIXED (exactly ceil(density * d) per vector).  With
    ``tree_offset`` t0 the index holds trees t0 .. t0+T-1 of the random
    source: one shard of a tree-sharded index."""
    lib = load_library()
    data = _as_f32(data)
    if len(data.shape) != 2:
        raise ValueError(f"data must be a 2-D (n, d) matrix, got shape {tuple(data.shape)}")
    n, d = data.shape
    h = ctypes.c_void_p()
    opts = BuildOpts(int(sparsity), int(tree_offset))
    _check(lib.mrpt_build_ex(_ptr(data), n, d, T, l, float(density), seed & (2**64 - 1),
                             ctypes.byref(opts), ctypes.byref(h)))
    if _is_torch(data) and data.is_cuda:
        # mrpt_build copies the data; keep the source alive until it returns (it is synchronous)
        pass
    return Index(h)


def mrpt_add_lowp(index: Index, precision: int = MRPT_PREC_BF16) -> None:
    """Add a bfloat16 (MRPT_PREC_BF16) or e4m3 + per-row scale
    (MRPT_PREC_FP8) copy of the data for reduced-precision distances."""
    _check(load_library().mrpt_add_lowp(index.handle, int(precision)))


def mrpt_save(index: Index, path: str) -> None:
    """Write the index (random matrix, splits, leaves, data) to `path`."""
    _check(load_library().mrpt_save(index.handle, os.fsencode(path)))


def mrpt_load(path: str) -> Index:
    """Read an index written by mrpt_save onto the current device."""
    h = ctypes.c_void_p()
    _check(load_library().mrpt_load(os.fsencode(path), ctypes.byref(h)))
    return Index(h)


def mrpt_free(index: Index) -> None:
    index.close()


def mrpt_set_stream(index: Index, stream) -> None:
    """Order the index's work on ``stream`` (torch.cuda.Stream, raw handle or None)."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(load_library().mrpt_set_stream(index.handle, ctypes.c_void_p(stream)))


def mrpt_sync(index: Index) -> None:
    _check(load_library().mrpt_sync(index.handle))


def mrpt_info(index: Index) -> IndexInfo:
    info = IndexInfo()
    _check(load_library().mrpt_info(index.handle, ctypes.byref(info)))
    return info


def mrpt_query_ex(index: Index, Q, k: int, v: int, n_trees: int = 0, out_ids=None,
                  out_dists=None, debug: bool = False, cand_cap: int | None = None,
                  stage_ms=None, path: int = 0, precision: int = 0, margin: int = 0,
                  chunk: int = 0, ring: int = 0, n_cand_out=None, vote_table: int = 0):
    """Algorithm 4 for the rows of Q.  Outputs live where Q lives (device
    tensors for a CUDA tensor, numpy arrays for host input) unless given.
    With ``debug`` also returns a dict of the internals: proj, leaf, votes,
    n_cand and cand (members of S, row padded).  ``n_cand_out`` (m int64,
    device or host) receives |S| of every query on its own, without the
    m x n debug buffers.  ``vote_table`` picks how votes are counted (0
    automatic, MRPT_VOTE_COUNTERS, MRPT_VOTE_HASH; see mrpt.h).  ``stage_ms`` (a float32
    numpy array of 4) receives the routing, voting, candidate-search and
    total device times of this call in ms.  ``path`` 0 runs the vote/emit
    and candidate-search kernels, 1 the fused kernel.  ``precision``
    MRPT_PREC_BF16 computes candidate distances from the bfloat16 copy
    (mrpt_add_lowp) and re-ranks the k + ``margin`` nearest in float32."""
    lib = load_library()
    Q = _as_f32(Q)
    m = _check_queries(Q, index)
    if out_ids is None:
        out_ids = _empty_like_input(Q, (m, k), np.int32)
    if out_dists is None:
        out_dists = _empty_like_input(Q, (m, k), np.float32)
    _check_matrix("out_ids", out_ids, m, k, np.int32)
    _check_matrix("out_dists", out_dists, m, k, np.float32)
    stream = _current_stream(Q)
    if stream is not None:
        _check(lib.mrpt_set_stream(index.handle, stream))
    opts = QueryOpts()
    opts.n_trees = int(n_trees)
    opts.path = int(path)
    opts.precision = int(precision)
    opts.margin = int(margin)
    opts.chunk = int(chunk)
    opts.ring = int(ring)
    opts.vote_table = int(vote_table)
    if stage_ms is not None:
        assert stage_ms.dtype == np.float32 and stage_ms.size >= 4
        opts.stage_ms = stage_ms.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    if n_cand_out is not None:
        assert not debug, "n_cand_out: debug already returns n_cand"
        _check_vector("n_cand_out", n_cand_out, m, np.int64)
        opts.n_cand = _ptr(n_cand_out).value
    dbg = None
    if debug:
        T_use = n_trees if n_trees > 0 else index.T
        cap = cand_cap if cand_cap is not None else index.n
        dbg = {
            "proj": _empty_like_input(Q, (m, T_use * index.l), np.float32),
            "leaf": _empty_like_input(Q, (m, T_use), np.int32),
            "votes": _empty_like_input(Q, (m, index.n), np.uint8),
            "n_cand": _empty_like_input(Q, (m,), np.int64),
            "cand": _empty_like_input(Q, (m, max(cap, 1)), np.int32),
        }
        opts.proj = _ptr(dbg["proj"]).value
        opts.leaf = _ptr(dbg["leaf"]).value
        opts.votes = _ptr(dbg["votes"]).value
        opts.n_cand = _ptr(dbg["n_cand"]).value
        opts.cand = _ptr(dbg["cand"]).value
        opts.cand_cap = max(cap, 1)
    _check(lib.mrpt_query_ex(index.handle, _ptr(Q), m, k, v, ctypes.byref(opts), _ptr(out_ids),
                             _ptr(out_dists)))
    if debug:
        return out_ids, out_dists, dbg
    return out_ids, out_dists


def mrpt_query(index: Index, Q, k: int, v: int, n_trees: int = 0, out_ids=None,
               out_dists=None):
    """Algorithm 4: k approximate nearest neighbours of each row of Q."""
    return mrpt_query_ex(index, Q, k, v, n_trees=n_trees, out_ids=out_ids,
                         out_dists=out_dists)


def mrpt_export(index: Index, what: str) -> np.ndarray:
    """Copy one part of the index to a host numpy array (see mrpt.h)."""
    lib = load_library()
    code, dt = EXPORT[what]
    nbytes = lib.mrpt_export_size(index.handle, code)
    if nbytes < 0:
        _check(int(nbytes))
    out = np.empty(max(nbytes, 1) // np.dtype(dt).itemsize, dtype=dt)
    _check(lib.mrpt_export(index.handle, code, ctypes.c_void_p(out.ctypes.data), out.nbytes))
    out = out[: nbytes // np.dtype(dt).itemsize]
    L = 1 << index.l
    if what == "SPLIT":
        return out.reshape(index.T, L - 1)
    if what == "LEAF_OFF":
        return out.reshape(index.T, L + 1)
    if what == "LEAF_IDS":
        return out.reshape(index.T, index.n)
    if what == "DATA":
        return out.reshape(index.n, index.d)
    return out


def mrpt_debug_fail_alloc_after(after: int) -> None:
    _check(load_library().mrpt_debug_fail_alloc_after(int(after)))


def vote_count_capacity(index: Index, n_trees: int = 0) -> int:
    """Row capacity that mrpt_vote_counts needs: min(n_trees ceil(n / 2^l), n)."""
    T_use = n_trees if n_trees > 0 else index.T
    leaf = -(-index.n // (1 << index.l))
    return min(T_use * leaf, index.n)


def mrpt_vote_counts(index: Index, Q, n_trees: int = 0):
    """Per query, the ids with at least one vote among this index's trees and
    their counts (one shard's part of F(x;q), Sec. III-A).  Q is a CUDA
    tensor; returns CUDA tensors (nnz [m] int32, ids [m, cap] int32,
    counts [m, cap] uint8), row i's first nnz[i] entries used."""
    import torch
    lib = load_library()
    m = _check_queries(Q, index)
    if not (_is_torch(Q) and Q.is_cuda):
        raise ValueError("mrpt_vote_counts: Q must be a CUDA tensor")
    cap = max(1, vote_count_capacity(index, n_trees))
    nnz = torch.empty((m,), dtype=torch.int32, device=Q.device)
    ids = torch.empty((m, cap), dtype=torch.int32, device=Q.device)
    counts = torch.empty((m, cap), dtype=torch.uint8, device=Q.device)
    stream = _current_stream(Q)
    if stream is not None:
        _check(lib.mrpt_set_stream(index.handle, stream))
    _check(lib.mrpt_vote_counts(index.handle, _ptr(Q), m, int(n_trees), cap, _ptr(nnz), _ptr(ids),
                                _ptr(counts)))
    return nnz, ids, counts


def mrpt_query_from_counts(index: Index, Q, k: int, v: int, off, ids, counts, out_ids=None,
                           out_dists=None, precision: int = 0, margin: int = 0, chunk: int = 0,
                           ring: int = 0):
    """Algorithm 4 from the shards' vote counts: query i's (id, count) pairs
    are entries off[i]..off[i+1]-1 of ids/counts (CUDA tensors: int64,
    int32, uint8); F is their sum per id, S = {F >= v}.  Returns the k-NN
    rows as CUDA tensors."""
    import torch
    lib = load_library()
    m = _check_queries(Q, index)
    for name, t, dt in (("off", off, torch.int64), ("ids", ids, torch.int32), ("counts", counts, torch.uint8)):
        if not (_is_torch(t) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA tensor of {dt}")
    if off.numel() != m + 1 or ids.numel() != counts.numel():
        raise ValueError("off must hold m + 1 offsets and ids/counts the same number of entries")
    if out_ids is None:
        out_ids = torch.empty((m, k), dtype=torch.int32, device=Q.device)
    if out_dists is None:
        out_dists = torch.empty((m, k), dtype=torch.float32, device=Q.device)
    _check_matrix("out_ids", out_ids, m, k, np.int32)
    _check_matrix("out_dists", out_dists, m, k, np.float32)
    stream = _current_stream(Q)
    if stream is not None:
        _check(lib.mrpt_set_stream(index.handle, stream))
    opts = QueryOpts()
    opts.precision, opts.margin, opts.chunk, opts.ring = int(precision), int(margin), int(chunk), int(ring)
    _check(lib.mrpt_query_from_counts(index.handle, _ptr(Q), m, int(k), int(v), _ptr(off),
                                      _ptr(ids) if ids.numel() else None,
                                      _ptr(counts) if counts.numel() else None, ctypes.byref(opts),
                                      _ptr(out_ids), _ptr(out_dists)))
    return out_ids, out_dists


def mrpt_debug_row_wait_tries(tries: int) -> None:
    """Testing aid: shorten the candidate search's row waits to `tries`
    tries (negative restores the full bound); see mrpt.h."""
    _check(load_library().mrpt_debug_row_wait_tries(int(tries)))


def mrpt_query_noalloc(index: Index, Q, k: int, v: int, out_ids, out_dists,
                       n_trees: int = 0) -> None:
    """mrpt_query without any device allocation, for callers that may not
    allocate (a latency-bound serving loop, or device memory owned by
    another framework's pool).  Q, out_ids and out_dists must be CUDA
    tensors; m * n_trees is limited to MRPT_NOALLOC_MAX_LEAF_ENTRIES; calls
    whose GPU work overlaps share one scratch array and race."""
    lib = load_library()
    m = _check_queries(Q, index)
    _check_matrix("out_ids", out_ids, m, k, np.int32)
    _check_matrix("out_dists", out_dists, m, k, np.float32)
    stream = _current_stream(Q)
    if stream is not None:
        _check(lib.mrpt_set_stream(index.handle, stream))
    _check(lib.mrpt_query_noalloc(index.handle, _ptr(Q), m, k, v, int(n_trees),
                                  _ptr(out_ids), _ptr(out_dists)))


class Plan:
    """A query captured into a CUDA graph (mrpt_plan_create): fixed k, v and
    options, any batch of up to m_max queries per run."""

    def __init__(self, index: Index, m_max: int, k: int, v: int, n_trees: int = 0, path: int = 0,
                 precision: int = 0, margin: int = 0, chunk: int = 0, ring: int = 0, vote_table: int = 0):
        self._lib = load_library()
        self.index, self.m_max, self.k, self.v = index, m_max, k, v
        opts = QueryOpts()
        opts.n_trees, opts.path, opts.precision = int(n_trees), int(path), int(precision)
        opts.margin, opts.chunk, opts.ring = int(margin), int(chunk), int(ring)
        opts.vote_table = int(vote_table)
        h = ctypes.c_void_p()
        _check(self._lib.mrpt_plan_create(index.handle, int(m_max), int(k), int(v),
                                          ctypes.byref(opts), ctypes.byref(h)))
        self._h = h

    def run(self, Q, out_ids=None, out_dists=None):
        Q = _as_f32(Q)
        m = _check_queries(Q, self.index)
        if out_ids is None:
            out_ids = _empty_like_input(Q, (m, self.k), np.int32)
        if out_dists is None:
            out_dists = _empty_like_input(Q, (m, self.k), np.float32)
        _check_matrix("out_ids", out_ids, m, self.k, np.int32)
        _check_matrix("out_dists", out_dists, m, self.k, np.float32)
        stream = _current_stream(Q)
        if stream is not None:
            _check(self._lib.mrpt_set_stream(self.index.handle, stream))
        _check(self._lib.mrpt_plan_run(self._h, _ptr(Q), m, _ptr(out_ids), _ptr(out_dists)))
        return out_ids, out_dists

    def close(self):
        if getattr(self, "_h", None) is not None:
            _check(self._lib.mrpt_plan_free(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mrpt_plan_create(index: Index, m_max: int, k: int, v: int, **opts) -> Plan:
    return Plan(index, m_max, k, v, **opts)


def mrpt_plan_run(plan: Plan, Q, out_ids=None, out_dists=None):
    return plan.run(Q, out_ids, out_dists)


def mrpt_plan_free(plan: Plan) -> None:
    plan.close()
