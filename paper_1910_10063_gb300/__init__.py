"""GB300 permutation index (Zhang & Ross, ICDE 2020, arXiv 1910.10063).

Thin ctypes binding over ``libskx.so`` (C ABI in ``include/skx.h``).  The
functions below carry the C entry points' names and only marshal arguments:
torch CUDA tensors supply device pointers, the current torch stream supplies
the CUDA stream, and every step of the path runs in the library's kernels.
There is no CPU fallback: without the built library every call raises.

    import torch, paper_1910_10063_gb300 as skx
    idx = skx.skx_build_index(fk, N)                  # Section III-A: count + sort
    fk2 = torch.empty_like(fk); skx.skx_remap(idx, fk, fk2)
    dim2 = torch.empty_like(dim); skx.skx_reorder(idx, dim, dim2)
    out = skx.skx_probe_aggregate(dim2, fk2, measure, skx.Query.groupby_sum())
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libskx.so")

SKX_OK, SKX_EINVAL, SKX_ENOMEM, SKX_EKEYRANGE, SKX_EGROUPRANGE = 0, 1, 2, 3, 4
SKX_ECUDA, SKX_ETIMEOUT, SKX_EBUSY, SKX_ENOTSUP = 5, 6, 7, 8
SKX_AGG_COUNT, SKX_AGG_SUM, SKX_AGG_GROUPBY_SUM = 0, 1, 2
SKX_COUNT_AUTO, SKX_COUNT_SINGLE_PASS, SKX_COUNT_PARTITIONED = 0, 1, 2

_lock = threading.Lock()
_lib = None


class SkxError(RuntimeError):
    def __init__(self, status: int, where: str, lib=None):
        msg = f"{where}: status {status}"
        if lib is not None:
            msg = f"{where}: {lib.skx_strerror(status).decode()}"
            if status == SKX_ECUDA:
                msg += f" ({lib.skx_last_cuda_error().decode()})"
        super().__init__(msg)
        self.status = status


class Query(ctypes.Structure):
    _fields_ = [("agg", ctypes.c_int32), ("filter_col", ctypes.c_int32), ("filter_lt", ctypes.c_int32),
                ("group_col", ctypes.c_int32), ("num_groups", ctypes.c_int32), ("payload_col", ctypes.c_int32)]

    @classmethod
    def groupby_sum(cls, num_groups=1000, filter_col=1, filter_lt=50, group_col=0, payload_col=2):
        return cls(SKX_AGG_GROUPBY_SUM, filter_col, filter_lt, group_col, num_groups, payload_col)

    @classmethod
    def sum(cls, filter_col=1, filter_lt=50, payload_col=2):
        return cls(SKX_AGG_SUM, filter_col, filter_lt, 0, 1, payload_col)

    @classmethod
    def count(cls, filter_col=1, filter_lt=50):
        return cls(SKX_AGG_COUNT, filter_col, filter_lt, 0, 1, -1)

    @property
    def nout(self) -> int:
        return self.num_groups if self.agg == SKX_AGG_GROUPBY_SUM else 1

    def __repr__(self):
        return (f"Query(agg={self.agg}, filter_col={self.filter_col}, filter_lt={self.filter_lt}, "
                f"group_col={self.group_col}, num_groups={self.num_groups}, payload_col={self.payload_col})")


class ProbeDesc(ctypes.Structure):
    _fields_ = [("fk", ctypes.c_void_p), ("measure", ctypes.c_void_p), ("F", ctypes.c_int64), ("q", Query),
                ("out", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("hot_keys", ctypes.c_int32),
                ("lane_keys", ctypes.c_int32), ("warp_aggregate", ctypes.c_int32), ("unroll", ctypes.c_int32),
                ("gather_policy", ctypes.c_int32), ("split_keys", ctypes.c_int32),
                ("split_bucket", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}

    @classmethod
    def plain(cls):
        """No hot prefix: the probe used on a layout without a permutation index."""
        t = cls()
        t.hot_keys = -1
        t.lane_keys = -1
        return t

    def __repr__(self):
        return f"Tuning({self.as_dict()})"


class Drift(ctypes.Structure):
    _fields_ = [("sample", ctypes.c_int64), ("t", ctypes.c_int64), ("share_stale", ctypes.c_double),
                ("share_fresh", ctypes.c_double), ("loss", ctypes.c_double), ("rebuild", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_int32), ("tile_rows", ctypes.c_int32), ("round_rows", ctypes.c_int64),
                ("memory_budget", ctypes.c_int64), ("timeout_ms", ctypes.c_int32), ("cpu_affinity", ctypes.c_int32),
                ("tuning", Tuning), ("reserved", ctypes.c_int32 * 8)]


class Request(ctypes.Structure):
    _fields_ = [("h_fk", ctypes.c_void_p), ("h_measure", ctypes.c_void_p), ("F", ctypes.c_int64), ("q", Query),
                ("h_out", ctypes.c_void_p)]


def lib():
    """Load libskx.so (raises if it has not been built -- there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libskx.so is not built at {LIB_PATH}; run "
                                   "`python -m paper_1910_10063_gb300.build` (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            st = ctypes.c_int
            L.skx_strerror.argtypes = [st]; L.skx_strerror.restype = ctypes.c_char_p
            L.skx_last_cuda_error.argtypes = []; L.skx_last_cuda_error.restype = ctypes.c_char_p
            L.skx_version.argtypes = []; L.skx_version.restype = i32
            L.skx_stream_status.argtypes = [P]; L.skx_stream_status.restype = st
            L.skx_build_index.argtypes = [P, i64, i32, P, ctypes.POINTER(P)]; L.skx_build_index.restype = st
            L.skx_count.argtypes = [P, i64, i32, P, P]; L.skx_count.restype = st
            L.skx_count_ex.argtypes = [P, i64, i32, P, i32, P]; L.skx_count_ex.restype = st
            L.skx_build_index_from_counts.argtypes = [P, i32, i64, P, ctypes.POINTER(P)]
            L.skx_build_index_from_counts.restype = st
            L.skx_sort_by_count_noalloc.argtypes = [P, i32, i64, P, P, P]
            L.skx_sort_by_count_noalloc.restype = st
            L.skx_sort_by_count_noalloc_max_n.argtypes = []; L.skx_sort_by_count_noalloc_max_n.restype = i32
            L.skx_kernel_launches.argtypes = []; L.skx_kernel_launches.restype = ctypes.c_uint64
            for n in ("skx_index_perm", "skx_index_rank", "skx_index_counts"):
                getattr(L, n).argtypes = [P, ctypes.POINTER(P)]
                getattr(L, n).restype = st
            L.skx_index_size.argtypes = [P]; L.skx_index_size.restype = i32
            L.skx_index_destroy.argtypes = [P]; L.skx_index_destroy.restype = None
            L.skx_remap.argtypes = [P, P, P, i64, P]; L.skx_remap.restype = st
            L.skx_reorder.argtypes = [P, P, P, i32, i32, P]; L.skx_reorder.restype = st
            L.skx_materialize.argtypes = [P, i32, i32, i32, P, i64, P, P]; L.skx_materialize.restype = st
            L.skx_reorder_columns.argtypes = [P, P, i32, i32, P, i32, P, P]; L.skx_reorder_columns.restype = st
            L.skx_reorder_query.argtypes = [P, P, i32, i32, ctypes.POINTER(Query), P, P]
            L.skx_reorder_query.restype = st
            L.skx_query_prefiltered.argtypes = [ctypes.POINTER(Query)]; L.skx_query_prefiltered.restype = Query
            L.skx_reorder_query_packed.argtypes = [P, P, i32, i32, ctypes.POINTER(Query), P, P, P]
            L.skx_reorder_query_packed.restype = st
            L.skx_query_packed_key_bits.argtypes = [ctypes.POINTER(Query)]; L.skx_query_packed_key_bits.restype = i32
            L.skx_probe_packed.argtypes = [P, P, i32, P, P, i64, ctypes.POINTER(Query), P, ctypes.POINTER(Tuning), P]
            L.skx_probe_packed.restype = st
            L.skx_probe_aggregate.argtypes = [P, i32, i32, P, P, i64, ctypes.POINTER(Query), P,
                                              ctypes.POINTER(Tuning), P]
            L.skx_probe_aggregate.restype = st
            L.skx_probe_default_tuning.argtypes = [i32, i32, i64, ctypes.POINTER(Query), ctypes.c_int,
                                                   ctypes.POINTER(Tuning)]
            L.skx_probe_default_tuning.restype = st
            L.skx_probe_resolve_tuning.argtypes = [i32, i32, i64, ctypes.POINTER(Query), ctypes.POINTER(Tuning),
                                                   ctypes.POINTER(Tuning)]
            L.skx_probe_resolve_tuning.restype = st
            L.skx_probe_autotune.argtypes = [P, i32, i32, P, P, i64, ctypes.POINTER(Query), ctypes.c_int, P, P,
                                             ctypes.POINTER(Tuning), ctypes.POINTER(ctypes.c_float)]
            L.skx_probe_autotune.restype = st
            L.skx_probe_autotune_ex.argtypes = [P, i32, i32, P, P, i64, ctypes.POINTER(Query), ctypes.c_int,
                                                ctypes.POINTER(Tuning), P, P, ctypes.POINTER(Tuning),
                                                ctypes.POINTER(ctypes.c_float)]
            L.skx_probe_autotune_ex.restype = st
            L.skx_split_threshold.argtypes = [P, i32, i64, ctypes.c_double, ctypes.POINTER(i64), P]
            L.skx_split_threshold.restype = st
            L.skx_index_drift.argtypes = [P, P, i64, i64, ctypes.c_double, ctypes.POINTER(Drift), P]
            L.skx_index_drift.restype = st
            L.skx_drift_from_counts.argtypes = [P, i32, i64, ctypes.c_double, ctypes.POINTER(Drift)]
            L.skx_drift_from_counts.restype = st
            L.skx_split_threshold_from_fit.argtypes = [ctypes.c_double, i32, i32, i64, ctypes.c_double,
                                                       ctypes.POINTER(i64)]
            L.skx_split_threshold_from_fit.restype = st
            L.skx_batch_plan_create.argtypes = [P, i32, i32, ctypes.POINTER(ProbeDesc), i32, ctypes.POINTER(Tuning), i32,
                                                P, ctypes.POINTER(P)]
            L.skx_batch_plan_create.restype = st
            L.skx_batch_plan_launch.argtypes = [P, ctypes.c_int, P]; L.skx_batch_plan_launch.restype = st
            L.skx_batch_plan_autotune.argtypes = [P, P, ctypes.POINTER(Tuning), ctypes.POINTER(i32),
                                                  ctypes.POINTER(ctypes.c_float)]
            L.skx_batch_plan_autotune.restype = st
            L.skx_batch_plan_destroy.argtypes = [P]; L.skx_batch_plan_destroy.restype = None
            L.skx_probe_batch.argtypes = [P, i32, i32, ctypes.POINTER(ProbeDesc), i32, ctypes.POINTER(Tuning), P]
            L.skx_probe_batch.restype = st
            L.skx_server_create.argtypes = [P, i32, i32, P, ctypes.POINTER(ServerConfig), ctypes.POINTER(P)]
            L.skx_server_create.restype = st
            L.skx_server_submit.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
            L.skx_server_submit.restype = st
            L.skx_server_wait.argtypes = [P, ctypes.c_uint64, i32]; L.skx_server_wait.restype = st
            L.skx_server_request_times.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            L.skx_server_request_times.restype = st
            L.skx_server_release.argtypes = [P, ctypes.c_uint64]; L.skx_server_release.restype = st
            L.skx_server_replay.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_double), i32, i32,
                                            ctypes.POINTER(ctypes.c_double)]
            L.skx_server_replay.restype = st
            L.skx_server_stats.argtypes = [P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(ctypes.c_uint64)]
            L.skx_server_stats.restype = st
            L.skx_server_destroy.argtypes = [P]; L.skx_server_destroy.restype = None
            L.skx_index_append.argtypes = [P, i32, P]; L.skx_index_append.restype = st
            L.skx_topk_counts.argtypes = [P, i64, i32, P, P]; L.skx_topk_counts.restype = st
            L.skx_select_bitmap.argtypes = [P, i32, i32, i32, i32, P, P]; L.skx_select_bitmap.restype = st
            L.skx_select.argtypes = [P, i32, P, i64, P, P, P]; L.skx_select.restype = st
            L.skx_cache_hit_rate.argtypes = [P, i64, i64, ctypes.POINTER(ctypes.c_double)]
            L.skx_cache_hit_rate.restype = st
            L.skx_cache_line_cdf.argtypes = [P, i64, i64, P]; L.skx_cache_line_cdf.restype = st
            L.skx_cache_threshold.argtypes = [P, i64, i64, ctypes.c_double, i32, ctypes.POINTER(i64)]
            L.skx_cache_threshold.restype = st
            L.skx_powerlaw_fit.argtypes = [P, P, i64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            L.skx_powerlaw_fit.restype = st
            L.skx_index_counts_at_ranks.argtypes = [P, P, i64, P, P]; L.skx_index_counts_at_ranks.restype = st
            L.skx_join_aggregate_host.argtypes = [P, i32, i32, P, P, i64, ctypes.POINTER(Query), P, P]
            L.skx_join_aggregate_host.restype = st
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != SKX_OK:
        raise SkxError(status, where, lib())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dptr(t, what, dtype=None):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


class Index:
    """Owner of an ``skx_index`` (perm, rank and counts on the device)."""

    def __init__(self, handle: ctypes.c_void_p, n: int):
        self._h = handle
        self.n = n

    def _view(self, fn, dtype):
        import torch
        p = ctypes.c_void_p()
        _check(getattr(lib(), fn)(self._h, ctypes.byref(p)), fn)
        return _device_view(p.value, self.n, dtype)

    @property
    def perm(self):
        """int32[N] new -> old (borrowed view, valid while the Index lives)."""
        import torch
        return self._view("skx_index_perm", torch.int32)

    @property
    def rank(self):
        """int32[N] old -> new (borrowed view)."""
        import torch
        return self._view("skx_index_rank", torch.int32)

    @property
    def counts(self):
        """uint32 counts viewed as int32[N] (borrowed view)."""
        import torch
        return self._view("skx_index_counts", torch.int32)

    def close(self):
        if self._h:
            lib().skx_index_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _device_view(ptr: int, n: int, dtype):
    """A torch tensor over library-owned device memory (no copy, no ownership)."""
    import torch
    itemsize = torch.empty((), dtype=dtype).element_size()

    class _Holder:
        pass

    h = _Holder()
    h.__cuda_array_interface__ = {"shape": (n,), "typestr": {1: "|i1", 4: "<i4", 8: "<i8"}[itemsize],
                                  "data": (ptr, False), "version": 3, "strides": None}
    return torch.as_tensor(h, device="cuda").view(dtype)


# ------------------------------------------------------------------ entry points
def skx_version() -> int:
    return lib().skx_version()


def skx_stream_status(stream=None) -> int:
    """Synchronise and return (and clear) the data-error status; see skx.h."""
    return lib().skx_stream_status(_stream(stream))


def skx_build_index(fk, n: int, stream=None) -> Index:
    import torch
    h = ctypes.c_void_p()
    _check(lib().skx_build_index(_dptr(fk, "fk", torch.int32), fk.numel(), int(n), _stream(stream), ctypes.byref(h)),
           "skx_build_index")
    return Index(h, int(n))


def skx_count(fk, n: int, counts=None, stream=None):
    """Q3 count: int32 view of uint32 counts[n] on the device."""
    import torch
    if counts is None:
        counts = torch.empty(n, dtype=torch.int32, device=fk.device)
    _check(lib().skx_count(_dptr(fk, "fk", torch.int32), fk.numel(), int(n), _dptr(counts, "counts", torch.int32),
                           _stream(stream)), "skx_count")
    return counts


def skx_count_ex(fk, n: int, method: int, counts=None, stream=None):
    """Q3 count with the algorithm chosen (SKX_COUNT_AUTO / _SINGLE_PASS / _PARTITIONED)."""
    import torch
    if counts is None:
        counts = torch.empty(n, dtype=torch.int32, device=fk.device)
    _check(lib().skx_count_ex(_dptr(fk, "fk", torch.int32), fk.numel(), int(n), _dptr(counts, "counts", torch.int32),
                              int(method), _stream(stream)), "skx_count_ex")
    return counts


def skx_build_index_from_counts(counts, f_bound: int, stream=None) -> Index:
    import torch
    h = ctypes.c_void_p()
    _check(lib().skx_build_index_from_counts(_dptr(counts, "counts", torch.int32), counts.numel(), int(f_bound),
                                             _stream(stream), ctypes.byref(h)), "skx_build_index_from_counts")
    return Index(h, counts.numel())


def skx_sort_by_count_noalloc(counts, f_bound: int, perm, rank, stream=None):
    """Frequency order from counts into caller buffers, without allocating (N <= 2^20)."""
    import torch
    n = counts.numel()
    if perm.numel() != n or rank.numel() != n:
        raise ValueError("perm and rank must have one entry per id")
    _check(lib().skx_sort_by_count_noalloc(_dptr(counts, "counts", torch.int32), n, int(f_bound),
                                           _dptr(perm, "perm", torch.int32), _dptr(rank, "rank", torch.int32),
                                           _stream(stream)), "skx_sort_by_count_noalloc")
    return perm, rank


def skx_kernel_launches() -> int:
    return lib().skx_kernel_launches()


def skx_remap(index: Index, fk_in, fk_out, stream=None):
    import torch
    if fk_out.numel() != fk_in.numel():
        raise ValueError("fk_out must have the same length as fk_in")
    _check(lib().skx_remap(index._h, _dptr(fk_in, "fk_in", torch.int32), _dptr(fk_out, "fk_out", torch.int32),
                           fk_in.numel(), _stream(stream)), "skx_remap")
    return fk_out


def _row_bytes(rows):
    if rows.dim() < 1 or rows.shape[0] == 0:
        raise ValueError("rows must have a leading row dimension")
    return rows.numel() * rows.element_size() // rows.shape[0]


def skx_reorder(index: Index, rows_in, rows_out, stream=None):
    if rows_out.shape != rows_in.shape or rows_out.dtype != rows_in.dtype:
        raise ValueError("rows_out must match rows_in")
    _check(lib().skx_reorder(index._h, _dptr(rows_in, "rows_in"), _dptr(rows_out, "rows_out"), rows_in.shape[0],
                             _row_bytes(rows_in), _stream(stream)), "skx_reorder")
    return rows_out


def skx_materialize(rows, fk, col: int, out=None, stream=None):
    """Q1: int32 out[i] = rows[fk[i], col] on the device (either layout)."""
    import torch
    if out is None:
        out = torch.empty(fk.numel(), dtype=torch.int32, device=fk.device)
    if out.numel() < fk.numel():
        raise ValueError("out is shorter than fk")
    _check(lib().skx_materialize(_dptr(rows, "rows"), rows.shape[0], _row_bytes(rows), int(col),
                                 _dptr(fk, "fk", torch.int32), fk.numel(), _dptr(out, "out", torch.int32),
                                 _stream(stream)), "skx_materialize")
    return out


def skx_reorder_columns(index: Index | None, rows_in, cols, out=None, stream=None):
    """Permuted (index) or identity-order (None) copy of the int32 columns `cols` -> int32[N, len(cols)]."""
    import numpy as np
    import torch
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    n = rows_in.shape[0]
    if out is None:
        out = torch.empty((n, cols.size), dtype=torch.int32, device=rows_in.device)
    _check(lib().skx_reorder_columns(index._h if index is not None else None, _dptr(rows_in, "rows_in"), n,
                                     _row_bytes(rows_in), cols.ctypes.data_as(ctypes.c_void_p), cols.size,
                                     _dptr(out, "out"), _stream(stream)), "skx_reorder_columns")
    return out


def skx_reorder_query(index: Index | None, rows_in, query: Query, out=None, stream=None):
    """8-byte {key or sentinel, payload} rows with the query's filter applied -> int32[N, 2]."""
    import torch
    n = rows_in.shape[0]
    if out is None:
        out = torch.empty((n, 2), dtype=torch.int32, device=rows_in.device)
    _check(lib().skx_reorder_query(index._h if index is not None else None, _dptr(rows_in, "rows_in"), n,
                                   _row_bytes(rows_in), ctypes.byref(query), _dptr(out, "out"), _stream(stream)),
           "skx_reorder_query")
    return out


def skx_query_prefiltered(query: Query) -> Query:
    return lib().skx_query_prefiltered(ctypes.byref(query))


def skx_reorder_query_packed(index: Index | None, rows_in, query: Query, out8=None, out4=None, stream=None):
    """The 8-byte query copy and its 32-bit packed form -> (int32[N, 2], int32[N])."""
    import torch
    n = rows_in.shape[0]
    if out8 is None:
        out8 = torch.empty((n, 2), dtype=torch.int32, device=rows_in.device)
    if out4 is None:
        out4 = torch.empty(n, dtype=torch.int32, device=rows_in.device)
    _check(lib().skx_reorder_query_packed(index._h if index is not None else None, _dptr(rows_in, "rows_in"), n,
                                          _row_bytes(rows_in), ctypes.byref(query), _dptr(out8, "out8"),
                                          _dptr(out4, "out4"), _stream(stream)), "skx_reorder_query_packed")
    return out8, out4


def skx_query_packed_key_bits(query: Query) -> int:
    return lib().skx_query_packed_key_bits(ctypes.byref(query))


def skx_probe_packed(rows4, rows8, fk, measure, query: Query, out=None, tuning: Tuning | None = None, stream=None):
    """The original query's int64 result over the packed copy (escapes read from rows8)."""
    import torch
    if out is None:
        out = torch.empty(query.nout, dtype=torch.int64, device=fk.device)
    if measure is not None and measure.numel() != fk.numel():
        raise ValueError("measure must have the same length as fk")
    if rows8.shape[0] != rows4.shape[0]:
        raise ValueError("rows4 and rows8 must have the same number of rows")
    _check(lib().skx_probe_packed(_dptr(rows4, "rows4"), _dptr(rows8, "rows8"), rows4.shape[0],
                                  _dptr(fk, "fk", torch.int32), _dptr(measure, "measure", torch.int32), fk.numel(),
                                  ctypes.byref(query), _dptr(out, "out", torch.int64),
                                  ctypes.byref(tuning) if tuning is not None else None, _stream(stream)),
           "skx_probe_packed")
    return out


def skx_probe_aggregate(rows, fk, measure, query: Query, out=None, tuning: Tuning | None = None, stream=None):
    """int64 result tensor ([num_groups] for GROUPBY_SUM, [1] otherwise) on the device."""
    import torch
    if out is None:
        out = torch.empty(query.nout, dtype=torch.int64, device=fk.device)
    if measure is not None and measure.numel() != fk.numel():
        raise ValueError("measure must have the same length as fk")
    _check(lib().skx_probe_aggregate(_dptr(rows, "rows"), rows.shape[0], _row_bytes(rows),
                                     _dptr(fk, "fk", torch.int32), _dptr(measure, "measure", torch.int32),
                                     fk.numel(), ctypes.byref(query), _dptr(out, "out", torch.int64),
                                     ctypes.byref(tuning) if tuning is not None else None, _stream(stream)),
           "skx_probe_aggregate")
    return out


def skx_probe_default_tuning(n: int, row_bytes: int, f: int, query: Query, remapped: bool = True) -> Tuning:
    t = Tuning()
    _check(lib().skx_probe_default_tuning(n, row_bytes, f, ctypes.byref(query), int(remapped), ctypes.byref(t)),
           "skx_probe_default_tuning")
    return t


def skx_probe_autotune(rows, fk, measure, query: Query, remapped: bool = True, out=None, stream=None,
                       split_hint: int = 0):
    """Returns (Tuning, estimated ms for the full F) chosen by timing candidates on this data.
    split_hint > 0 (a split threshold, e.g. from skx_split_threshold) adds the split probe's
    candidates around it (skx_probe_autotune_ex)."""
    import torch
    if out is None:
        out = torch.empty(query.nout, dtype=torch.int64, device=fk.device)
    t = Tuning()
    ms = ctypes.c_float()
    hint = None
    if split_hint and split_hint > 0:
        hint = Tuning()
        hint.split_keys = int(split_hint)
    _check(lib().skx_probe_autotune_ex(_dptr(rows, "rows"), rows.shape[0], _row_bytes(rows),
                                       _dptr(fk, "fk", torch.int32), _dptr(measure, "measure", torch.int32),
                                       fk.numel(), ctypes.byref(query), int(remapped),
                                       ctypes.byref(hint) if hint is not None else None,
                                       _dptr(out, "out", torch.int64), _stream(stream), ctypes.byref(t),
                                       ctypes.byref(ms)), "skx_probe_autotune_ex")
    return t, ms.value


def skx_index_drift(index: "Index", fk_sample, t: int, max_loss: float = 0.02, stream=None) -> Drift:
    """Staleness of the index against a device sample of the fact column (original ids)."""
    import torch
    d = Drift()
    _check(lib().skx_index_drift(index._h, _dptr(fk_sample, "fk_sample", torch.int32), fk_sample.numel(), int(t),
                                 float(max_loss), ctypes.byref(d), _stream(stream)), "skx_index_drift")
    return d


def skx_drift_from_counts(counts_by_rank, t: int, max_loss: float = 0.02) -> Drift:
    """Host half of skx_index_drift from counts by current rank (numpy, uint32)."""
    import numpy as np
    c = np.ascontiguousarray(counts_by_rank, dtype=np.uint32)
    d = Drift()
    _check(lib().skx_drift_from_counts(c.ctypes.data_as(ctypes.c_void_p), c.size, int(t), float(max_loss),
                                       ctypes.byref(d)), "skx_drift_from_counts")
    return d


def skx_probe_resolve_tuning(n: int, row_bytes: int, f: int, query: Query, tuning: Tuning) -> Tuning:
    """The tuning the probe resolves `tuning` to (host only)."""
    out = Tuning()
    _check(lib().skx_probe_resolve_tuning(int(n), int(row_bytes), int(f), ctypes.byref(query), ctypes.byref(tuning),
                                          ctypes.byref(out)), "skx_probe_resolve_tuning")
    return out


def skx_split_threshold_from_fit(slope: float, n: int, row_bytes: int, cache_bytes: int, p: float = 0.5) -> int:
    """Host half of skx_split_threshold: the model's t for counts proportional to (rank + 1)^slope."""
    t = ctypes.c_int64()
    _check(lib().skx_split_threshold_from_fit(float(slope), int(n), int(row_bytes), int(cache_bytes), float(p),
                                              ctypes.byref(t)), "skx_split_threshold_from_fit")
    return t.value


def skx_split_threshold(index: "Index", row_bytes: int, cache_bytes: int = 0, p: float = 0.5, stream=None) -> int:
    """The split threshold t (Section IV-B) from the index's counts through the Section III-C model."""
    t = ctypes.c_int64()
    _check(lib().skx_split_threshold(index._h, int(row_bytes), int(cache_bytes), float(p), ctypes.byref(t),
                                     _stream(stream)), "skx_split_threshold")
    return t.value


def _descs(items):
    """items: iterable of (fk, measure_or_None, Query, out) with CUDA tensors -> ctypes array."""
    import torch
    items = list(items)
    arr = (ProbeDesc * len(items))()
    for i, (fk, m, q, out) in enumerate(items):
        if out.numel() < q.nout:
            raise ValueError("output too small for the query")
        arr[i] = ProbeDesc(_dptr(fk, "fk", torch.int32), _dptr(m, "measure", torch.int32) if m is not None else None,
                           fk.numel(), q, _dptr(out, "out", torch.int64))
    return arr


class BatchPlan:
    """Many probes against one dimension table in one persistent launch (optionally a CUDA graph)."""

    def __init__(self, rows, items, tuning: Tuning | None = None, tile_rows: int = 0, stream=None):
        self._keep = list(items)  # the tensors must outlive the plan
        arr = _descs(self._keep)
        self._h = ctypes.c_void_p()
        _check(lib().skx_batch_plan_create(_dptr(rows, "rows"), rows.shape[0], _row_bytes(rows), arr, len(arr),
                                           ctypes.byref(tuning) if tuning is not None else None, int(tile_rows),
                                           _stream(stream), ctypes.byref(self._h)), "skx_batch_plan_create")
        self.rows = rows

    def launch(self, use_graph: bool = False, stream=None):
        _check(lib().skx_batch_plan_launch(self._h, int(use_graph), _stream(stream)), "skx_batch_plan_launch")

    def autotune(self, stream=None):
        t, tile, ms = Tuning(), ctypes.c_int32(), ctypes.c_float()
        _check(lib().skx_batch_plan_autotune(self._h, _stream(stream), ctypes.byref(t), ctypes.byref(tile),
                                             ctypes.byref(ms)), "skx_batch_plan_autotune")
        return t, tile.value, ms.value

    def close(self):
        if self._h:
            lib().skx_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def skx_probe_batch(rows, items, tuning: Tuning | None = None, stream=None):
    arr = _descs(items)
    _check(lib().skx_probe_batch(_dptr(rows, "rows"), rows.shape[0], _row_bytes(rows), arr, len(arr),
                                 ctypes.byref(tuning) if tuning is not None else None, _stream(stream)),
           "skx_probe_batch")


class Server:
    """Continuous-batching request loop over a resident reordered table and rank array.

    Requests are (fk_host, measure_host_or_None, Query) with host numpy arrays or CPU tensors
    holding ORIGINAL keys; results come back as int64 numpy arrays."""

    def __init__(self, rows, rank=None, config: ServerConfig | None = None):
        import torch
        self._h = ctypes.c_void_p()
        _check(lib().skx_server_create(_dptr(rows, "rows"), rows.shape[0], _row_bytes(rows),
                                       _dptr(rank, "rank", torch.int32) if rank is not None else None,
                                       ctypes.byref(config) if config is not None else None, ctypes.byref(self._h)),
               "skx_server_create")
        self.rows, self.rank = rows, rank
        self._keep = {}

    @staticmethod
    def _host(a):
        import numpy as np
        import torch
        if a is None:
            return None, None
        if isinstance(a, torch.Tensor):
            return ctypes.c_void_p(a.data_ptr()), a
        a = np.ascontiguousarray(a, dtype=np.int32)
        return a.ctypes.data_as(ctypes.c_void_p), a

    def make_request(self, fk, measure, query: Query):
        import numpy as np
        pf, kf = self._host(fk)
        pm, km = self._host(measure)
        out = np.zeros(query.nout, dtype=np.int64)
        n = fk.numel() if hasattr(fk, "numel") else np.asarray(fk).size
        req = Request(pf, pm, n, query, out.ctypes.data_as(ctypes.c_void_p))
        return req, (kf, km, out)

    def submit(self, fk, measure, query: Query) -> int:
        req, keep = self.make_request(fk, measure, query)
        t = ctypes.c_uint64()
        _check(lib().skx_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "skx_server_submit")
        self._keep[t.value] = keep
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 60000):
        st = lib().skx_server_wait(self._h, ticket, timeout_ms)
        _check(st, "skx_server_wait")
        out = self._keep.pop(ticket)[2]
        lib().skx_server_release(self._h, ticket)
        return out

    def replay(self, requests, arrival_s, timeout_ms: int = 120000):
        """requests: list of (Request, keep) from make_request; returns latencies in seconds."""
        import numpy as np
        arr = (Request * len(requests))(*[r for r, _ in requests])
        t = np.ascontiguousarray(arrival_s, dtype=np.float64)
        lat = np.zeros(len(requests), dtype=np.float64)
        _check(lib().skx_server_replay(self._h, arr, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(requests),
                                       timeout_ms, lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "skx_server_replay")
        return lat

    def stats(self):
        r, n, m = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().skx_server_stats(self._h, ctypes.byref(r), ctypes.byref(n), ctypes.byref(m)), "skx_server_stats")
        return {"rounds": r.value, "rows": n.value, "max_active": m.value}

    def close(self):
        if self._h:
            lib().skx_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def skx_index_append(index: Index, n_new: int, stream=None) -> Index:
    _check(lib().skx_index_append(index._h, int(n_new), _stream(stream)), "skx_index_append")
    index.n += int(n_new)
    return index


def skx_topk_counts(fk, k: int, out=None, stream=None):
    """int64[k] counts of the transformed ids 0..k-1 (the k heavy hitters)."""
    import torch
    if out is None:
        out = torch.empty(k, dtype=torch.int64, device=fk.device)
    _check(lib().skx_topk_counts(_dptr(fk, "fk", torch.int32), fk.numel(), int(k), _dptr(out, "out", torch.int64),
                                 _stream(stream)), "skx_topk_counts")
    return out


def skx_select_bitmap(rows, filter_col: int = 1, filter_lt: int = 50, out=None, stream=None):
    import torch
    n = rows.shape[0]
    if out is None:
        out = torch.empty((n + 31) // 32, dtype=torch.int32, device=rows.device)
    _check(lib().skx_select_bitmap(_dptr(rows, "rows"), n, _row_bytes(rows), int(filter_col), int(filter_lt),
                                   _dptr(out, "bits"), _stream(stream)), "skx_select_bitmap")
    return out


def skx_select(bits, n: int, fk, offsets=None, count=None, stream=None):
    """(offsets int32 view of uint32[F], count int64[1]) of the qualifying fact rows, in order."""
    import torch
    if offsets is None:
        offsets = torch.empty(max(fk.numel(), 1), dtype=torch.int32, device=fk.device)
    if count is None:
        count = torch.empty(1, dtype=torch.int64, device=fk.device)
    _check(lib().skx_select(_dptr(bits, "bits"), int(n), _dptr(fk, "fk", torch.int32), fk.numel(),
                            _dptr(offsets, "offsets"), _dptr(count, "count", torch.int64), _stream(stream)),
           "skx_select")
    return offsets, count


def skx_cache_hit_rate(f, S: int) -> float:
    import numpy as np
    f = np.ascontiguousarray(f, dtype=np.float64)
    hit = ctypes.c_double()
    _check(lib().skx_cache_hit_rate(f.ctypes.data_as(ctypes.c_void_p), f.size, int(S), ctypes.byref(hit)),
           "skx_cache_hit_rate")
    return hit.value


def skx_cache_line_cdf(f, S: int):
    """Per-line hit probabilities of the Section III-C model (numpy float64, order of f)."""
    import numpy as np
    f = np.ascontiguousarray(f, dtype=np.float64)
    cdf = np.empty_like(f)
    _check(lib().skx_cache_line_cdf(f.ctypes.data_as(ctypes.c_void_p), f.size, int(S),
                                    cdf.ctypes.data_as(ctypes.c_void_p)), "skx_cache_line_cdf")
    return cdf


def skx_cache_threshold(f, S: int, p: float = 0.5, rows_per_line: int = 1) -> int:
    """Threshold t of Section IV-B from the model: ids below t are likely cache hits."""
    import numpy as np
    f = np.ascontiguousarray(f, dtype=np.float64)
    t = ctypes.c_int64()
    _check(lib().skx_cache_threshold(f.ctypes.data_as(ctypes.c_void_p), f.size, int(S), float(p),
                                     int(rows_per_line), ctypes.byref(t)), "skx_cache_threshold")
    return t.value


def skx_powerlaw_fit(x, y):
    """(slope, intercept) of the least-squares line log y = intercept + slope log x."""
    import numpy as np
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    if x.shape != y.shape:
        raise ValueError("x and y must have the same length")
    b, a = ctypes.c_double(), ctypes.c_double()
    _check(lib().skx_powerlaw_fit(x.ctypes.data_as(ctypes.c_void_p), y.ctypes.data_as(ctypes.c_void_p), x.size,
                                  ctypes.byref(b), ctypes.byref(a)), "skx_powerlaw_fit")
    return b.value, a.value


def skx_index_counts_at_ranks(index: "Index", ranks, stream=None):
    """counts of the ids with the given transformed ids (numpy uint32), gathered on the device."""
    import numpy as np
    r = np.ascontiguousarray(ranks, dtype=np.int64)
    out = np.zeros(r.size, dtype=np.uint32)
    _check(lib().skx_index_counts_at_ranks(index._h, r.ctypes.data_as(ctypes.c_void_p), r.size,
                                           out.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
           "skx_index_counts_at_ranks")
    return out


def skx_join_aggregate_host(rows, fk, measure, query: Query, out=None, stream=None):
    """Whole path from host memory (numpy arrays or CPU tensors, pinned is fastest)."""
    import numpy as np
    import torch

    def hptr(a, what):
        if a is None:
            return None, 0
        if isinstance(a, torch.Tensor):
            if a.is_cuda or not a.is_contiguous():
                raise ValueError(f"{what} must be a contiguous host tensor")
            return ctypes.c_void_p(a.data_ptr()), a
        a = np.ascontiguousarray(a)
        return a.ctypes.data_as(ctypes.c_void_p), a

    prow, rows_keep = hptr(rows, "rows")
    pfk, fk_keep = hptr(fk, "fk")
    pm, m_keep = hptr(measure, "measure")
    n = rows.shape[0]
    row_bytes = (rows.numel() * rows.element_size() if isinstance(rows, torch.Tensor) else rows.nbytes) // n
    nf = fk.numel() if isinstance(fk, torch.Tensor) else np.asarray(fk).size
    if out is None:
        out = np.zeros(query.nout, dtype=np.int64)
    pout, out_keep = hptr(out, "out")
    _check(lib().skx_join_aggregate_host(prow, n, row_bytes, pfk, pm, nf, ctypes.byref(query), pout, _stream(stream)),
           "skx_join_aggregate_host")
    return out_keep
