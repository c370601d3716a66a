"""CPU oracle for the permutation index (TEST INFRASTRUCTURE ONLY).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this package.  The product path (``paper_1910_10063_gb300``) never imports it.

The arithmetic lives in ``skx_oracle.c`` (plain C, compiled with gcc into
``liboracle.so`` next to this file); this module only marshals numpy arrays.
Each function follows one passage of Zhang & Ross, "Exploiting Data Skew for
Improved Query Performance" (ICDE 2020, arXiv 1910.10063):

* ``histogram``          Q3 count per value (Section I; Section III-A, step 1)
* ``sort_by_frequency``  offset representation, values by decreasing frequency
                         (Section III; Section III-A, step 2)
* ``invert``             rank representation (Section III)
* ``build_index``        the three steps above (Section III-A)
* ``remap``              recode C'[i] = Rank(C[i]) (Section III-A, step 3)
* ``reorder``            permuted copy of the dimension rows (Section III-B)
* ``materialize``        Q1: the referenced dimension attribute per fact row
                         (Sections I, IV-A)
* ``probe``              FK gather + filter + aggregation (Sections I, IV-A;
                         threads over fact chunks with independent buffers,
                         Section IV-C)
* ``topk_counts``        Q3a heavy hitters: counts of transformed ids < k
                         (Sections I, IV-B)
* ``select``             Q2: offsets of qualifying fact rows (Sections I, IV-A)
* ``index_append``       maintenance: new rows appended as least frequent
                         (Section III-A)
* ``cache_hit_rate``     the stack-distance cache model (Section III-C)
* ``cache_threshold``    the threshold t of Section IV-B derived from that model
* ``powerlaw_fit``       least-squares line in a log-log plot (Section III-C)

Every function has at least one pin in ``tests/test_oracle_pins.py`` that
does not go through this code (worked example of Fig. 2, brute force, closed
forms, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "skx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EKEY, EGROUP = 0, 1, 3, 4
AGG_COUNT, AGG_SUM, AGG_GROUPBY_SUM = 0, 1, 2


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        names = {EINVAL: "invalid argument", EKEY: "foreign key outside [0, N)",
                 EGROUP: "group key outside [0, G)"}
        super().__init__(f"oracle {what}: {names.get(code, code)}")
        self.code = code


def build(src: str = _SRC, out: str = _LIB, force: bool = False) -> str:
    """Compile the C oracle with gcc (no GPU needed)."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                    "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def load(path: str | None = None):
    """Load (building if needed) the oracle library; returns the ctypes handle."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            build()
            _lib = _declare(ctypes.CDLL(_LIB))
    return _lib


def _declare(lib):
    P = ctypes.c_void_p
    i32, i64, cint = ctypes.c_int32, ctypes.c_int64, ctypes.c_int
    lib.orc_histogram.argtypes = [P, i64, i32, P]
    lib.orc_sort_by_frequency.argtypes = [P, i32, P]
    lib.orc_invert.argtypes = [P, i32, P]
    lib.orc_build_index.argtypes = [P, i64, i32, P, P, P]
    lib.orc_remap.argtypes = [P, i32, P, i64, P]
    lib.orc_reorder.argtypes = [P, i32, P, i32, P]
    lib.orc_probe.argtypes = [P, i32, i32, P, P, i64, cint, cint, i32, cint, i32, cint, P, cint]
    lib.orc_topk_counts.argtypes = [P, i64, i32, P]
    lib.orc_select.argtypes = [P, i32, i32, P, i64, cint, i32, P, P]
    lib.orc_index_append.argtypes = [P, P, i32, i32, P, P]
    lib.orc_cache_hit_rate.argtypes = [P, i64, i64, P, P]
    lib.orc_cache_threshold.argtypes = [P, i64, i64, ctypes.c_double, i32, P]
    lib.orc_powerlaw_fit.argtypes = [P, P, i64, P, P]
    lib.orc_materialize.argtypes = [P, i32, i32, i32, P, i64, P]
    for f in ("orc_histogram", "orc_sort_by_frequency", "orc_invert", "orc_build_index",
              "orc_remap", "orc_reorder", "orc_probe", "orc_topk_counts", "orc_select", "orc_index_append",
              "orc_cache_hit_rate", "orc_cache_threshold", "orc_powerlaw_fit", "orc_materialize"):
        getattr(lib, f).restype = cint
    return lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def histogram(fk, n: int, lib=None) -> np.ndarray:
    lib = lib or load()
    fk = _c(fk, np.int32)
    cnt = np.zeros(n, dtype=np.uint64)
    st = lib.orc_histogram(_ptr(fk), fk.shape[0], n, _ptr(cnt))
    if st:
        raise OracleError(st, "histogram")
    return cnt


def sort_by_frequency(cnt, lib=None) -> np.ndarray:
    lib = lib or load()
    cnt = _c(cnt, np.uint64)
    perm = np.zeros(cnt.shape[0], dtype=np.int32)
    st = lib.orc_sort_by_frequency(_ptr(cnt), cnt.shape[0], _ptr(perm))
    if st:
        raise OracleError(st, "sort_by_frequency")
    return perm


def invert(perm, lib=None) -> np.ndarray:
    lib = lib or load()
    perm = _c(perm, np.int32)
    rank = np.zeros(perm.shape[0], dtype=np.int32)
    st = lib.orc_invert(_ptr(perm), perm.shape[0], _ptr(rank))
    if st:
        raise OracleError(st, "invert")
    return rank


def build_index(fk, n: int, lib=None):
    """Returns (cnt uint64[n], perm int32[n] new->old, rank int32[n] old->new)."""
    lib = lib or load()
    fk = _c(fk, np.int32)
    cnt = np.zeros(n, dtype=np.uint64)
    perm = np.zeros(n, dtype=np.int32)
    rank = np.zeros(n, dtype=np.int32)
    st = lib.orc_build_index(_ptr(fk), fk.shape[0], n, _ptr(cnt), _ptr(perm), _ptr(rank))
    if st:
        raise OracleError(st, "build_index")
    return cnt, perm, rank


def remap(rank, fk, lib=None) -> np.ndarray:
    lib = lib or load()
    rank = _c(rank, np.int32)
    fk = _c(fk, np.int32)
    out = np.empty_like(fk)
    st = lib.orc_remap(_ptr(rank), rank.shape[0], _ptr(fk), fk.shape[0], _ptr(out))
    if st:
        raise OracleError(st, "remap")
    return out


def reorder(perm, rows, lib=None) -> np.ndarray:
    """rows: array whose first axis is the dimension row (any dtype/shape per row)."""
    lib = lib or load()
    perm = _c(perm, np.int32)
    rows = np.ascontiguousarray(rows)
    out = np.empty_like(rows)
    row_bytes = rows.nbytes // max(rows.shape[0], 1)
    st = lib.orc_reorder(_ptr(perm), perm.shape[0], _ptr(rows), row_bytes, _ptr(out))
    if st:
        raise OracleError(st, "reorder")
    return out


def probe(rows, fk, measure, agg: int = AGG_GROUPBY_SUM, filter_col: int = 1,
          filter_lt: int = 50, group_col: int = 0, num_groups: int = 1000,
          payload_col: int = 2, nthreads: int = 1, lib=None) -> np.ndarray:
    """int64 result: [num_groups] for GROUPBY_SUM, [1] for COUNT and SUM.

    Sums wrap modulo 2^64 (computed as uint64, returned reinterpreted as int64)."""
    lib = lib or load()
    rows = _c(rows, np.int32)
    if rows.ndim != 2:
        raise ValueError("rows must be int32[N, W]")
    fk = _c(fk, np.int32)
    measure = None if measure is None else _c(measure, np.int32)
    nout = num_groups if agg == AGG_GROUPBY_SUM else 1
    out = np.zeros(nout, dtype=np.uint64)
    st = lib.orc_probe(_ptr(rows), rows.shape[0], rows.shape[1], _ptr(fk), _ptr(measure),
                       fk.shape[0], agg, filter_col, filter_lt, group_col, num_groups,
                       payload_col, _ptr(out), nthreads)
    if st:
        raise OracleError(st, "probe")
    return out.view(np.int64)


def topk_counts(fk_remapped, k: int, lib=None) -> np.ndarray:
    lib = lib or load()
    fk = _c(fk_remapped, np.int32)
    out = np.zeros(k, dtype=np.uint64)
    st = lib.orc_topk_counts(_ptr(fk), fk.shape[0], k, _ptr(out))
    if st:
        raise OracleError(st, "topk_counts")
    return out


def select(rows, fk, filter_col: int = 1, filter_lt: int = 50, lib=None) -> np.ndarray:
    """uint32 offsets (increasing) of the fact rows whose dimension row passes col < c."""
    lib = lib or load()
    rows = _c(rows, np.int32)
    fk = _c(fk, np.int32)
    offs = np.zeros(max(fk.shape[0], 1), dtype=np.uint32)
    cnt = np.zeros(1, dtype=np.int64)
    st = lib.orc_select(_ptr(rows), rows.shape[0], rows.shape[1], _ptr(fk), fk.shape[0], filter_col, filter_lt,
                        _ptr(offs), _ptr(cnt))
    if st:
        raise OracleError(st, "select")
    return offs[:int(cnt[0])].copy()


def index_append(perm, rank, n_new: int, lib=None):
    lib = lib or load()
    perm = _c(perm, np.int32)
    rank = _c(rank, np.int32)
    n = perm.shape[0]
    po = np.zeros(n + n_new, dtype=np.int32)
    ro = np.zeros(n + n_new, dtype=np.int32)
    st = lib.orc_index_append(_ptr(perm), _ptr(rank), n, n_new, _ptr(po), _ptr(ro))
    if st:
        raise OracleError(st, "index_append")
    return po, ro


def cache_hit_rate(f, S: int, lib=None):
    """(hit rate, cdf per line) of the Section III-C model for line frequencies f and S lines."""
    lib = lib or load()
    f = _c(f, np.float64)
    hit = np.zeros(1, dtype=np.float64)
    cdf = np.zeros(f.shape[0], dtype=np.float64)
    st = lib.orc_cache_hit_rate(_ptr(f), f.shape[0], S, _ptr(hit), _ptr(cdf))
    if st:
        raise OracleError(st, "cache_hit_rate")
    return float(hit[0]), cdf


def cache_threshold(f, S: int, p: float, rows_per_line: int, lib=None) -> int:
    """Threshold t (ids below it likely cache hits) for lines f in transformed-id order."""
    lib = lib or load()
    f = _c(f, np.float64)
    t = np.zeros(1, dtype=np.int64)
    st = lib.orc_cache_threshold(_ptr(f), f.shape[0], S, float(p), rows_per_line, _ptr(t))
    if st:
        raise OracleError(st, "cache_threshold")
    return int(t[0])


def powerlaw_fit(x, y, lib=None):
    """(slope, intercept) of the least-squares line log y = intercept + slope log x."""
    lib = lib or load()
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    out = np.zeros(2, dtype=np.float64)
    st = lib.orc_powerlaw_fit(_ptr(x), _ptr(y), x.shape[0], _ptr(out[:1]), _ptr(out[1:]))
    if st:
        raise OracleError(st, "powerlaw_fit")
    return float(out[0]), float(out[1])


def materialize(rows, fk, col: int, lib=None) -> np.ndarray:
    """Q1: int32 out[i] = rows[fk[i]][col] (rows: int32[N, W])."""
    lib = lib or load()
    rows = _c(rows, np.int32)
    if rows.ndim != 2:
        raise ValueError("rows must be int32[N, W]")
    fk = _c(fk, np.int32)
    out = np.zeros(fk.shape[0], dtype=np.int32)
    st = lib.orc_materialize(_ptr(rows), rows.shape[0], rows.shape[1], col, _ptr(fk), fk.shape[0], _ptr(out))
    if st:
        raise OracleError(st, "materialize")
    return out
