"""Seeded synthetic inputs for the permutation-index workloads.

This module only *makes inputs*: it holds none of the permutation index's
arithmetic (no counting, sorting, remapping or joining).  Both the CUDA path
and the CPU oracle consume what it produces, so it is the one piece of code
the two share.

Every value is a pure function of ``(seed, stream, index)`` through a
counter-based generator, so any element of a billion-row column can be
recomputed on the host without generating the rest.  The device generator
(``synth.cu``, loaded as ``libskx_synth.so``) implements the same definitions
and is tested equal to the host twin below.

Definitions
-----------
* ``mix64`` is the SplitMix64 output function (Steele, Lea & Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014; constants as
  published by Vigna).  Element ``i`` of a stream with key ``k`` is
  ``mix64(k + (i + 1) * GAMMA)`` with ``GAMMA = 0x9E3779B97F4A7C15``.
* Stream keys: ``key(seed, stream) = mix64(mix64(seed) ^ (stream * GAMMA))``.
* Unit uniform: ``u = (x >> 11) * 2**-53`` (53 exact bits, ``0 <= u < 1``).
* Bounded integer in ``[lo, lo + range)``: ``lo + (((x >> 32) * range) >> 32)``
  (multiply-shift on the high 32 bits).  ``range == 0`` means the full int32
  range: ``int32(x >> 32)``.
* Zipf(s) over ranks ``0..N-1`` (the paper's skew model, Section II-A: the
  item of rank r has frequency proportional to r^-s, ranks counted from 1):
  ``cdf[r] = (sum_{j<=r} (j+1)^-s) / (sum_{j<N} (j+1)^-s)`` built once on the
  host in float64 with a sequential cumulative sum (``cdf[N-1] == 1``), and a
  draw is the rank ``r = min{r : cdf[r] > u}``.  Ranks are mapped to ids by a
  seeded random permutation ``rank_to_id`` (the paper draws keys "in random
  order", Section V-A), so popular ids are scattered over the dimension.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1

# stream ids (one independent counter stream per column family)
STREAM_FK = 1
STREAM_MEASURE = 2
STREAM_DIM = 3
STREAM_SHUFFLE = 4
STREAM_DRIFT = 5

# Column value ranges of the synthetic dimension table: (lo, range); range 0 = full int32.
#   col 0 attr0    uniform [0, 1000)   group key
#   col 1 attr1    uniform [0, 100)    filter column (attr1 < 50)
#   col 2 payload0 uniform [0, 1e6)
#   col 3 payload1 uniform [0, 1e6)
#   col 4.. filler uniform int32
def dim_column_ranges(width: int, num_groups: int = 1000):
    base = [(0, num_groups), (0, 100), (0, 1_000_000), (0, 1_000_000)]
    cols = base[:width] + [(0, 0)] * max(0, width - 4)
    return cols


def mix64_scalar(z: int) -> int:
    z &= _MASK
    z ^= z >> 30
    z = (z * _M1) & _MASK
    z ^= z >> 27
    z = (z * _M2) & _MASK
    z ^= z >> 31
    return z


def stream_key(seed: int, stream: int) -> int:
    return mix64_scalar(mix64_scalar(seed) ^ ((stream * GAMMA) & _MASK))


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= np.uint64(_M1)
    z ^= z >> np.uint64(27)
    z *= np.uint64(_M2)
    z ^= z >> np.uint64(31)
    return z


def raw_draws(key: int, start: int, count: int) -> np.ndarray:
    """uint64 draws ``mix64(key + (i+1)*GAMMA)`` for i in [start, start+count)."""
    i = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (i + np.uint64(1)) * np.uint64(GAMMA)
        return _mix64(z)


def raw_draws_at(key: int, idx: np.ndarray) -> np.ndarray:
    i = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (i + np.uint64(1)) * np.uint64(GAMMA)
        return _mix64(z)


def bounded(x: np.ndarray, lo: int, rng: int) -> np.ndarray:
    """Map uint64 draws to int32 values in [lo, lo+rng) (rng == 0: full int32)."""
    hi32 = x >> np.uint64(32)
    if rng == 0:
        return hi32.astype(np.uint32).view(np.int32)
    with np.errstate(over="ignore"):
        v = (hi32 * np.uint64(rng)) >> np.uint64(32)
    return (v.astype(np.int64) + lo).astype(np.int32)


def unit_uniform(x: np.ndarray) -> np.ndarray:
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ---------------------------------------------------------------- Zipf tables
def zipf_cdf(n: int, s: float) -> np.ndarray:
    """float64 CDF over ranks 0..n-1 with weights (r+1)^-s (Section II-A)."""
    if n <= 0:
        raise ValueError("n must be positive")
    w = np.arange(1, n + 1, dtype=np.float64)
    if s == 0.0:
        w[:] = 1.0
    else:
        np.power(w, -float(s), out=w)
    c = np.cumsum(w)  # sequential, so the table is reproducible
    c /= c[-1]
    c[-1] = 1.0
    return c


def rank_to_id(n: int, seed: int) -> np.ndarray:
    """Seeded random bijection rank -> dimension id (int32)."""
    g = np.random.Generator(np.random.PCG64(stream_key(seed, STREAM_SHUFFLE)))
    return g.permutation(n).astype(np.int32)


def drift_rank_to_id(r2id: np.ndarray, seed: int, fraction: float = 0.1) -> np.ndarray:
    """Re-shuffle the ids held by a seeded `fraction` of rank positions.

    Used for the drifting-popularity variant: the popularity of 10% of the keys
    changes, the rest keep their rank."""
    n = r2id.shape[0]
    g = np.random.Generator(np.random.PCG64(stream_key(seed, STREAM_DRIFT)))
    k = int(round(n * fraction))
    pos = np.sort(g.choice(n, size=k, replace=False))
    out = r2id.copy()
    out[pos] = r2id[pos][g.permutation(k)]
    return out


# ---------------------------------------------------------------- host twin
def zipf_fk_host(cdf: np.ndarray, r2id: np.ndarray, seed: int, start: int, count: int) -> np.ndarray:
    u = unit_uniform(raw_draws(stream_key(seed, STREAM_FK), start, count))
    r = np.searchsorted(cdf, u, side="right")
    return r2id[r]


def zipf_fk_host_at(cdf, r2id, seed, idx) -> np.ndarray:
    u = unit_uniform(raw_draws_at(stream_key(seed, STREAM_FK), idx))
    return r2id[np.searchsorted(cdf, u, side="right")]


def measure_host(seed: int, start: int, count: int, lo: int = 1, rng: int = 100) -> np.ndarray:
    return bounded(raw_draws(stream_key(seed, STREAM_MEASURE), start, count), lo, rng)


def measure_host_at(seed: int, idx, lo: int = 1, rng: int = 100) -> np.ndarray:
    return bounded(raw_draws_at(stream_key(seed, STREAM_MEASURE), idx), lo, rng)


def dim_rows_host(n: int, width: int, seed: int, num_groups: int = 1000,
                  start: int = 0, count: int | None = None) -> np.ndarray:
    """int32[count, width] dimension rows start..start+count-1."""
    if count is None:
        count = n - start
    key = stream_key(seed, STREAM_DIM)
    out = np.empty((count, width), dtype=np.int32)
    base = np.arange(start, start + count, dtype=np.uint64) * np.uint64(width)
    for c, (lo, rng) in enumerate(dim_column_ranges(width, num_groups)):
        out[:, c] = bounded(raw_draws_at(key, base + np.uint64(c)), lo, rng)
    return out


def dim_rows_host_at(idx, width: int, seed: int, num_groups: int = 1000) -> np.ndarray:
    idx = np.asarray(idx, dtype=np.uint64)
    key = stream_key(seed, STREAM_DIM)
    out = np.empty((idx.shape[0], width), dtype=np.int32)
    for c, (lo, rng) in enumerate(dim_column_ranges(width, num_groups)):
        out[:, c] = bounded(raw_draws_at(key, idx * np.uint64(width) + np.uint64(c)), lo, rng)
    return out


class Workload:
    """One star-schema instance: dimension table, Zipf FK column and measure."""

    def __init__(self, n: int, f: int, s: float, seed: int = 0, width: int = 4,
                 num_groups: int = 1000, r2id: np.ndarray | None = None):
        self.n, self.f, self.s, self.seed = int(n), int(f), float(s), int(seed)
        self.width, self.num_groups = int(width), int(num_groups)
        self.cdf = zipf_cdf(self.n, self.s)
        self.r2id = rank_to_id(self.n, self.seed) if r2id is None else r2id

    def fk(self) -> np.ndarray:
        return zipf_fk_host(self.cdf, self.r2id, self.seed, 0, self.f)

    def measure(self) -> np.ndarray:
        return measure_host(self.seed, 0, self.f)

    def dim(self) -> np.ndarray:
        return dim_rows_host(self.n, self.width, self.seed, self.num_groups)


def lognormal_sizes(count: int, seed: int, median: float = 2e5, sigma: float = 1.5,
                    lo: int = 1000, hi: int = 20_000_000) -> np.ndarray:
    """Per-query fact-batch sizes: clip(round(median * exp(sigma * Z)), lo, hi)."""
    g = np.random.Generator(np.random.PCG64(stream_key(seed, 6)))
    z = g.standard_normal(count)
    return np.clip(np.round(median * np.exp(sigma * z)), lo, hi).astype(np.int64)


# ---------------------------------------------------------------- device twin
_dev_lib = None


def _synth_lib():
    """libskx_synth.so (the CUDA twin of the functions above)."""
    global _dev_lib
    if _dev_lib is None:
        import ctypes
        import os
        path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "libskx_synth.so")
        if not os.path.exists(path):
            raise RuntimeError(f"libskx_synth.so is not built at {path}; run `python -m paper_1910_10063_gb300.build`")
        L = ctypes.CDLL(path)
        P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        L.skx_synth_zipf.argtypes = [P, P, i32, u64, i64, i64, P, P]
        L.skx_synth_uniform.argtypes = [u64, i64, i64, i32, ctypes.c_uint32, P, P]
        L.skx_synth_rows.argtypes = [u64, i64, i32, P, P, P, P]
        for f in ("skx_synth_zipf", "skx_synth_uniform", "skx_synth_rows"):
            getattr(L, f).restype = ctypes.c_int
        _dev_lib = L
    return _dev_lib


def _stream_ptr(stream):
    import ctypes
    import torch
    stream = stream or torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def zipf_fk_device(d_cdf, d_r2id, seed: int, count: int, start: int = 0, out=None, stream=None):
    """int32 CUDA tensor of `count` Zipf FKs, elements start..start+count-1 of the stream."""
    import ctypes
    import torch
    if out is None:
        out = torch.empty(count, dtype=torch.int32, device=d_cdf.device)
    st = _synth_lib().skx_synth_zipf(ctypes.c_void_p(d_cdf.data_ptr()), ctypes.c_void_p(d_r2id.data_ptr()),
                                     d_cdf.numel(), stream_key(seed, STREAM_FK), start, count,
                                     ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))
    if st:
        raise RuntimeError(f"skx_synth_zipf failed ({st})")
    return out


def measure_device(seed: int, count: int, start: int = 0, lo: int = 1, rng: int = 100, out=None, device="cuda",
                   stream=None):
    import ctypes
    import torch
    if out is None:
        out = torch.empty(count, dtype=torch.int32, device=device)
    st = _synth_lib().skx_synth_uniform(stream_key(seed, STREAM_MEASURE), start, count, lo, rng,
                                        ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))
    if st:
        raise RuntimeError(f"skx_synth_uniform failed ({st})")
    return out


def dim_rows_device(n: int, width: int, seed: int, num_groups: int = 1000, out=None, device="cuda", stream=None):
    import ctypes
    import torch
    cols = dim_column_ranges(width, num_groups)
    lo = np.array([c[0] for c in cols], dtype=np.int32)
    rg = np.array([c[1] for c in cols], dtype=np.uint32)
    if out is None:
        out = torch.empty((n, width), dtype=torch.int32, device=device)
    st = _synth_lib().skx_synth_rows(stream_key(seed, STREAM_DIM), n, width, lo.ctypes.data_as(ctypes.c_void_p),
                                     rg.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(out.data_ptr()),
                                     _stream_ptr(stream))
    if st:
        raise RuntimeError(f"skx_synth_rows failed ({st})")
    return out


class DeviceWorkload:
    """A Workload generated on the device (same values as the host twin)."""

    def __init__(self, n: int, f: int, s: float, seed: int = 0, width: int = 16, num_groups: int = 1000,
                 r2id: np.ndarray | None = None, device="cuda", with_measure: bool = True,
                 with_dim: bool = True):
        import torch
        self.n, self.f, self.s, self.seed, self.width = int(n), int(f), float(s), int(seed), int(width)
        self.num_groups = num_groups
        self.r2id_host = rank_to_id(self.n, self.seed) if r2id is None else r2id
        cdf = zipf_cdf(self.n, self.s)
        self.cdf = torch.from_numpy(cdf).to(device)
        self.r2id = torch.from_numpy(self.r2id_host).to(device)
        self.fk = zipf_fk_device(self.cdf, self.r2id, self.seed, self.f)
        self.measure = measure_device(self.seed, self.f, device=device) if with_measure else None
        self.dim = dim_rows_device(self.n, self.width, self.seed, num_groups, device=device) if with_dim else None
