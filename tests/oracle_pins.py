"""Pins of the CPU oracle against things other than itself.

Each ``pin_*`` function takes a loaded oracle library (``oracle.load()`` or a
deliberately broken copy) and raises AssertionError when the oracle disagrees
with the paper's worked example, a brute-force definition, a closed form or
an invariant.  ``test_oracle_pins.py`` runs them on the real oracle;
``test_oracle_mutations.py`` runs them on mutants and expects failures.
"""
from __future__ import annotations

import collections
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
MOD64 = 1 << 64


def _signed64(x: int) -> int:
    x %= MOD64
    return x - MOD64 if x >= (1 << 63) else x


def load_fig2():
    fields = {}
    with open(os.path.join(GOLDEN, "fig2_permutation_example.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            fields[k.strip()] = v.split()
    return fields


# ------------------------------------------------------------------ Fig. 2
def pin_fig2_example(lib):
    """Section III / III-B worked example: order 5,1,8,4,... and rows E,A,H,D,C,G,F,B."""
    g = load_fig2()
    order = [int(x) - 1 for x in g["offset_order"]]  # 0-based ids, most frequent first
    names = g["dimension_rows"]
    n = len(names)
    # a fact column whose counts strictly decrease along `order`, rows shuffled
    fk = np.concatenate([np.full(n - r, v, dtype=np.int32) for r, v in enumerate(order)])
    fk = fk[np.random.default_rng(7).permutation(fk.shape[0])]
    cnt, perm, rank = oracle.build_index(fk, n, lib=lib)
    assert list(perm) == order, (list(perm), order)
    rows = np.array([[ord(c)] for c in names], dtype=np.int32)
    reordered = oracle.reorder(perm, rows, lib=lib)
    assert [chr(int(x)) for x in reordered[:, 0]] == g["reordered_rows"]
    # rank representation (Fig. 2b): popularity rank stored per dimension row
    assert [int(rank[v]) for v in order] == list(range(n))
    fk2 = oracle.remap(rank, fk, lib=lib)
    # the most frequent value becomes offset 0 (1 in the paper's 1-based text)
    assert collections.Counter(fk2.tolist()).most_common(1)[0][0] == 0
    assert np.array_equal(perm[fk2], fk)


# ------------------------------------------------------------------ histogram
def pin_histogram(lib):
    rng = np.random.default_rng(1)
    for n, f in [(1, 0), (1, 5), (7, 100), (64, 1000), (1000, 333)]:
        fk = rng.integers(0, n, size=f, dtype=np.int32)
        cnt = oracle.histogram(fk, n, lib=lib)
        brute = collections.Counter(fk.tolist())
        assert [int(c) for c in cnt] == [brute.get(v, 0) for v in range(n)]
        assert int(cnt.sum()) == f
    # closed form: fk[i] = i mod N
    n, f = 97, 10_001
    cnt = oracle.histogram(np.arange(f, dtype=np.int64) % n, n, lib=lib)
    expect = [f // n + (1 if v < f % n else 0) for v in range(n)]
    assert [int(c) for c in cnt] == expect
    # all rows the same key
    cnt = oracle.histogram(np.full(500, 3, dtype=np.int32), 10, lib=lib)
    assert int(cnt[3]) == 500 and int(cnt.sum()) == 500
    # key outside [0, N) is an error, not a silent count
    for bad in (-1, 10):
        fk = np.array([0, 1, bad], dtype=np.int32)
        try:
            oracle.histogram(fk, 10, lib=lib)
        except oracle.OracleError as e:
            assert e.code == oracle.EKEY
        else:
            raise AssertionError("out-of-range key not reported")


# ------------------------------------------------------------------ sort + invert
def pin_sort_by_frequency(lib):
    rng = np.random.default_rng(2)
    for n in (1, 2, 5, 33, 64):
        cnt = rng.integers(0, 4, size=n).astype(np.uint64)  # many ties
        perm = oracle.sort_by_frequency(cnt, lib=lib)
        assert sorted(perm.tolist()) == list(range(n))
        # O(N^2) pairwise: every earlier id has larger count, or equal count and smaller id
        pos = {int(v): r for r, v in enumerate(perm)}
        for a in range(n):
            for b in range(n):
                if pos[a] < pos[b]:
                    assert cnt[a] > cnt[b] or (cnt[a] == cnt[b] and a < b)
        # Python's own sort with the same ordering key
        assert perm.tolist() == sorted(range(n), key=lambda v: (-int(cnt[v]), v))
    # all counts equal -> identity; strictly increasing counts -> reversed ids
    assert oracle.sort_by_frequency(np.full(9, 4, dtype=np.uint64), lib=lib).tolist() == list(range(9))
    assert oracle.sort_by_frequency(np.arange(9, dtype=np.uint64), lib=lib).tolist() == list(range(8, -1, -1))
    # counts beyond 32 bits keep their order
    big = np.array([1 << 40, (1 << 40) + 1, 5], dtype=np.uint64)
    assert oracle.sort_by_frequency(big, lib=lib).tolist() == [1, 0, 2]


def pin_invert(lib):
    rng = np.random.default_rng(3)
    for n in (1, 2, 17, 1000):
        perm = rng.permutation(n).astype(np.int32)
        rank = oracle.invert(perm, lib=lib)
        assert np.array_equal(rank, np.argsort(perm))  # inverse permutation = argsort
        assert np.array_equal(rank[perm], np.arange(n))


# ------------------------------------------------------------------ remap + reorder
def pin_remap(lib):
    rng = np.random.default_rng(4)
    n, f = 50, 2000
    fk = (rng.zipf(1.3, size=f) % n).astype(np.int32)
    cnt, perm, rank = oracle.build_index(fk, n, lib=lib)
    fk2 = oracle.remap(rank, fk, lib=lib)
    assert np.array_equal(perm[fk2], fk)          # C'[i] names the same row as C[i]
    h2 = collections.Counter(fk2.tolist())
    h2 = np.array([h2.get(r, 0) for r in range(n)])
    assert np.array_equal(h2, cnt[perm].astype(np.int64))
    assert np.all(np.diff(h2) <= 0)                # new ids are frequency ranks
    try:
        oracle.remap(rank, np.array([n], dtype=np.int32), lib=lib)
    except oracle.OracleError as e:
        assert e.code == oracle.EKEY
    else:
        raise AssertionError("out-of-range key not reported")


def pin_reorder(lib):
    rng = np.random.default_rng(5)
    for n, w in [(1, 1), (8, 3), (100, 4), (257, 16)]:
        rows = rng.integers(-2**31, 2**31 - 1, size=(n, w), dtype=np.int64).astype(np.int32)
        perm = rng.permutation(n).astype(np.int32)
        out = oracle.reorder(perm, rows, lib=lib)
        assert out.tobytes() == rows[perm].tobytes()
        assert sorted(map(bytes, out)) == sorted(map(bytes, rows))  # multiset of rows kept


# ------------------------------------------------------------------ probe
def brute_force_join(rows, fk, measure, agg, filter_col, filter_lt, group_col, G, payload_col):
    """Nested-loop FK join in Python integers: for every fact row, every dimension row."""
    n = len(rows)
    out = [0] * (G if agg == oracle.AGG_GROUPBY_SUM else 1)
    for i in range(len(fk)):
        for v in range(n):
            if v != int(fk[i]):
                continue
            row = [int(x) for x in rows[v]]
            if filter_col >= 0 and not row[filter_col] < filter_lt:
                continue
            if agg == oracle.AGG_COUNT:
                out[0] += 1
                continue
            p = row[payload_col] if payload_col >= 0 else 1
            prod = int(measure[i]) * p
            if agg == oracle.AGG_SUM:
                out[0] += prod
            else:
                out[row[group_col]] += prod
    return [_signed64(x) for x in out]


def pin_probe_brute_force(lib):
    rng = np.random.default_rng(6)
    for trial in range(6):
        n, f, G = int(rng.integers(1, 12)), int(rng.integers(0, 60)), int(rng.integers(1, 6))
        rows = np.stack([rng.integers(0, G, n), rng.integers(0, 10, n),
                         rng.integers(-1000, 1000, n), rng.integers(0, 9, n)], axis=1).astype(np.int32)
        fk = rng.integers(0, n, f).astype(np.int32)
        m = rng.integers(-50, 100, f).astype(np.int32)
        for agg in (oracle.AGG_COUNT, oracle.AGG_SUM, oracle.AGG_GROUPBY_SUM):
            for fcol, flt, pcol in [(1, 5, 2), (-1, 0, 2), (3, 4, 3), (1, 7, -1)]:
                got = oracle.probe(rows, fk, m, agg, fcol, flt, 0, G, pcol, nthreads=1 + trial % 3, lib=lib)
                want = brute_force_join(rows, fk, m, agg, fcol, flt, 0, G, pcol)
                assert got.tolist() == want, (trial, agg, fcol, got.tolist(), want)


def pin_probe_closed_forms(lib):
    rng = np.random.default_rng(8)
    n, f, G = 300, 5000, 7
    rows = np.stack([rng.integers(0, G, n), rng.integers(0, 100, n),
                     rng.integers(0, 10**6, n), rng.integers(0, 10**6, n)], axis=1).astype(np.int32)
    fk = (rng.zipf(1.2, f) % n).astype(np.int32)
    m = rng.integers(1, 101, f).astype(np.int32)
    # filter always true, measure = payload = 1, one group  =>  SUM = F
    ones = rows.copy(); ones[:, 0] = 0; ones[:, 2] = 1
    one_m = np.ones(f, dtype=np.int32)
    assert oracle.probe(ones, fk, one_m, oracle.AGG_SUM, 1, 1000, 0, 1, 2, lib=lib).tolist() == [f]
    assert oracle.probe(ones, fk, one_m, oracle.AGG_GROUPBY_SUM, 1, 1000, 0, 1, 2, lib=lib).tolist() == [f]
    # COUNT = sum of counts of the ids that pass the filter
    c = collections.Counter(fk.tolist())
    want = sum(c.get(v, 0) for v in range(n) if rows[v, 1] < 50)
    assert oracle.probe(rows, fk, m, oracle.AGG_COUNT, 1, 50, 0, G, 2, lib=lib).tolist() == [want]
    # strict "<": rows equal to the constant are excluded
    eq = rows.copy(); eq[:, 1] = 50
    assert oracle.probe(eq, fk, m, oracle.AGG_COUNT, 1, 50, 0, G, 2, lib=lib).tolist() == [0]
    # per-group sums add up to the ungrouped sum; one group equals SUM
    gsum = oracle.probe(rows, fk, m, oracle.AGG_GROUPBY_SUM, 1, 50, 0, G, 2, lib=lib)
    s = oracle.probe(rows, fk, m, oracle.AGG_SUM, 1, 50, 0, G, 2, lib=lib)
    assert int(gsum.sum()) == int(s[0])
    # SUM(measure * payload) = sum_v payload[v] * (sum of measures of rows with fk = v)
    msum = collections.defaultdict(int)
    for i in range(f):
        msum[int(fk[i])] += int(m[i])
    want = sum(int(rows[v, 2]) * msum[v] for v in msum if rows[v, 1] < 50)
    assert int(s[0]) == want
    # thread count does not change the result
    for t in (2, 3, 16):
        assert np.array_equal(oracle.probe(rows, fk, m, nthreads=t, num_groups=G, lib=lib),
                              oracle.probe(rows, fk, m, nthreads=1, num_groups=G, lib=lib))


def pin_probe_wraparound(lib):
    """Products in int64, sums modulo 2^64 (reported as int64)."""
    big = 2**31 - 1
    rows = np.array([[0, 0, big, 0], [0, 0, -big - 1, 0]], dtype=np.int32)
    fk = np.array([0] * 6 + [1] * 3, dtype=np.int32)
    m = np.array([big] * 6 + [-big - 1] * 3, dtype=np.int32)
    got = oracle.probe(rows, fk, m, oracle.AGG_SUM, 1, 1, 0, 1, 2, lib=lib)
    want = _signed64(6 * big * big + 3 * (big + 1) * (big + 1))
    assert got.tolist() == [want]


def pin_probe_layout_invariance(lib):
    """Result on (dim, fk) equals result on (dim', fk') -- Section III-B."""
    rng = np.random.default_rng(9)
    n, f, G = 2000, 20000, 11
    rows = np.stack([rng.integers(0, G, n), rng.integers(0, 100, n),
                     rng.integers(0, 10**6, n), rng.integers(0, 10**6, n)], axis=1).astype(np.int32)
    fk = (rng.zipf(1.1, f) % n).astype(np.int32)
    m = rng.integers(1, 101, f).astype(np.int32)
    cnt, perm, rank = oracle.build_index(fk, n, lib=lib)
    rows2 = oracle.reorder(perm, rows, lib=lib)
    fk2 = oracle.remap(rank, fk, lib=lib)
    for agg in (oracle.AGG_COUNT, oracle.AGG_SUM, oracle.AGG_GROUPBY_SUM):
        a = oracle.probe(rows, fk, m, agg, 1, 50, 0, G, 2, lib=lib)
        b = oracle.probe(rows2, fk2, m, agg, 1, 50, 0, G, 2, lib=lib)
        assert np.array_equal(a, b)


def pin_probe_errors(lib):
    rows = np.array([[0, 0, 1, 1], [5, 0, 1, 1]], dtype=np.int32)
    m = np.ones(2, dtype=np.int32)
    for fk, code in [(np.array([0, 2], dtype=np.int32), oracle.EKEY),
                     (np.array([0, 1], dtype=np.int32), oracle.EGROUP)]:
        try:
            oracle.probe(rows, fk, m, oracle.AGG_GROUPBY_SUM, 1, 10, 0, 3, 2, lib=lib)
        except oracle.OracleError as e:
            assert e.code == code
        else:
            raise AssertionError("error not reported")


# ------------------------------------------------------------------ Q3a, Q2, maintenance, cache model
def pin_topk_counts(lib):
    rng = np.random.default_rng(10)
    n, f, k = 3000, 50_000, 100
    fk = (rng.zipf(1.2, f) % n).astype(np.int32)
    cnt, perm, rank = oracle.build_index(fk, n, lib=lib)
    fk2 = oracle.remap(rank, fk, lib=lib)
    top = oracle.topk_counts(fk2, k, lib=lib)
    c = collections.Counter(fk2.tolist())
    assert [int(x) for x in top] == [c.get(r, 0) for r in range(k)]   # brute force
    assert np.array_equal(top, cnt[perm[:k]])                          # ranks < k are the k most frequent
    assert np.all(np.diff(top.astype(np.int64)) <= 0)
    assert oracle.topk_counts(np.array([-1, 5, 2, 2], dtype=np.int32), 3, lib=lib).tolist() == [0, 0, 2]


def pin_select(lib):
    rng = np.random.default_rng(11)
    n, f = 40, 500
    rows = np.stack([rng.integers(0, 5, n), rng.integers(0, 10, n)], axis=1).astype(np.int32)
    fk = rng.integers(0, n, f).astype(np.int32)
    for c in (0, 3, 5, 10):
        got = oracle.select(rows, fk, 1, c, lib=lib)
        want = [i for i in range(f) if rows[fk[i], 1] < c]
        assert got.tolist() == want
        count = oracle.probe(rows, fk, None, oracle.AGG_COUNT, 1, c, 0, 1, -1, lib=lib)
        assert int(count[0]) == len(want)                              # Q2 count == COUNT query
    eq = rows.copy(); eq[:, 1] = 3
    assert oracle.select(eq, fk, 1, 3, lib=lib).size == 0              # strict "<"


def pin_index_append(lib):
    rng = np.random.default_rng(12)
    perm = rng.permutation(50).astype(np.int32)
    rank = np.argsort(perm).astype(np.int32)
    p2, r2 = oracle.index_append(perm, rank, 7, lib=lib)
    assert p2.tolist() == perm.tolist() + list(range(50, 57))
    assert np.array_equal(r2[p2], np.arange(57))
    assert np.array_equal(r2[:50], rank)


def _lru_hit_rate(p, S, n_acc, seed):
    rng = np.random.default_rng(seed)
    acc = rng.choice(p.size, size=n_acc, p=p)
    od, hits = collections.OrderedDict(), 0
    for a in acc.tolist():
        if a in od:
            hits += 1
            od.move_to_end(a)
        else:
            od[a] = None
            if len(od) > S:
                od.popitem(last=False)
    return hits / n_acc


def pin_cache_model(lib):
    # S = 1: d(1) = 1 for every line, so K = 1 and the model is exact LRU: sum of f_i^2
    f = np.array([0.5, 0.3, 0.15, 0.05])
    hit, cdf = oracle.cache_hit_rate(f, 1, lib=lib)
    assert abs(hit - float(np.sum(f * f))) < 1e-12 and np.allclose(cdf, f)
    # uniform lines: n_j <= 1 up to k = L - 1, so K = S and hit = 1 - (1 - 1/L)^S
    for L, S in ((100, 50), (1000, 10), (64, 63)):
        hit, _ = oracle.cache_hit_rate(np.full(L, 1.0 / L), S, lib=lib)
        assert abs(hit - (1 - (1 - 1.0 / L) ** S)) < 1e-12
    # worked by hand: f = (0.9, 0.07, 0.015, 0.01, 0.005), S = 3.  Hot line: n_j = k f_j / 0.1 =
    # k (0.7, 0.15, 0.1, 0.05), so d(6) = 6 - 3.2 = 2.8 < 3 <= d(7) = 7 - 3.9 - 0.05 = 3.05 -> K = 7.
    _, cdf = oracle.cache_hit_rate(np.array([0.9, 0.07, 0.015, 0.01, 0.005]), 3, lib=lib)
    assert abs(cdf[0] - (1 - 0.1 ** 7)) < 1e-12
    # a cache holding every used line never misses
    assert oracle.cache_hit_rate(np.array([0.6, 0.4, 0.0]), 2, lib=lib)[0] == 1.0
    assert oracle.cache_hit_rate(np.array([1.0]), 1, lib=lib)[0] == 1.0
    # more cache never hurts
    z = 1.0 / np.arange(1, 301)
    z /= z.sum()
    hits = [oracle.cache_hit_rate(z, S, lib=lib)[0] for S in (1, 5, 20, 80, 200)]
    assert all(b >= a for a, b in zip(hits, hits[1:]))
    # within the paper's stated error (< 5 %) of a simulated LRU cache on Zipf traces
    for s, L, S in ((1.0, 2000, 200), (0.5, 2000, 100), (1.5, 2000, 50)):
        p = 1.0 / np.arange(1, L + 1) ** s
        p /= p.sum()
        assert abs(oracle.cache_hit_rate(p, S, lib=lib)[0] - _lru_hit_rate(p, S, 200_000, 1)) < 0.05


def pin_cache_threshold(lib):
    # the threshold counts the leading lines whose modelled hit probability is >= p, times the rows
    # per line; on the hand-worked lines of pin_cache_model (whose cdf is pinned there) ...
    f = np.array([0.9, 0.07, 0.015, 0.01, 0.005])
    _, cdf = oracle.cache_hit_rate(f, 3, lib=lib)
    for p in (0.3, 0.5, 0.9, 0.99):
        want = 0
        while want < f.size and cdf[want] >= p:
            want += 1
        assert oracle.cache_threshold(f, 3, p, 1, lib=lib) == want
        assert oracle.cache_threshold(f, 3, p, 16, lib=lib) == 16 * want
    # every line is a hit when the cache holds them all; p = 1 keeps exactly those
    assert oracle.cache_threshold(np.array([0.5, 0.3, 0.2]), 3, 1.0, 4, lib=lib) == 12
    # S = 1: cdf_i = f_i (exact LRU), so the threshold is the leading run of lines with f >= p
    assert oracle.cache_threshold(np.array([0.6, 0.25, 0.1, 0.05]), 1, 0.2, 1, lib=lib) == 2
    assert oracle.cache_threshold(np.array([0.6, 0.25, 0.1, 0.05]), 1, 0.7, 1, lib=lib) == 0
    # a colder line out of order stops the run (lines are in transformed-id order)
    assert oracle.cache_threshold(np.array([0.1, 0.6, 0.25, 0.05]), 1, 0.2, 1, lib=lib) == 0
    for bad in ((f, 3, 0.0, 1), (f, 3, 1.5, 1), (f, 3, 0.5, 0)):
        try:
            oracle.cache_threshold(*bad, lib=lib)
        except oracle.OracleError:
            continue
        raise AssertionError("invalid threshold arguments accepted")


def pin_powerlaw_fit(lib):
    # an exact power law c x^b is a line of slope b and intercept log c in a log-log plot
    x = np.arange(1, 501, dtype=np.float64)
    for c, b in ((3.0, -1.2), (1e6, -1.0), (0.5, -0.3), (2.0, 0.7)):
        slope, icpt = oracle.powerlaw_fit(x, c * x ** b, lib=lib)
        assert abs(slope - b) < 1e-12 and abs(icpt - np.log(c)) < 1e-10
    # two points fix the line; y = 8 at x = 2 and y = 2 at x = 8 give slope -1, intercept log 16
    slope, icpt = oracle.powerlaw_fit([2.0, 8.0], [8.0, 2.0], lib=lib)
    assert abs(slope + 1.0) < 1e-14 and abs(icpt - np.log(16.0)) < 1e-13
    # points with x <= 0 or y <= 0 are skipped (zero counts have no logarithm)
    slope, icpt = oracle.powerlaw_fit([1.0, 2.0, 3.0, 0.0, 5.0], [1.0, 0.25, 0.0, 7.0, 1.0 / 25.0], lib=lib)
    assert abs(slope + 2.0) < 1e-13 and abs(icpt) < 1e-13
    # least squares, not interpolation: (1, e), (e, 1), (e^2, e) -> u = 0, 1, 2 and v = 1, 0, 1 -> slope 0,
    # intercept 2/3
    e = np.e
    slope, icpt = oracle.powerlaw_fit([1.0, e, e * e], [e, 1.0, e], lib=lib)
    assert abs(slope) < 1e-14 and abs(icpt - 2.0 / 3.0) < 1e-14
    for bad in (([1.0], [1.0]), ([2.0, 2.0], [1.0, 3.0]), ([1.0, 2.0], [0.0, -1.0])):
        try:
            oracle.powerlaw_fit(*bad, lib=lib)
        except oracle.OracleError:
            continue
        raise AssertionError("degenerate fit accepted")


def pin_materialize(lib):
    # brute force: the attribute of the referenced row, for every fact row
    rng = np.random.default_rng(31)
    rows = rng.integers(-1000, 1000, size=(57, 5), dtype=np.int32)
    fk = rng.integers(0, 57, size=1001).astype(np.int32)
    for col in range(5):
        want = np.array([int(rows[int(k), col]) for k in fk], dtype=np.int32)
        assert np.array_equal(oracle.materialize(rows, fk, col, lib=lib), want)
    # Fig. 2 style check of layout invariance: reorder the rows and recode the keys with the
    # index, and every fact row still sees the same attribute
    cnt, perm, rank = oracle.build_index(fk, 57, lib=lib)
    rows2 = rows[perm]
    fk2 = rank[fk].astype(np.int32)
    for col in (0, 3):
        assert np.array_equal(oracle.materialize(rows2, fk2, col, lib=lib), oracle.materialize(rows, fk, col, lib=lib))
    assert oracle.materialize(rows, np.zeros(0, dtype=np.int32), 0, lib=lib).size == 0
    for bad_fk, bad_col in ((np.array([0, 57], dtype=np.int32), 0), (np.array([-1], dtype=np.int32), 0), (fk, 5)):
        try:
            oracle.materialize(rows, bad_fk, bad_col, lib=lib)
        except oracle.OracleError:
            continue
        raise AssertionError("invalid materialisation accepted")


ALL_PINS = [pin_fig2_example, pin_histogram, pin_sort_by_frequency, pin_invert, pin_remap,
            pin_reorder, pin_probe_brute_force, pin_probe_closed_forms, pin_probe_wraparound,
            pin_probe_layout_invariance, pin_probe_errors, pin_topk_counts, pin_select, pin_index_append,
            pin_cache_model, pin_cache_threshold, pin_powerlaw_fit, pin_materialize]
