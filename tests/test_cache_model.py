"""The library's fast Section III-C cache model (host code in libskx.so) against
the oracle's plain restatement, on Zipf line distributions in any order (no GPU)."""
import numpy as np
import pytest

import oracle
import paper_1910_10063_gb300 as skx


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1910_10063_gb300 import build
    build.build()


@pytest.mark.parametrize("s", [0.0, 0.5, 1.0, 1.5, 2.0])
def test_fast_model_equals_oracle(s):
    for L, S in ((2000, 200), (5000, 17), (300, 1), (100, 99), (1000, 1000), (3000, 2500), (7, 3)):
        for seed in (1, 2):
            p = 1.0 / np.arange(1, L + 1) ** s
            p /= p.sum()
            np.random.default_rng(seed).shuffle(p)
            assert abs(skx.skx_cache_hit_rate(p, S) - oracle.cache_hit_rate(p, S)[0]) < 1e-9


def test_fast_model_closed_forms():
    f = np.array([0.5, 0.3, 0.15, 0.05])
    assert abs(skx.skx_cache_hit_rate(f, 1) - float(np.sum(f * f))) < 1e-12
    assert abs(skx.skx_cache_hit_rate(np.full(100, 0.01), 50) - (1 - 0.99 ** 50)) < 1e-12
    assert skx.skx_cache_hit_rate(np.array([0.6, 0.4, 0.0]), 2) == 1.0


@pytest.mark.parametrize("s", [0.0, 1.0, 1.5])
def test_line_cdf_and_threshold_equal_oracle(s):
    for L, S in ((2000, 200), (300, 1), (1000, 1000), (7, 3)):
        p = 1.0 / np.arange(1, L + 1) ** s
        p /= p.sum()
        want_hit, want_cdf = oracle.cache_hit_rate(p, S)
        assert np.allclose(skx.skx_cache_line_cdf(p, S), want_cdf, rtol=0, atol=1e-9)
        shuffled = p.copy()
        np.random.default_rng(3).shuffle(shuffled)
        assert np.allclose(skx.skx_cache_line_cdf(shuffled, S), oracle.cache_hit_rate(shuffled, S)[1], rtol=0,
                           atol=1e-9)
        for q in (0.25, 0.5, 0.9):
            # both sides decide cdf >= q in double; skip a boundary line the two round differently
            if np.any(np.abs(want_cdf - q) < 1e-9):
                continue
            for rpl in (1, 2):
                assert skx.skx_cache_threshold(p, S, q, rpl) == oracle.cache_threshold(p, S, q, rpl)


def test_powerlaw_fit_equals_oracle():
    rng = np.random.default_rng(5)
    for n in (2, 10, 64, 1000):
        x = np.sort(rng.uniform(1, 1e6, n))
        y = 1e7 * x ** -1.1 * np.exp(rng.normal(0, 0.3, n))
        b, a = skx.skx_powerlaw_fit(x, y)
        ob, oa = oracle.powerlaw_fit(x, y)
        assert abs(b - ob) < 1e-9 * max(1, abs(ob)) and abs(a - oa) < 1e-8 * max(1, abs(oa))
    with pytest.raises(skx.SkxError):
        skx.skx_powerlaw_fit([1.0], [1.0])
    with pytest.raises(skx.SkxError):
        skx.skx_cache_threshold([0.5, 0.5], 1, 0.0, 1)


def test_split_threshold_from_fit_equals_oracle_pipeline():
    """The model-derived split threshold (Sections III-C and IV-B): frequencies from a fitted
    power law summed per 128-byte line, then the model's threshold, against the oracle's model on
    the same lines."""
    for n, row_bytes, slope, S, p in ((6000, 64, -1.0, 400, 0.5), (4000, 16, -1.3, 150, 0.5),
                                      (3001, 64, -0.8, 700, 0.75), (2048, 128, -1.5, 64, 0.5)):
        rpl = max(1, 128 // row_bytes)
        fr = np.arange(1, n + 1, dtype=np.float64) ** slope
        pad = np.zeros(-(-n // rpl) * rpl)
        pad[:n] = fr
        lines = pad.reshape(-1, rpl).sum(axis=1) / fr.sum()
        _, cdf = oracle.cache_hit_rate(lines, S)
        if np.any(np.abs(cdf - p) < 1e-9):
            continue
        want = min(n, oracle.cache_threshold(lines, S, p, rpl))
        assert skx.skx_split_threshold_from_fit(slope, n, row_bytes, S * 128, p) == want
    # a bigger cache never gives a smaller threshold; a stricter p never a larger one
    t1 = skx.skx_split_threshold_from_fit(-1.0, 20_000, 64, 256 * 128, 0.5)
    assert skx.skx_split_threshold_from_fit(-1.0, 20_000, 64, 1024 * 128, 0.5) >= t1
    assert skx.skx_split_threshold_from_fit(-1.0, 20_000, 64, 256 * 128, 0.9) <= t1
    for bad in ((float("nan"), 100, 64, 1 << 20, 0.5), (-1.0, 0, 64, 1 << 20, 0.5), (-1.0, 100, 6, 1 << 20, 0.5),
                (-1.0, 100, 64, 64, 0.5), (-1.0, 100, 64, 1 << 20, 0.0)):
        with pytest.raises(skx.SkxError):
            skx.skx_split_threshold_from_fit(*bad)


def test_model_threshold_is_what_the_probe_resolves():
    """The split threshold from the model is kept as given when the probe resolves its tuning,
    with the bucket size raised until at most 512 buckets cover the keys above it; a threshold
    outside (hot_keys, N) turns the split off."""
    q = skx.Query.sum()  # no group sums: the split's staging fits even the 48 KB a CPU-only process assumes
    n = 20_000_000
    t_model = skx.skx_split_threshold_from_fit(-1.0, n, 64, 88_000_000, 0.5)
    assert 0 < t_model < n
    tun = skx.Tuning()
    tun.split_keys = t_model
    tun.hot_keys = -1
    r = skx.skx_probe_resolve_tuning(n, 64, 500_000_000, q, tun)
    assert r.split_keys == t_model
    assert -(-(n - t_model) // (1 << r.split_bucket)) <= 512 and r.split_bucket >= 19
    big = skx.Tuning()
    big.split_keys = 100
    big.split_bucket = 12
    r = skx.skx_probe_resolve_tuning(400_000_000, 64, 500_000_000, q, big)
    assert -(-(400_000_000 - 100) // (1 << r.split_bucket)) <= 512 < -(-(400_000_000 - 100) // (1 << (r.split_bucket - 1)))
    for t_bad, hot in ((n, -1), (n + 5, -1), (50, 64)):
        x = skx.Tuning()
        x.split_keys = t_bad
        x.hot_keys = hot
        assert skx.skx_probe_resolve_tuning(n, 64, 500_000_000, q, x).split_keys == -1
    again = skx.skx_probe_resolve_tuning(n, 64, 500_000_000, q, r)
    assert again.split_keys == r.split_keys and again.split_bucket == r.split_bucket  # idempotent
    # whatever the shared memory, a resolved hot prefix is a real size or off, never negative
    g = skx.Query.groupby_sum(num_groups=4096)
    for hot in (0, 64, 100_000):
        x = skx.Tuning()
        x.hot_keys = hot
        x.split_keys = 1000
        r = skx.skx_probe_resolve_tuning(n, 64, 500_000_000, g, x)
        assert r.hot_keys == -1 or r.hot_keys >= 1
        assert r.split_keys in (-1, 1000)
        if r.split_keys == 1000:
            assert r.hot_keys < 1000


def _drift_case(drift, seed=3, n=20_000, f=400_000):
    """An index built from one Zipf(1) column and a second column whose popularity drifted: a
    fraction of the ranks re-shuffled among themselves (0 = the same distribution).  Returns the
    second column's counts by the first index's ranks, computed by the oracle."""
    from paper_1910_10063_gb300 import synth
    w = synth.Workload(n, f, 1.0, seed=seed)
    _, perm, rank = oracle.build_index(w.fk(), n)
    r2 = synth.drift_rank_to_id(w.r2id, seed, drift) if drift > 0 else w.r2id
    w2 = synth.Workload(n, f, 1.0, seed=seed + 1, r2id=r2)
    by_rank = oracle.histogram(oracle.remap(rank, w2.fk()), n)
    return by_rank.astype(np.uint32)


def test_drift_from_counts_equals_oracle_and_decides():
    """Section III-A rebuild decision: the shares below t under the stale ranks and under the
    sample's own order, against a plain restatement over the oracle's counts; an undrifted
    column keeps the index, a 10 % re-shuffle of the ranks asks for a rebuild."""
    t = 500
    for drift, want_rebuild in ((0.0, 0), (0.1, 1)):
        c = _drift_case(drift)
        d = skx.skx_drift_from_counts(c, t, max_loss=0.02)
        total = int(c.astype(np.int64).sum())
        stale = int(c[:t].astype(np.int64).sum())
        fresh = int(np.sort(c.astype(np.int64))[::-1][:t].sum())
        assert d.sample == total and d.t == t
        assert d.share_stale == stale / total and d.share_fresh == fresh / total
        assert abs(d.loss - (fresh - stale) / total) < 1e-15
        assert d.rebuild == want_rebuild, (drift, d.as_dict())
    # the fresh share is the best any order can do: never below the stale one
    for t in (1, 10, 19_999, 20_000):
        d = skx.skx_drift_from_counts(_drift_case(0.1), t)
        assert d.share_fresh >= d.share_stale and d.loss >= 0
    with pytest.raises(skx.SkxError):
        skx.skx_drift_from_counts(np.zeros(10, np.uint32), 3)
    with pytest.raises(skx.SkxError):
        skx.skx_drift_from_counts(np.ones(10, np.uint32), 11)
