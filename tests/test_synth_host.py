"""Seeded input generator (host twin): determinism, ranges and the Zipf shape."""
import numpy as np

from paper_1910_10063_gb300 import synth


def test_splitmix_reference_values():
    # SplitMix64 with seed 0 (state += GAMMA, then mix): first outputs as published
    # with the algorithm (Steele, Lea & Flood 2014 / Vigna's splitmix64.c).
    x = synth.raw_draws(0, 0, 3)
    assert [int(v) for v in x] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_based_random_access():
    key = synth.stream_key(3, synth.STREAM_FK)
    full = synth.raw_draws(key, 0, 1000)
    idx = np.array([0, 7, 999, 500])
    assert np.array_equal(synth.raw_draws_at(key, idx), full[idx])
    assert np.array_equal(synth.raw_draws(key, 100, 50), full[100:150])


def test_ranges():
    rows = synth.dim_rows_host(5000, 16, seed=1)
    assert rows[:, 0].min() >= 0 and rows[:, 0].max() < 1000
    assert rows[:, 1].min() >= 0 and rows[:, 1].max() < 100
    assert rows[:, 2].min() >= 0 and rows[:, 2].max() < 10**6
    assert rows[:, 4:].min() < -2**30 and rows[:, 4:].max() > 2**30  # full int32 filler
    m = synth.measure_host(1, 0, 100000)
    assert m.min() == 1 and m.max() == 100
    assert np.array_equal(synth.dim_rows_host_at([3, 4000], 16, 1), rows[[3, 4000]])


def test_zipf_shape():
    n, f = 1000, 400_000
    for s in (0.0, 1.0, 1.5):
        w = synth.Workload(n, f, s, seed=2)
        fk = w.fk()
        assert fk.min() >= 0 and fk.max() < n
        cnt = np.bincount(fk, minlength=n)
        by_rank = cnt[w.r2id]                       # count of the item of rank r
        p = np.arange(1, n + 1, dtype=float) ** -s
        p /= p.sum()
        expect = f * p
        top = slice(0, 20)
        assert np.all(np.abs(by_rank[top] - expect[top]) < 6 * np.sqrt(expect[top]) + 3)
        assert abs(by_rank.sum() - f) == 0


def test_rank_to_id_is_bijection_and_drift():
    r2id = synth.rank_to_id(10000, seed=4)
    assert np.array_equal(np.sort(r2id), np.arange(10000))
    d = synth.drift_rank_to_id(r2id, seed=4, fraction=0.1)
    assert np.array_equal(np.sort(d), np.arange(10000))
    moved = np.count_nonzero(d != r2id)
    assert 900 <= moved <= 1000


def test_lognormal_sizes():
    sz = synth.lognormal_sizes(512, seed=0)
    assert sz.min() >= 1000 and sz.max() <= 20_000_000
    assert 1e5 < np.median(sz) < 4e5
