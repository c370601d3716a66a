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
