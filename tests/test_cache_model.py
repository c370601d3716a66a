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
