"""Host-side logic of bench.py that needs no GPU: the expected number of
distinct keys used for the probe's algorithmic bytes, the committed-DRAM-
traffic lookup (voided by a source change or another workload), and the
oracle baseline's bookkeeping."""
import json
import types

import numpy as np
import pytest

import bench
from paper_1910_10063_gb300 import synth


def test_expected_distinct_closed_forms():
    # uniform keys: n (1 - (1 - 1/n)^f)
    for n, f in [(10, 1), (1000, 500), (100_000, 3_000_000)]:
        want = n * (1 - (1 - 1 / n) ** f)
        assert bench.expected_distinct(n, f, 0.0) == pytest.approx(want, rel=1e-9)
    # one draw touches exactly one key; very many draws touch them all
    assert bench.expected_distinct(5000, 1, 1.0) == pytest.approx(1.0, rel=1e-9)
    assert bench.expected_distinct(200, 10**9, 1.0) == pytest.approx(200.0, rel=1e-9)


def test_expected_distinct_matches_sampling():
    n, f, s = 20_000, 50_000, 1.0
    rng = np.random.default_rng(3)
    cdf = synth.zipf_cdf(n, s)
    got = [np.unique(np.searchsorted(cdf, rng.random(f), side="right")).size for _ in range(20)]
    assert np.mean(got) == pytest.approx(bench.expected_distinct(n, f, s), rel=0.01)


def _shape_args(rec):
    n, f, s, row_b = rec["shape"]
    return types.SimpleNamespace(n=n, f=f, s=s, width=row_b // 4)


def test_ncu_traffic_lookup(tmp_path, monkeypatch):
    with open(bench.TRAFFIC_PATH) as fh:
        table = json.load(fh)
    rec = table["k_probe_p4/query4"]
    a = _shape_args(rec)
    # the committed entry is used only while its kernel sources are unchanged
    live = bench.ncu_traffic("k_probe_p4/query4", a)
    same = bench.source_sha([bench.os.path.join(bench.ROOT, x) for x in rec["sources"]]) == rec["source_sha"]
    assert live == (rec["bytes_per_launch"] if same else None)

    # a private copy: stage sums, shape mismatch, stale source
    t = {"x": dict(rec, bytes_per_launch=5), "y": dict(rec, bytes_per_launch=7)}
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(t))
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(p))
    if same:
        assert bench.ncu_traffic("x+y", a) == 12
        assert bench.ncu_traffic("x", None) == 5
    other = types.SimpleNamespace(n=a.n + 1, f=a.f, s=a.s, width=a.width)
    assert bench.ncu_traffic("x", other) is None
    t["x"]["source_sha"] = "0" * 16
    p.write_text(json.dumps(t))
    assert bench.ncu_traffic("x+y", a) is None
    assert bench.ncu_traffic("missing", a) is None


def test_cpu_baseline_bookkeeping():
    w = synth.Workload(5_000, 200_000, 1.0, seed=1, width=16)
    a = types.SimpleNamespace(f=200_000)
    r = bench.cpu_baseline(a, w.fk(), w.measure(), w.dim(), nthreads=2)
    assert r["kind"] == "oracle" and r["cores"] == 2 and r["unit"] == bench.UNIT
    assert r["value"] > 0 and r["probe_results_identical"]
    assert set(r["seconds"]) == {"build", "remap", "reorder", "probe", "probe_plain"}
    # the value covers the whole path (the per-stage times are rounded to 1 ms)
    whole = sum(v for k, v in r["seconds"].items() if k != "probe_plain")
    assert r["value"] == pytest.approx(200_000 / max(whole, 1e-3) / 1e9, rel=0.5)
