"""The split probe (Section IV-B threshold split, with a rank-bucketed second
pass) against the oracle, element by element, through the C ABI.

The split only moves work between two passes and between shared memory, direct
gathers and the deferred buffer; every result must equal the oracle's join
over the original layout bit for bit, for every query kind, row path, split
threshold, bucket size, hot-prefix size, ragged or unaligned column, a buffer
that overflows (rows then resolved in the first pass), and bad keys.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1910_10063_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1910_10063_gb300 as skx  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def offset_view(a, offset):
    buf = torch.zeros(a.size + offset + 8, dtype=torch.int32, device=DEV)
    v = buf[offset:offset + a.size]
    v.copy_(torch.from_numpy(np.ascontiguousarray(a).reshape(-1)))
    return v


def tun(**kw):
    t = skx.Tuning()
    for k, v in kw.items():
        setattr(t, k, v)
    return t


QUERIES = {
    "groupby": dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=1, filter_lt=50, group_col=0, num_groups=1000, payload_col=2),
    "sum": dict(agg=oracle.AGG_SUM, filter_col=1, filter_lt=50, group_col=0, num_groups=1, payload_col=2),
    "count": dict(agg=oracle.AGG_COUNT, filter_col=1, filter_lt=50, group_col=0, num_groups=1, payload_col=-1),
    "groupby_nofilter_payload1": dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=-1, filter_lt=0, group_col=0,
                                      num_groups=1000, payload_col=-1),
    "generic_cols": dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=5, filter_lt=0, group_col=0, num_groups=1000,
                         payload_col=9),
}

SPLITS = {
    "t1000_b12": dict(split_keys=1000, split_bucket=12, hot_keys=-1),
    "t5000_hot1000_lane32": dict(split_keys=5000, hot_keys=1000, lane_keys=32),
    "t100_hot64_b12": dict(split_keys=100, hot_keys=64, lane_keys=8, split_bucket=12),
    "t30000_b26": dict(split_keys=30000, split_bucket=26, hot_keys=-1),
    "t_last": dict(split_keys=59_999, hot_keys=-1),
    "one_cta_per_sm": dict(split_keys=2000, hot_keys=-1, ctas_per_sm=1, block_threads=512),
}


def q_of(d):
    return skx.Query(d["agg"], d["filter_col"], d["filter_lt"], d["group_col"], d["num_groups"], d["payload_col"])


def want_of(rows, fk, m, d):
    return oracle.probe(rows, fk, m, d["agg"], d["filter_col"], d["filter_lt"], d["group_col"], d["num_groups"],
                        d["payload_col"], nthreads=8)


@pytest.fixture(scope="module")
def data():
    w = synth.Workload(60_000, 1_000_003, 1.2, seed=21, width=16)
    fk, m, dim = w.fk(), w.measure(), w.dim()
    cnt, perm, rank = oracle.build_index(fk, w.n)
    fk2, dim2 = oracle.remap(rank, fk), oracle.reorder(perm, dim)
    return dict(fk=fk, m=m, dim=dim, fk2=fk2, dim2=dim2, d_m=dev(m), d_dim=dev(dim), d_fk=dev(fk),
                d_fk2=dev(fk2), d_dim2=dev(dim2))


@pytest.mark.parametrize("qname", list(QUERIES))
@pytest.mark.parametrize("sname", list(SPLITS))
def test_split_probe_parity(data, qname, sname):
    d = QUERIES[qname]
    want = want_of(data["dim"], data["fk"], data["m"], d)
    for rows, fk in [(data["d_dim2"], data["d_fk2"]), (data["d_dim"], data["d_fk"])]:  # both layouts
        got = skx.skx_probe_aggregate(rows, fk, data["d_m"], q_of(d), tuning=tun(**SPLITS[sname]))
        assert np.array_equal(got.cpu().numpy(), want), (qname, sname)
    assert skx.skx_stream_status() == skx.SKX_OK


def test_split_probe_narrow_rows(data):
    # 8-byte query copy rows and 12-byte rows (generic path)
    for width in (2, 3):
        rows = np.ascontiguousarray(data["dim2"][:, [0, 2]] if width == 2 else data["dim2"][:, :3])
        d = dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=-1, filter_lt=0, group_col=0, num_groups=1000,
                 payload_col=1 if width == 2 else 2)
        want = want_of(rows, data["fk2"], data["m"], d)
        got = skx.skx_probe_aggregate(dev(rows), data["d_fk2"], data["d_m"], q_of(d),
                                      tuning=tun(split_keys=3000, hot_keys=512))
        assert np.array_equal(got.cpu().numpy(), want)


def test_split_probe_many_buckets_and_groups():
    """Hundreds of buckets (short runs, the bucket count raised past 1024), and more groups than
    shared memory holds (global group atomics in both passes)."""
    n, f, G = 5_000_000, 2_000_001, 50_000
    w = synth.Workload(n, f, 0.9, seed=8, width=4, num_groups=G)
    fk, m, dim = w.fk(), w.measure(), w.dim()
    _, perm, rank = oracle.build_index(fk, n)
    fk2, dim2 = oracle.remap(rank, fk), oracle.reorder(perm, dim)
    for G_, t in ((1000, tun(split_keys=10_000, split_bucket=12)), (G, tun(split_keys=4096, split_bucket=12)),
                  (1000, tun(split_keys=1, split_bucket=12, hot_keys=-1))):
        d = dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=1, filter_lt=50, group_col=0, num_groups=G_, payload_col=2)
        rows = dim2.copy()
        rows[:, 0] %= G_
        want = want_of(rows, fk2, m, d)
        got = skx.skx_probe_aggregate(dev(rows), dev(fk2), dev(m), q_of(d), tuning=t)
        assert np.array_equal(got.cpu().numpy(), want)
    assert skx.skx_stream_status() == skx.SKX_OK


def test_split_probe_buffer_overflow():
    """Uniform keys with t = 1 defer nearly every row, more than the buffer holds (F/2 plus one
    stage per CTA): the rows that do not fit are resolved in the first pass, exactly."""
    n, f = 1_000_000, 8_000_000
    w = synth.Workload(n, f, 0.0, seed=4, width=4)
    fk, m, dim = w.fk(), w.measure(), w.dim()
    for qname in ("groupby", "count", "sum"):
        d = QUERIES[qname]
        want = want_of(dim, fk, m, d)
        got = skx.skx_probe_aggregate(dev(dim), dev(fk), dev(m), q_of(d), tuning=tun(split_keys=1, hot_keys=-1))
        assert np.array_equal(got.cpu().numpy(), want), qname
    assert skx.skx_stream_status() == skx.SKX_OK


@pytest.mark.parametrize("f", [0, 1, 3, 5, 4097, 2049 * 4 + 3, 300_001])
@pytest.mark.parametrize("off_fk,off_m", [(0, 0), (1, 1), (3, 3), (1, 2)])
def test_split_probe_ragged_and_unaligned(data, f, off_fk, off_m):
    fk, m = data["fk2"][:f], data["m"][:f]
    for qname in ("groupby", "count", "sum"):
        d = QUERIES[qname]
        want = want_of(data["dim2"], fk, m, d)
        got = skx.skx_probe_aggregate(data["d_dim2"], offset_view(fk, off_fk), offset_view(m, off_m), q_of(d),
                                      tuning=tun(split_keys=2500, hot_keys=256, split_bucket=12))
        assert np.array_equal(got.cpu().numpy(), want), (qname, f, off_fk, off_m)


def test_split_probe_wraparound_and_negative():
    big = 2**31 - 1
    rows = np.array([[0, 0, big, 0], [1, 0, -big - 1, 0], [1, 0, -7, 0], [0, 0, 5, 0]], dtype=np.int32)
    fk = np.array(([0] * 6 + [1] * 3 + [2] * 5 + [3] * 2) * 5000, dtype=np.int32)
    m = np.array(([big] * 6 + [-big - 1] * 3 + [-3] * 5 + [big] * 2) * 5000, dtype=np.int32)
    for d in (QUERIES["groupby"], QUERIES["sum"]):
        d = dict(d, num_groups=2 if d["agg"] == oracle.AGG_GROUPBY_SUM else 1)
        want = want_of(rows, fk, m, d)
        for t in (tun(split_keys=1, hot_keys=-1), tun(split_keys=2, hot_keys=1, lane_keys=1),
                  tun(split_keys=3, hot_keys=-1, split_bucket=12)):
            got = skx.skx_probe_aggregate(dev(rows), dev(fk), dev(m), q_of(d), tuning=t)
            assert np.array_equal(got.cpu().numpy(), want)


def test_split_probe_data_errors(data):
    """A key >= N among the deferred range and a group key >= G: both reported, rows skipped."""
    fk = data["fk2"][:500_000].copy()
    bad = np.arange(7, fk.size, 9973)
    fk[bad] = 60_000 + 5
    ok = np.ones(fk.size, dtype=bool)
    ok[bad] = False
    d = QUERIES["groupby"]
    want = want_of(data["dim2"], fk[ok], data["m"][:500_000][ok], d)
    got = skx.skx_probe_aggregate(data["d_dim2"], dev(fk), data["d_m"][:500_000].contiguous(), q_of(d),
                                  tuning=tun(split_keys=1000, hot_keys=-1))
    assert skx.skx_stream_status() == skx.SKX_EKEYRANGE
    assert np.array_equal(got.cpu().numpy(), want)
    rows = data["dim2"].copy()
    rows[5000, 0] = 5000  # a deferred-range row with a group key beyond G = 1000
    rows[5000, 1] = 0     # that passes the filter
    got = skx.skx_probe_aggregate(dev(rows), data["d_fk2"], data["d_m"], q_of(d),
                                  tuning=tun(split_keys=1000, hot_keys=-1))
    st = skx.skx_stream_status()
    assert (data["fk2"] == 5000).any()
    assert st == skx.SKX_EGROUPRANGE
    keep = data["fk2"] != 5000
    assert np.array_equal(got.cpu().numpy(), want_of(rows, data["fk2"][keep], data["m"][keep], d))


def test_split_threshold_from_index_matches_oracle_pipeline():
    """skx_split_threshold: counts at log-spaced ranks, the power-law fit and the cache model's
    threshold, recomputed here with the oracle's fit and model on the oracle's counts."""
    n, f = 6000, 600_000  # the oracle's model is O(L^2): keep it to 3000 lines
    w = synth.DeviceWorkload(n, f, 1.0, seed=6, width=1, with_measure=False, with_dim=False)
    idx = skx.skx_build_index(w.fk, n)
    S_bytes = 400 * 128
    t = skx.skx_split_threshold(idx, 64, S_bytes, 0.5)
    cnt, perm, _ = oracle.build_index(w.fk.cpu().numpy(), n)
    by_rank = cnt[perm].astype(np.float64)
    ranks = []
    for k in range(48):
        r = min(n - 1, max(0, int(np.floor(np.exp(np.log(n) * k / 47.0))) - 1))
        if not ranks or r > ranks[-1]:
            ranks.append(r)
    ranks = np.array(ranks)
    slope, icpt = oracle.powerlaw_fit(ranks + 1.0, by_rank[ranks])
    fr = np.arange(1, n + 1, dtype=np.float64) ** slope
    lines = fr.reshape(-1, 2).sum(axis=1) / fr.sum()
    t_orc = oracle.cache_threshold(lines, S_bytes // 128, 0.5, 2)
    assert abs(t - t_orc) <= 4 and 0 < t < n
    # more cache -> a larger threshold; p = 1 -> only lines that always hit
    assert skx.skx_split_threshold(idx, 64, 4 * S_bytes, 0.5) >= t
    assert skx.skx_split_threshold(idx, 64, S_bytes, 0.99) <= t
    with pytest.raises(skx.SkxError):
        skx.skx_split_threshold(idx, 63, S_bytes, 0.5)
    idx.close()


def test_autotune_with_split_hint_is_exact(data):
    d = QUERIES["groupby"]
    q = q_of(d)
    t, ms = skx.skx_probe_autotune(data["d_dim2"], data["d_fk2"], data["d_m"], q, remapped=True, split_hint=3000)
    assert ms > 0
    want = want_of(data["dim"], data["fk"], data["m"], d)
    got = skx.skx_probe_aggregate(data["d_dim2"], data["d_fk2"], data["d_m"], q, tuning=t)
    assert np.array_equal(got.cpu().numpy(), want)
    got = skx.skx_probe_aggregate(data["d_dim2"], data["d_fk2"], data["d_m"], q)  # the cached choice
    assert np.array_equal(got.cpu().numpy(), want)


def test_index_drift_device_equals_host_half():
    """skx_index_drift (sample recoded and counted on the device) against its host half run on the
    oracle's counts by rank, on an undrifted and a 10 % drifted column."""
    n, f = 50_000, 2_000_000
    w = synth.Workload(n, f, 1.0, seed=12)
    fk = w.fk()
    _, perm, rank = oracle.build_index(fk, n)
    idx = skx.skx_build_index(dev(fk), n)
    for drift in (0.0, 0.1):
        r2 = synth.drift_rank_to_id(w.r2id, 12, drift) if drift else w.r2id
        sample = synth.Workload(n, 1_000_000, 1.0, seed=13, r2id=r2).fk()
        got = skx.skx_index_drift(idx, dev(sample), 1000, max_loss=0.02)
        by_rank = oracle.histogram(oracle.remap(rank, sample), n).astype(np.uint32)
        want = skx.skx_drift_from_counts(by_rank, 1000, max_loss=0.02)
        assert got.as_dict() == want.as_dict()
        assert got.rebuild == (1 if drift else 0)
    assert skx.skx_stream_status() == skx.SKX_OK
    idx.close()
