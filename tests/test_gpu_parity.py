"""Parity of every CUDA step with the CPU oracle, element by element, through
the C ABI (via the ctypes binding).  Integer work: the bar is bit-exact."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1910_10063_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # the -m gpu suite runs only where a GPU exists
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1910_10063_gb300 as skx  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def offset_view(a: np.ndarray, offset: int):
    """Device copy of `a` starting `offset` int32 elements into a larger buffer
    (exercises the unaligned head/tail paths)."""
    buf = torch.zeros(a.size + offset + 8, dtype=torch.int32, device=DEV)
    v = buf[offset:offset + a.size]
    v.copy_(torch.from_numpy(np.ascontiguousarray(a).reshape(-1)))
    return v


def status():
    return skx.skx_stream_status()


# ------------------------------------------------------------------ generator
def test_synth_device_matches_host():
    for n, f, s in [(1, 10, 1.0), (1000, 12345, 0.0), (5000, 100_000, 1.0), (300, 50_001, 1.5)]:
        w = synth.Workload(n, f, s, seed=3, width=16)
        d = synth.DeviceWorkload(n, f, s, seed=3, width=16)
        assert np.array_equal(d.fk.cpu().numpy(), w.fk())
        assert np.array_equal(d.measure.cpu().numpy(), w.measure())
        assert np.array_equal(d.dim.cpu().numpy(), w.dim())


def test_synth_device_sampled_at_scale():
    n, f = 2_000_000, 50_000_000
    d = synth.DeviceWorkload(n, f, 1.0, seed=11, width=16)
    idx = np.random.default_rng(0).integers(0, f, 20000)
    cdf = synth.zipf_cdf(n, 1.0)
    fk = d.fk.cpu().numpy()
    assert np.array_equal(fk[idx], synth.zipf_fk_host_at(cdf, d.r2id_host, 11, idx))
    assert np.array_equal(d.measure.cpu().numpy()[idx], synth.measure_host_at(11, idx))
    rows = np.random.default_rng(1).integers(0, n, 5000)
    assert np.array_equal(d.dim.cpu().numpy()[rows], synth.dim_rows_host_at(rows, 16, 11))


# ------------------------------------------------------------------ build index
CASES = [  # (N, F, s, seed)
    (1, 0, 1.0, 0),
    (1, 17, 1.0, 0),
    (7, 1, 0.0, 1),
    (100, 4099, 1.0, 2),        # ragged tail, > 1 tile of ids? (no: N small) several vectors
    (4097, 100_003, 1.2, 3),    # two sort tiles with a ragged last tile
    (50_000, 1_000_001, 1.0, 4),
    (20_000, 300_000, 0.0, 5),  # uniform: many equal counts -> ties by id
    (9000, 2_000_000, 1.5, 6),  # heavy skew, counts > 2^16 (3 radix passes)
    (100_000, 1_000_000, 1.0, 0),  # the 100K x 1M case, seed 0
]


@pytest.mark.parametrize("n,f,s,seed", CASES)
def test_build_index_parity(n, f, s, seed):
    w = synth.Workload(n, f, s, seed=seed, width=4)
    fk = w.fk()
    idx = skx.skx_build_index(dev(fk), n)
    cnt, perm, rank = oracle.build_index(fk, n)
    assert status() == skx.SKX_OK
    assert np.array_equal(idx.counts.cpu().numpy().view(np.uint32).astype(np.uint64), cnt)
    assert np.array_equal(idx.perm.cpu().numpy(), perm)
    assert np.array_equal(idx.rank.cpu().numpy(), rank)


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_build_index_unaligned(offset):
    w = synth.Workload(3000, 77_777, 1.0, seed=9)
    fk = w.fk()
    idx = skx.skx_build_index(offset_view(fk, offset), 3000)
    cnt, perm, rank = oracle.build_index(fk, 3000)
    assert np.array_equal(idx.perm.cpu().numpy(), perm)
    assert np.array_equal(idx.counts.cpu().numpy().view(np.uint32).astype(np.uint64), cnt)


# ------------------------------------------------------------------ count methods
METHODS = [skx.SKX_COUNT_SINGLE_PASS, skx.SKX_COUNT_PARTITIONED]


def _counts_np(c):
    return c.cpu().numpy().view(np.uint32).astype(np.uint64)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("n,f,s,seed,offset", [
    (1, 9, 1.0, 0, 0),
    (8, 10, 0.0, 1, 3),               # tiny: head and tail only, no full vector in most CTAs
    (32768, 100_001, 1.0, 2, 1),      # exactly one bucket of 2^15 ids
    (100_003, 3_000_001, 1.0, 3, 2),  # 4 buckets, the last ragged; many phase-C tiles
    (2_500_000, 6_000_007, 1.0, 4, 0),  # 77 buckets, a few million keys
    (300_000, 4_000_000, 0.0, 5, 1),  # uniform
    (70_000, 5_000_000, 1.5, 6, 0),   # heavy skew: hot ids' buckets span several 2^20-key chunks
])
def test_count_methods_parity(method, n, f, s, seed, offset):
    w = synth.Workload(n, f, s, seed=seed, width=4)
    fk = w.fk()
    c = skx.skx_count_ex(offset_view(fk, offset), n, method)
    assert status() == skx.SKX_OK
    assert np.array_equal(_counts_np(c), oracle.histogram(fk, n))


@pytest.mark.parametrize("n,f,s", [
    (1 << 24, (1 << 28) + 5, 1.0),        # about 45 % of the sampled keys repeat: partitioned
    (1 << 24, (1 << 28) + 5, 1.5),        # heavy skew (95 %): the single pass
    (1 << 16, (1 << 26) + 3, 0.0),        # the fewest sampled ids, flat: partitioned (2 buckets)
    ((1 << 20) + 7, (1 << 26) + 3, 0.0),  # flat: partitioned
    ((1 << 20) + 7, (1 << 26) + 3, 1.2),  # 60-85 % repeat, below 2^24 ids: the single pass
    ((1 << 24) + 3, (1 << 26) + 9, 1.2),  # 60-85 % repeat, from 2^24 ids, sampled layout: partitioned
    ((1 << 25) + 5, (1 << 26) + 3, 1.1),  # 60-70 % repeat, exact layout (1025 buckets): partitioned
    ((1 << 25) + 5, (1 << 26) + 3, 1.2),  # 70-85 % repeat, exact layout: the single pass
])
def test_count_auto_choice_parity(n, f, s):
    """Sizes where the automatic count samples the column and picks an
    algorithm on the device; every branch of the choice gives exact counts."""
    w = synth.DeviceWorkload(n, f, s, seed=12, width=1, device=DEV, with_measure=False, with_dim=False)
    expect = oracle.histogram(w.fk.cpu().numpy(), n)
    c = skx.skx_count(w.fk, n)
    assert status() == skx.SKX_OK
    assert np.array_equal(_counts_np(c), expect)
    del w, c
    torch.cuda.empty_cache()


@pytest.mark.parametrize("method", METHODS)
def test_count_methods_skewed_layouts(method):
    """Hot ids packed into bucket 0 (same-address shared atomics in every
    phase), one id holding every key (one bucket split into several chunks),
    ids that leave most buckets empty, and columns where about 40 % of the
    keys fall in one bucket (or on one id) at random positions, so that a
    warp's 32 sampled keys land on both sides of the register-path threshold
    within one launch."""
    rng = np.random.default_rng(23)
    n = 1_000_000
    cdf = synth.zipf_cdf(n, 1.0)
    ident = np.arange(n, dtype=np.int32)  # rank r -> id r: popularity follows the id order
    fk_ident = synth.zipf_fk_host(cdf, ident, 5, 0, 4_000_003)
    fk_one = np.full(3_000_005, 777_777, dtype=np.int32)
    fk_sparse = rng.integers(0, 1000, 2_000_000).astype(np.int32) * 997
    m = 3_000_017
    in_b0 = rng.random(m) < 0.4
    fk_mixed = np.where(in_b0, rng.integers(0, 32768, m), rng.integers(32768, n, m)).astype(np.int32)
    fk_mixed_one = np.where(in_b0, 12_345, rng.integers(0, n, m)).astype(np.int32)
    for fk in (fk_ident, fk_one, fk_sparse, fk_mixed, fk_mixed_one):
        c = skx.skx_count_ex(dev(fk), n, method)
        assert status() == skx.SKX_OK
        assert np.array_equal(_counts_np(c), oracle.histogram(fk, n))


@pytest.mark.parametrize("method", METHODS)
def test_count_methods_key_range(method):
    n = 100_000
    fk = synth.Workload(n, 500_001, 1.0, seed=8).fk()
    bad = fk.copy()
    bad[[0, 12345, 500_000]] = [n, -1, 2**31 - 1]
    c = skx.skx_count_ex(dev(bad), n, method)
    assert status() == skx.SKX_EKEYRANGE
    keep = np.ones(bad.size, dtype=bool)
    keep[[0, 12345, 500_000]] = False
    assert np.array_equal(_counts_np(c), oracle.histogram(bad[keep], n))


@pytest.mark.parametrize("offset", [0, 3])
def test_count_sampled_layout_fallbacks(offset):
    """The partitioned count sizes its bucket regions from 65536 keys at an even stride.
    - Every 4th key (exactly the sampled ones) is one id: the sample sees one bucket, the
      others outgrow their regions in the partition pass, and the exact layout recounts.
    - 90 % of the keys out of range over 1024 buckets: too few valid samples for the regions
      to fit, so the exact layout runs from the start (and the range error is reported).
    - N = 2^25 (1024 buckets) is the largest sampled layout, 2^25 + 5 the smallest exact one."""
    rng = np.random.default_rng(31 + offset)
    n = 1 << 20
    fk = rng.integers(0, n, 65536 * 4).astype(np.int32)
    fk[::4] = 5  # the sampled positions: stride F / 65536 = 4
    c = skx.skx_count_ex(offset_view(fk, offset), n, skx.SKX_COUNT_PARTITIONED)
    assert status() == skx.SKX_OK
    assert np.array_equal(_counts_np(c), oracle.histogram(fk, n))

    n = 1 << 25
    bad = rng.integers(0, n, 65536 * 8).astype(np.int32)
    out = rng.random(bad.size) < 0.9
    bad[out] = -3
    c = skx.skx_count_ex(offset_view(bad, offset), n, skx.SKX_COUNT_PARTITIONED)
    assert status() == skx.SKX_EKEYRANGE
    assert np.array_equal(_counts_np(c), oracle.histogram(bad[~out], n))

    for n in (1 << 25, (1 << 25) + 5):
        fk = synth.Workload(n, 2_000_003, 1.0, seed=9).fk()
        c = skx.skx_count_ex(offset_view(fk, offset), n, skx.SKX_COUNT_PARTITIONED)
        assert status() == skx.SKX_OK
        assert np.array_equal(_counts_np(c), oracle.histogram(fk, n))
        del c
    torch.cuda.empty_cache()


def test_count_method_errors():
    fk = dev(np.zeros(16, dtype=np.int32))
    with pytest.raises(skx.SkxError) as e:
        skx.skx_count_ex(fk, 10, 7)
    assert e.value.status == skx.SKX_EINVAL
    with pytest.raises(skx.SkxError) as e:
        skx.skx_count_ex(fk, (1 << 28) + 1, skx.SKX_COUNT_PARTITIONED,
                         counts=torch.empty(1, dtype=torch.int32, device=DEV))
    assert e.value.status == skx.SKX_ENOTSUP


def test_sort_heavy_light_split_cases():
    """Counts >= 255 take the multi-pass path, smaller ones the single clamped pass."""
    rng = np.random.default_rng(17)
    cases = []
    # heavy ties: ids 0..999 each exactly 300 times, plus a light tail over 50K ids
    fk = np.concatenate([np.repeat(np.arange(1000, dtype=np.int32), 300),
                         rng.integers(1000, 50_000, 600_000, dtype=np.int32)])
    cases.append((fk[rng.permutation(fk.size)], 50_000))
    # no heavy id at all (every count < 255), F/N <= 64
    cases.append((rng.integers(0, 5000, 300_000, dtype=np.int32), 5000))
    # one heavy id with a count above 2^24, everything else light
    cases.append((np.concatenate([np.full(17_000_000, 7, dtype=np.int32),
                                  rng.integers(0, 400_000, 1_000_000, dtype=np.int32)]), 400_000))
    # F > 64 N: the plain multi-pass sort
    cases.append((rng.integers(0, 1000, 200_000, dtype=np.int32), 1000))
    for fk, n in cases:
        idx = skx.skx_build_index(dev(fk), n)
        cnt, perm, rank = oracle.build_index(fk, n)
        assert np.array_equal(idx.perm.cpu().numpy(), perm)
        assert np.array_equal(idx.rank.cpu().numpy(), rank)


def test_build_index_all_same_key_and_ties():
    n = 5000
    fk = np.full(123_457, 4321, dtype=np.int32)
    idx = skx.skx_build_index(dev(fk), n)
    perm = idx.perm.cpu().numpy()
    assert perm[0] == 4321
    assert np.array_equal(perm[1:], np.delete(np.arange(n), 4321))  # the zero counts, ascending ids
    fk = np.arange(n, dtype=np.int32)[::-1].copy()  # every count 1 -> identity
    assert np.array_equal(skx.skx_build_index(dev(fk), n).perm.cpu().numpy(), np.arange(n))


def test_fig2_worked_example_on_gpu():
    from oracle_pins import load_fig2
    g = load_fig2()
    order = [int(x) - 1 for x in g["offset_order"]]
    fk = np.concatenate([np.full(8 - r, v, dtype=np.int32) for r, v in enumerate(order)])
    fk = fk[np.random.default_rng(7).permutation(fk.size)]
    idx = skx.skx_build_index(dev(fk), 8)
    assert idx.perm.cpu().numpy().tolist() == order
    rows = dev(np.array([[ord(c)] * 4 for c in g["dimension_rows"]], dtype=np.int32))
    out = torch.empty_like(rows)
    skx.skx_reorder(idx, rows, out)
    assert [chr(x) for x in out[:, 0].cpu().tolist()] == g["reordered_rows"]


# ------------------------------------------------------------------ remap / reorder
@pytest.mark.parametrize("n,f,s,seed", CASES[1:7])
def test_remap_parity(n, f, s, seed):
    w = synth.Workload(n, f, s, seed=seed)
    fk = w.fk()
    d_fk = dev(fk)
    idx = skx.skx_build_index(d_fk, n)
    _, perm, rank = oracle.build_index(fk, n)
    want = oracle.remap(rank, fk)
    out = torch.empty_like(d_fk)
    skx.skx_remap(idx, d_fk, out)
    assert np.array_equal(out.cpu().numpy(), want)
    skx.skx_remap(idx, d_fk, d_fk)  # in place
    assert np.array_equal(d_fk.cpu().numpy(), want)
    for off_in, off_out in [(1, 1), (2, 3), (0, 1)]:
        a = offset_view(fk, off_in)
        b = offset_view(np.zeros_like(fk), off_out)
        skx.skx_remap(idx, a, b)
        assert np.array_equal(b.cpu().numpy(), want)
    assert status() == skx.SKX_OK


@pytest.mark.parametrize("width", [1, 3, 4, 16, 17])
def test_reorder_parity(width):
    n = 10_007
    w = synth.Workload(n, 200_000, 1.0, seed=width, width=width)
    fk, dim = w.fk(), w.dim()
    idx = skx.skx_build_index(dev(fk), n)
    _, perm, _ = oracle.build_index(fk, n)
    d_in = dev(dim)
    d_out = torch.empty_like(d_in)
    skx.skx_reorder(idx, d_in, d_out)
    assert np.array_equal(d_out.cpu().numpy(), oracle.reorder(perm, dim))


def test_reorder_unaligned_rows():
    n, width = 999, 4
    w = synth.Workload(n, 20_000, 1.0, seed=2, width=width)
    fk, dim = w.fk(), w.dim()
    idx = skx.skx_build_index(dev(fk), n)
    _, perm, _ = oracle.build_index(fk, n)
    buf = torch.zeros(n * width + 1, dtype=torch.int32, device=DEV)
    src = buf[1:].view(n, width)
    src.copy_(dev(dim))
    dst = torch.empty_like(src)
    skx.skx_reorder(idx, src, dst)
    assert np.array_equal(dst.cpu().numpy(), oracle.reorder(perm, dim))


# ------------------------------------------------------------------ probe
TUNINGS = {
    "plain": lambda: skx.Tuning.plain(),
    "default": lambda: None,
    "hot64_lane8": lambda: _tuning(hot_keys=64, lane_keys=8),
    "hot1_nolane": lambda: _tuning(hot_keys=1, lane_keys=-1),
    "block128_u1": lambda: _tuning(block_threads=128, unroll=1),
    "block256_u4": lambda: _tuning(block_threads=256, unroll=4, hot_keys=3000, lane_keys=32),
}


def _tuning(**kw):
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
    "sum_payload3": dict(agg=oracle.AGG_SUM, filter_col=1, filter_lt=10, group_col=0, num_groups=1, payload_col=3),
}


def _q(d):
    return skx.Query(d["agg"], d["filter_col"], d["filter_lt"], d["group_col"], d["num_groups"], d["payload_col"])


def _oracle(rows, fk, m, d):
    return oracle.probe(rows, fk, m, d["agg"], d["filter_col"], d["filter_lt"], d["group_col"], d["num_groups"],
                        d["payload_col"], nthreads=8)


@pytest.fixture(scope="module")
def probe_data():
    w = synth.Workload(60_000, 1_000_003, 1.2, seed=21, width=16)
    fk, m, dim = w.fk(), w.measure(), w.dim()
    cnt, perm, rank = oracle.build_index(fk, w.n)
    fk2, dim2 = oracle.remap(rank, fk), oracle.reorder(perm, dim)
    return dict(fk=fk, m=m, dim=dim, fk2=fk2, dim2=dim2, d_fk=dev(fk), d_m=dev(m), d_dim=dev(dim),
                d_fk2=dev(fk2), d_dim2=dev(dim2))


@pytest.mark.parametrize("qname", list(QUERIES))
@pytest.mark.parametrize("tname", list(TUNINGS))
def test_probe_parity(probe_data, qname, tname):
    d = QUERIES[qname]
    want = _oracle(probe_data["dim"], probe_data["fk"], probe_data["m"], d)
    q = _q(d)
    for rows, fk in [(probe_data["d_dim"], probe_data["d_fk"]), (probe_data["d_dim2"], probe_data["d_fk2"])]:
        got = skx.skx_probe_aggregate(rows, fk, probe_data["d_m"], q, tuning=TUNINGS[tname]())
        assert np.array_equal(got.cpu().numpy(), want), (qname, tname)
    assert status() == skx.SKX_OK


def test_probe_generic_columns_and_narrow_rows(probe_data):
    # filter/group/payload outside the first 16 bytes -> per-column gathers
    d = dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=5, filter_lt=0, group_col=0, num_groups=1000, payload_col=9)
    want = _oracle(probe_data["dim"], probe_data["fk"], probe_data["m"], d)
    got = skx.skx_probe_aggregate(probe_data["d_dim2"], probe_data["d_fk2"], probe_data["d_m"], _q(d))
    assert np.array_equal(got.cpu().numpy(), want)
    # 12-byte rows (not a multiple of 16)
    dim3 = np.ascontiguousarray(probe_data["dim2"][:, :3])
    d = QUERIES["groupby"]
    want = _oracle(dim3, probe_data["fk2"], probe_data["m"], d)
    got = skx.skx_probe_aggregate(dev(dim3), probe_data["d_fk2"], probe_data["d_m"], _q(d))
    assert np.array_equal(got.cpu().numpy(), want)


def test_probe_many_groups_global_path():
    n, f, G = 20_000, 300_001, 50_000
    w = synth.Workload(n, f, 1.0, seed=5, width=4, num_groups=G)
    fk, m, dim = w.fk(), w.measure(), w.dim()
    d = dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=1, filter_lt=50, group_col=0, num_groups=G, payload_col=2)
    want = _oracle(dim, fk, m, d)
    for t in (skx.Tuning.plain(), None):
        got = skx.skx_probe_aggregate(dev(dim), dev(fk), dev(m), _q(d), tuning=t)
        assert np.array_equal(got.cpu().numpy(), want)


@pytest.mark.parametrize("off_fk,off_m", [(1, 1), (3, 3), (1, 2), (0, 3)])
def test_probe_unaligned(probe_data, off_fk, off_m):
    d = QUERIES["groupby"]
    fk, m = probe_data["fk2"][:200_001], probe_data["m"][:200_001]
    want = _oracle(probe_data["dim2"], fk, m, d)
    got = skx.skx_probe_aggregate(probe_data["d_dim2"], offset_view(fk, off_fk), offset_view(m, off_m), _q(d))
    assert np.array_equal(got.cpu().numpy(), want)


@pytest.mark.parametrize("f", [0, 1, 2, 3, 5, 31, 4097])
def test_probe_tiny_and_ragged(probe_data, f):
    for qname in ("groupby", "count", "sum"):
        d = QUERIES[qname]
        want = _oracle(probe_data["dim2"], probe_data["fk2"][:f], probe_data["m"][:f], d)
        got = skx.skx_probe_aggregate(probe_data["d_dim2"], probe_data["d_fk2"][:f].contiguous(),
                                      probe_data["d_m"][:f].contiguous(), _q(d))
        assert np.array_equal(got.cpu().numpy(), want)


def test_probe_wraparound_and_negative():
    big = 2**31 - 1
    rows = np.array([[0, 0, big, 0], [1, 0, -big - 1, 0], [1, 0, -7, 0]], dtype=np.int32)
    fk = np.array(([0] * 6 + [1] * 3 + [2] * 5) * 1000, dtype=np.int32)
    m = np.array(([big] * 6 + [-big - 1] * 3 + [-3] * 5) * 1000, dtype=np.int32)
    for d in (QUERIES["groupby"], QUERIES["sum"]):
        d = dict(d, num_groups=2 if d["agg"] == oracle.AGG_GROUPBY_SUM else 1)
        want = _oracle(rows, fk, m, d)
        for t in (skx.Tuning.plain(), None, _tuning(hot_keys=1, lane_keys=1)):
            got = skx.skx_probe_aggregate(dev(rows), dev(fk), dev(m), _q(d), tuning=t)
            assert np.array_equal(got.cpu().numpy(), want)


# ------------------------------------------------------------------ query preprocessing copies
@pytest.mark.parametrize("cols", [[0, 1, 2, 3], [2, 0], [5, 1, 0], [0]])
def test_reorder_columns_parity(probe_data, cols):
    n = probe_data["dim"].shape[0]
    idx = skx.skx_build_index(probe_data["d_fk"], n)
    _, perm, _ = oracle.build_index(probe_data["fk"], n)
    want = oracle.reorder(perm, np.ascontiguousarray(probe_data["dim"][:, cols]))
    got = skx.skx_reorder_columns(idx, probe_data["d_dim"], cols)
    assert np.array_equal(got.cpu().numpy(), want)
    plain = skx.skx_reorder_columns(None, probe_data["d_dim"], cols)
    assert np.array_equal(plain.cpu().numpy(), probe_data["dim"][:, cols])


@pytest.mark.parametrize("qname", ["groupby", "sum", "count", "groupby_nofilter_payload1", "sum_payload3"])
def test_query_copy_end_to_end(probe_data, qname):
    """Probe over the 8-byte prefiltered copy == oracle on the original layout."""
    d = QUERIES[qname]
    want = _oracle(probe_data["dim"], probe_data["fk"], probe_data["m"], d)
    q = _q(d)
    qp = skx.skx_query_prefiltered(q)
    n = probe_data["dim"].shape[0]
    idx = skx.skx_build_index(probe_data["d_fk"], n)
    fk2 = torch.empty_like(probe_data["d_fk"])
    skx.skx_remap(idx, probe_data["d_fk"], fk2)
    for index, keys in [(idx, fk2), (None, probe_data["d_fk"])]:
        rows8 = skx.skx_reorder_query(index, probe_data["d_dim"], q)
        for t in (None, skx.Tuning.plain(), _tuning(hot_keys=2048, lane_keys=16)):
            got = skx.skx_probe_aggregate(rows8, keys, probe_data["d_m"], qp, tuning=t)
            assert np.array_equal(got.cpu().numpy(), want), (qname, t)
    # the copy itself, element by element
    _, perm, _ = oracle.build_index(probe_data["fk"], n)
    src = oracle.reorder(perm, probe_data["dim"])
    passes = src[:, d["filter_col"]] < d["filter_lt"] if d["filter_col"] >= 0 else np.ones(n, bool)
    key = (src[:, d["group_col"]] if d["agg"] == oracle.AGG_GROUPBY_SUM else np.zeros(n, np.int32))
    key = np.where(passes, key, qp.num_groups)
    pay = src[:, d["payload_col"]] if (d["payload_col"] >= 0 and d["agg"] != oracle.AGG_COUNT) else np.ones(n, np.int32)
    got = skx.skx_reorder_query(idx, probe_data["d_dim"], q).cpu().numpy()
    assert np.array_equal(got[:, 0], key) and np.array_equal(got[:, 1], pay)


@pytest.mark.parametrize("width,offset", [(3, 0), (4, 0), (4, 1), (5, 0), (8, 2), (16, 0), (16, 3)])
def test_query_copy_layouts(width, offset):
    """The query copy over rows of 12 to 64 bytes, 16-byte aligned and not, with the used columns
    in one aligned 16-byte chunk (one vector load per row) or spread over several, and N not a
    multiple of the rows one grid step covers: element by element against the oracle's permuted
    rows, in both orders (the index's and the identity)."""
    rng = np.random.default_rng(40 + width + offset)
    n = 70_001
    dim = rng.integers(0, 150, (n, width)).astype(np.int32)  # every group in [0, 160)
    fk = rng.integers(0, n, 300_007).astype(np.int32)
    idx = skx.skx_build_index(dev(fk), n)
    _, perm, _ = oracle.build_index(fk, n)
    buf = torch.zeros(n * width + offset + 8, dtype=torch.int32, device=DEV)
    rows = buf[offset:offset + n * width].view(n, width)
    rows.copy_(torch.from_numpy(dim))
    cases = [(1, 0, 2), (width - 1, 0, width - 1), (-1, width // 2, 0), (2, width - 1, 1)]
    for index, src in ((idx, oracle.reorder(perm, dim)), (None, dim)):
        for fcol, gcol, pcol in cases:
            for agg, ng in ((oracle.AGG_GROUPBY_SUM, 160), (oracle.AGG_SUM, 1), (oracle.AGG_COUNT, 1)):
                q = skx.Query(agg, fcol, 40, gcol, ng, pcol)
                got = skx.skx_reorder_query(index, rows, q).cpu().numpy()
                passes = src[:, fcol] < 40 if fcol >= 0 else np.ones(n, bool)
                key = src[:, gcol] if agg == oracle.AGG_GROUPBY_SUM else np.zeros(n, np.int32)
                key = np.where(passes, key, ng if agg == oracle.AGG_GROUPBY_SUM else 1)
                pay = src[:, pcol] if agg != oracle.AGG_COUNT else np.ones(n, np.int32)
                assert np.array_equal(got[:, 0], key), (fcol, gcol, pcol, agg)
                assert np.array_equal(got[:, 1], pay), (fcol, gcol, pcol, agg)
    assert status() == skx.SKX_OK


@pytest.mark.parametrize("offset", [0, 1, 3])
def test_probe_8byte_rows_lean_kernel(offset):
    """8-byte rows without a hot prefix take a lean kernel (k_probe_r8); it must agree with the
    oracle for every aggregation and every column arrangement of the pair, with group sums in
    shared memory (G <= 4096) and in global memory (G > 4096), fk and measure at any offset
    (head and tail rows), at one to three CTAs per SM, and with the general kernel (two vectors
    per thread); key and group range errors are still reported."""
    rng = np.random.default_rng(50 + offset)
    n, f = 90_001, 700_003
    rows = np.stack([rng.integers(0, 5000, n), rng.integers(-1000, 100_000, n)], axis=1).astype(np.int32)
    fk = rng.integers(0, n, f).astype(np.int32)
    m = rng.integers(-50, 100, f).astype(np.int32)
    d_rows, d_fk, d_m = dev(rows), offset_view(fk, offset), offset_view(m, offset)
    cases = [dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=0, filter_lt=4000, group_col=0, num_groups=4000,
                  payload_col=1),
             dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=1, filter_lt=50_000, group_col=0, num_groups=5000,
                  payload_col=-1),
             dict(agg=oracle.AGG_SUM, filter_col=-1, filter_lt=0, group_col=0, num_groups=1, payload_col=1),
             dict(agg=oracle.AGG_SUM, filter_col=0, filter_lt=2500, group_col=0, num_groups=1, payload_col=0),
             dict(agg=oracle.AGG_COUNT, filter_col=1, filter_lt=0, group_col=0, num_groups=1, payload_col=-1)]
    tunings = [_tuning(hot_keys=-1, lane_keys=-1, ctas_per_sm=c) for c in (1, 2, -1)]
    tunings.append(_tuning(hot_keys=-1, lane_keys=-1, unroll=2))
    for d in cases:
        want = _oracle(rows, fk, m, d)
        for t in tunings:
            got = skx.skx_probe_aggregate(d_rows, d_fk, d_m, _q(d), tuning=t)
            assert np.array_equal(got.cpu().numpy(), want), (d, t.ctas_per_sm, t.unroll)
    assert status() == skx.SKX_OK
    bad = fk.copy()
    bad[[7, f - 1]] = [n, -2]
    d = cases[0]
    keep = np.ones(f, bool)
    keep[[7, f - 1]] = False
    got = skx.skx_probe_aggregate(d_rows, offset_view(bad, offset), d_m, _q(d), tuning=tunings[2])
    assert status() == skx.SKX_EKEYRANGE
    assert np.array_equal(got.cpu().numpy(), _oracle(rows, fk[keep], m[keep], d))
    d = dict(cases[0], num_groups=3000)  # group keys 3000..3999 pass the filter: out of range
    skx.skx_probe_aggregate(d_rows, d_fk, d_m, _q(d), tuning=tunings[2])
    assert status() == skx.SKX_EGROUPRANGE


def _packed_expect(src, d):
    """The packed copy of rows `src` for query d, written out from the definition in skx.h."""
    grp = d["agg"] == oracle.AGG_GROUPBY_SUM
    G = d["num_groups"] if grp else 1
    b = 1
    while (1 << b) < G + 2:
        b += 1
    pb = 32 - b
    n = src.shape[0]
    passes = src[:, d["filter_col"]] < d["filter_lt"] if d["filter_col"] >= 0 else np.ones(n, bool)
    key = (src[:, d["group_col"]].astype(np.int64) if grp else np.zeros(n, np.int64))
    key = np.where(passes, key, G)
    pay = (src[:, d["payload_col"]].astype(np.int64) if (d["payload_col"] >= 0 and d["agg"] != oracle.AGG_COUNT)
           else np.ones(n, np.int64))
    pay_code = np.where(passes, pay, 0)  # a filtered row's payload is packed as 0
    fits = (key >= 0) & (key <= G) & (pay_code >= -(1 << (pb - 1))) & (pay_code < (1 << (pb - 1)))
    code = np.where(fits, (key << pb) | (pay_code & ((1 << pb) - 1)), ((1 << b) - 1) << pb)
    return code.astype(np.uint32).view(np.int32), key.astype(np.int32), pay.astype(np.int32)


@pytest.mark.parametrize("offset_m", [0, 1])
def test_packed_query_copy_and_probe(offset_m):
    """The 32-bit packed query copy, element by element against its definition over the oracle's
    permuted rows (payloads that fit and that escape, negative ones, groups outside [0, G) that
    escape, G on both sides of a power of two, shared and global group sums), and the probe over
    it exactly equal to the oracle's join on the original layout; measure at the key column's
    offset (16-byte path) and at another (the 8-byte copy's path); range errors reported."""
    rng = np.random.default_rng(60 + offset_m)
    n, f = 50_003, 600_007
    dim = np.stack([rng.integers(0, 1100, n), rng.integers(0, 100, n), rng.integers(-3000, 3000, n),
                    rng.integers(0, 10, n)], axis=1).astype(np.int32)
    big = rng.random(n) < 0.02
    dim[big, 2] = rng.integers(-2_000_000_000, 2_000_000_000, int(big.sum()))  # payloads that escape
    fk = rng.integers(0, n, f).astype(np.int32)
    m = rng.integers(-100, 100, f).astype(np.int32)
    idx = skx.skx_build_index(dev(fk), n)
    _, perm, rank = oracle.build_index(fk, n)
    src = oracle.reorder(perm, dim)
    fk2 = oracle.remap(rank, fk)
    d_fk2 = offset_view(fk2, 1)
    d_m = offset_view(m, 1 + offset_m)
    d_dim = dev(dim)
    cases = [dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=1, filter_lt=50, group_col=0, num_groups=1100, payload_col=2),
             dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=1, filter_lt=90, group_col=3, num_groups=1022, payload_col=2),
             dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=-1, filter_lt=0, group_col=3, num_groups=1023, payload_col=0),
             dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=1, filter_lt=70, group_col=0, num_groups=5000, payload_col=2),
             dict(agg=oracle.AGG_SUM, filter_col=1, filter_lt=30, group_col=0, num_groups=1, payload_col=2),
             dict(agg=oracle.AGG_COUNT, filter_col=1, filter_lt=30, group_col=0, num_groups=1, payload_col=-1)]
    for d in cases:
        q = _q(d)
        rows8, rows4 = skx.skx_reorder_query_packed(idx, d_dim, q)
        code, key, pay = _packed_expect(src, d)
        assert np.array_equal(rows4.cpu().numpy(), code), d
        assert np.array_equal(rows8.cpu().numpy()[:, 0], key) and np.array_equal(rows8.cpu().numpy()[:, 1], pay)
        want = _oracle(dim, fk, m, d)
        for t in (None, _tuning(ctas_per_sm=1), _tuning(block_threads=256)):
            got = skx.skx_probe_packed(rows4, rows8, d_fk2, d_m, q, tuning=t)
            assert np.array_equal(got.cpu().numpy(), want), (d, t)
        assert status() == skx.SKX_OK
    # group keys 1000..1099 pass the filter: outside [0, 1000); the copy reports it
    d = dict(cases[0], num_groups=1000)
    rows8, rows4 = skx.skx_reorder_query_packed(idx, d_dim, _q(d))
    assert status() == skx.SKX_EGROUPRANGE
    rows8 = skx.skx_reorder_query(idx, d_dim, _q(d))
    assert status() == skx.SKX_EGROUPRANGE
    # a negative group escapes the packing and the probe reports it too
    neg = dim.copy()
    neg[dim[:, 1] < 50, 0] = -5
    rows8, rows4 = skx.skx_reorder_query_packed(idx, dev(neg), _q(cases[0]))
    assert status() == skx.SKX_EGROUPRANGE
    skx.skx_probe_packed(rows4, rows8, d_fk2, d_m, _q(cases[0]))
    assert status() == skx.SKX_EGROUPRANGE
    bad = fk2.copy()
    bad[[3, f - 2]] = [n, -1]
    d = cases[0]
    rows8, rows4 = skx.skx_reorder_query_packed(idx, d_dim, _q(d))
    got = skx.skx_probe_packed(rows4, rows8, offset_view(bad, 1), d_m, _q(d))
    assert status() == skx.SKX_EKEYRANGE
    keep = np.ones(f, bool)
    keep[[3, f - 2]] = False
    assert np.array_equal(got.cpu().numpy(), _oracle(dim, fk[keep], m[keep], d))


# ------------------------------------------------------------------ Q3a, Q2, maintenance
@pytest.mark.parametrize("k", [1, 31, 32, 33, 4000, 60_000])
def test_topk_counts_parity(probe_data, k):
    want = oracle.topk_counts(probe_data["fk2"], k).astype(np.int64)
    got = skx.skx_topk_counts(probe_data["d_fk2"], k)
    assert np.array_equal(got.cpu().numpy(), want)
    for off in (1, 3):
        got = skx.skx_topk_counts(offset_view(probe_data["fk2"][:100_003], off), k)
        assert np.array_equal(got.cpu().numpy(), oracle.topk_counts(probe_data["fk2"][:100_003], k).astype(np.int64))
    assert np.array_equal(skx.skx_topk_counts(probe_data["d_fk2"][:0].contiguous(), k).cpu().numpy(), np.zeros(k))


@pytest.mark.parametrize("c", [0, 1, 50, 100])
def test_select_parity(probe_data, c):
    n = probe_data["dim"].shape[0]
    for dim, d_dim, fk, d_fk in [(probe_data["dim"], probe_data["d_dim"], probe_data["fk"], probe_data["d_fk"]),
                                 (probe_data["dim2"], probe_data["d_dim2"], probe_data["fk2"], probe_data["d_fk2"])]:
        bits = skx.skx_select_bitmap(d_dim, 1, c)
        want_bits = np.packbits((dim[:, 1] < c).astype(np.uint8), bitorder="little")
        want_bits = np.pad(want_bits, (0, bits.numel() * 4 - want_bits.size)).view(np.int32)
        assert np.array_equal(bits.cpu().numpy(), want_bits)
        offs, cnt = skx.skx_select(bits, n, d_fk)
        want = oracle.select(dim, fk, 1, c)
        assert int(cnt.item()) == want.size
        assert np.array_equal(offs[:want.size].cpu().numpy().view(np.uint32), want)
    # the same offsets from both layouts: the fact order is unchanged by the remap
    assert status() == skx.SKX_OK


def test_select_ragged_and_errors(probe_data):
    n = probe_data["dim"].shape[0]
    bits = skx.skx_select_bitmap(probe_data["d_dim"], 1, 50)
    for f in (0, 1, 31, 8193):
        offs, cnt = skx.skx_select(bits, n, probe_data["d_fk"][:f].contiguous())
        want = oracle.select(probe_data["dim"], probe_data["fk"][:f], 1, 50)
        assert int(cnt.item()) == want.size
        assert np.array_equal(offs[:want.size].cpu().numpy().view(np.uint32), want)
    bad = dev(np.array([0, n, 1], dtype=np.int32))
    offs, cnt = skx.skx_select(bits, n, bad)
    assert status() == skx.SKX_EKEYRANGE


@pytest.mark.parametrize("f", [0, 1, 3, 5, 4097, 300_001])
@pytest.mark.parametrize("off_fk,off_out", [(0, 0), (1, 1), (2, 0), (3, 1)])
def test_materialize_parity(f, off_fk, off_out):
    """Q1 on the plain layout and on the remapped one, against the oracle; unaligned and
    mismatched offsets (vector and scalar paths), ragged tails."""
    w = synth.Workload(20_000, f, 1.0, seed=29, width=16)
    fk, dim = w.fk(), w.dim()
    want = oracle.materialize(dim, fk, 2)
    out_buf = torch.zeros(f + off_out + 8, dtype=torch.int32, device=DEV)
    out = out_buf[off_out:off_out + f]
    skx.skx_materialize(dev(dim), offset_view(fk, off_fk), 2, out=out)
    assert status() == skx.SKX_OK
    assert np.array_equal(out.cpu().numpy(), want)
    if f:
        idx = skx.skx_build_index(dev(fk), 20_000)
        _, perm, rank = oracle.build_index(fk, 20_000)
        fk2 = rank[fk].astype(np.int32)
        got = skx.skx_materialize(dev(dim[perm]), dev(fk2), 2).cpu().numpy()
        assert np.array_equal(got, want)                                  # layout invariance


def test_materialize_errors_and_columns():
    dim = np.arange(40, dtype=np.int32).reshape(10, 4)
    fk = np.array([0, 9, 10, 3, -1, 5], dtype=np.int32)
    out = skx.skx_materialize(dev(dim), dev(fk), 3).cpu().numpy()
    assert status() == skx.SKX_EKEYRANGE
    assert np.array_equal(out, [3, 39, 0, 15, 0, 23])
    for col in range(4):
        ok = np.array([0, 9, 3, 5], dtype=np.int32)
        assert np.array_equal(skx.skx_materialize(dev(dim), dev(ok), col).cpu().numpy(), dim[ok, col])
    with pytest.raises(skx.SkxError):
        skx.skx_materialize(dev(dim), dev(fk), 4)


def test_index_counts_at_ranks():
    """Counts by transformed id, gathered on the device, equal the oracle's cnt[perm[r]]."""
    n = 50_000
    fk = synth.Workload(n, 1_000_003, 1.1, seed=21).fk()
    idx = skx.skx_build_index(dev(fk), n)
    cnt, perm, _ = oracle.build_index(fk, n)
    ranks = np.concatenate([np.arange(10), np.random.default_rng(4).integers(0, n, 1000), [n - 1]])
    got = skx.skx_index_counts_at_ranks(idx, ranks)
    assert np.array_equal(got.astype(np.uint64), cnt[perm[ranks]])
    assert skx.skx_index_counts_at_ranks(idx, np.zeros(0, dtype=np.int64)).size == 0
    with pytest.raises(skx.SkxError):
        skx.skx_index_counts_at_ranks(idx, [n])
    # the fitted exponent of a Zipf(1.1) column's counts is near -1.1 over the well-sampled head
    r = np.unique(np.geomspace(1, 2000, 40).astype(np.int64)) - 1
    slope, _ = skx.skx_powerlaw_fit(r + 1.0, skx.skx_index_counts_at_ranks(idx, r).astype(np.float64))
    assert abs(slope + 1.1) < 0.1


def test_index_append_and_probe():
    n, extra = 20_000, 3_000
    w = synth.Workload(n + extra, 400_000, 1.0, seed=13, width=16)
    dim_all = w.dim()
    fk_old = (w.fk() % n).astype(np.int32)              # the index is built before the new rows exist
    idx = skx.skx_build_index(dev(fk_old), n)
    cnt, perm, rank = oracle.build_index(fk_old, n)
    skx.skx_index_append(idx, extra)
    p2, r2 = oracle.index_append(perm, rank, extra)
    assert np.array_equal(idx.perm.cpu().numpy(), p2)
    assert np.array_equal(idx.rank.cpu().numpy(), r2)
    assert np.array_equal(idx.counts.cpu().numpy()[n:], np.zeros(extra, np.int32))
    # facts that reference old and new rows, remapped through the stale-but-extended index
    fk_new = w.fk()
    d_fk = dev(fk_new)
    fk2 = torch.empty_like(d_fk)
    skx.skx_remap(idx, d_fk, fk2)
    dim2 = torch.empty((n + extra, 16), dtype=torch.int32, device=DEV)
    skx.skx_reorder(idx, dev(dim_all), dim2)
    got = skx.skx_probe_aggregate(dim2, fk2, dev(w.measure()), skx.Query.groupby_sum())
    assert np.array_equal(got.cpu().numpy(), oracle.probe(dim_all, fk_new, w.measure(), nthreads=8))
    assert status() == skx.SKX_OK


# ------------------------------------------------------------------ batched probes
@pytest.fixture(scope="module")
def batch_data():
    n = 200_000
    w = synth.Workload(n, 2_000_000, 1.0, seed=31, width=16)
    fk_all, m_all, dim = w.fk(), w.measure(), w.dim()
    cnt, perm, rank = oracle.build_index(fk_all, n)
    rng = np.random.default_rng(5)
    qs = []
    kinds = [QUERIES["groupby"], QUERIES["sum"], QUERIES["count"], QUERIES["groupby_nofilter_payload1"],
             QUERIES["sum_payload3"], dict(QUERIES["groupby"], num_groups=4096),
             dict(agg=oracle.AGG_GROUPBY_SUM, filter_col=1, filter_lt=90, group_col=1, num_groups=100, payload_col=3)]
    sizes = [0, 1, 3, 4, 5, 17, 1000, 4099, 65536, 65537, 250_001, 2_000_000]
    for i in range(40):
        f = sizes[i % len(sizes)] if i < len(sizes) else int(rng.integers(1, 300_000))
        start = int(rng.integers(0, fk_all.size - f + 1))
        d = kinds[i % len(kinds)]
        qs.append((start, f, d, int(rng.integers(0, 4)) if i % 5 == 0 else 0))
    return dict(n=n, fk=fk_all, m=m_all, dim=dim, rank=rank, perm=perm, qs=qs,
                d_dim2=dev(oracle.reorder(perm, dim)), fk2=oracle.remap(rank, fk_all))


def _batch_items(bd):
    items, wants = [], []
    for start, f, d, off in bd["qs"]:
        fk2 = bd["fk2"][start:start + f]
        m = bd["m"][start:start + f]
        d_fk = offset_view(fk2, off) if off else dev(fk2)
        d_m = offset_view(m, off) if off else dev(m)
        q = _q(d)
        out = torch.full((q.nout,), -1, dtype=torch.int64, device=DEV)
        items.append((d_fk, None if d["agg"] == oracle.AGG_COUNT else d_m, q, out))
        wants.append(_oracle(bd["dim"], bd["fk"][start:start + f], m, d))
    return items, wants


def test_probe_batch_parity(batch_data):
    items, wants = _batch_items(batch_data)
    skx.skx_probe_batch(batch_data["d_dim2"], items)
    for (_, _, _, out), want in zip(items, wants):
        assert np.array_equal(out.cpu().numpy(), want)
    assert status() == skx.SKX_OK


def test_batch_plan_graph_replay_and_autotune(batch_data):
    items, wants = _batch_items(batch_data)
    plan = skx.BatchPlan(batch_data["d_dim2"], items, tile_rows=4096)
    for use_graph in (False, True, True):
        for _, _, _, out in items:
            out.fill_(-1)
        plan.launch(use_graph=use_graph)
        torch.cuda.synchronize()
        for (_, _, _, out), want in zip(items, wants):
            assert np.array_equal(out.cpu().numpy(), want)
    t, tile, ms = plan.autotune()
    assert ms > 0 and tile > 0
    for _, _, _, out in items:
        out.fill_(-1)
    plan.launch(use_graph=True)
    torch.cuda.synchronize()
    for (_, _, _, out), want in zip(items, wants):
        assert np.array_equal(out.cpu().numpy(), want)
    plan.close()
    assert status() == skx.SKX_OK


def test_batch_rejects_too_many_groups(batch_data):
    fk = dev(batch_data["fk2"][:100])
    out = torch.empty(5000, dtype=torch.int64, device=DEV)
    with pytest.raises(skx.SkxError) as e:
        skx.skx_probe_batch(batch_data["d_dim2"], [(fk, fk, skx.Query.groupby_sum(num_groups=5000), out)])
    assert e.value.status == skx.SKX_ENOTSUP


# ------------------------------------------------------------------ errors
def test_key_and_group_range_errors():
    status()  # clear
    rows = dev(np.array([[0, 0, 1, 1], [5, 0, 1, 1]], dtype=np.int32))
    m = dev(np.ones(8, dtype=np.int32))
    q = skx.Query.groupby_sum(num_groups=3, filter_lt=10)
    skx.skx_probe_aggregate(rows, dev(np.array([0, 0, 0, 0, 0, 0, 0, 2], dtype=np.int32)), m, q,
                            tuning=skx.Tuning.plain())
    assert status() == skx.SKX_EKEYRANGE
    skx.skx_probe_aggregate(rows, dev(np.array([0, 1, 0, 0, 0, 0, 0, 0], dtype=np.int32)), m, q,
                            tuning=skx.Tuning.plain())
    assert status() == skx.SKX_EGROUPRANGE
    skx.skx_build_index(dev(np.array([0, 1, 9], dtype=np.int32)), 3)
    assert status() == skx.SKX_EKEYRANGE
    assert status() == skx.SKX_OK  # cleared
    with pytest.raises(skx.SkxError) as e:
        skx.skx_probe_aggregate(rows, dev(np.zeros(4, dtype=np.int32)), m[:4].contiguous(),
                                skx.Query.groupby_sum(num_groups=0))
    assert e.value.status == skx.SKX_EINVAL
    with pytest.raises(skx.SkxError):
        skx.skx_build_index(dev(np.zeros(4, dtype=np.int32)), 0)


# ------------------------------------------------------------------ whole path
def test_small_config_end_to_end():
    """N = 100K x 4 int32, F = 1M, Zipf s = 1.0, seed 0: build -> remap -> reorder -> probe."""
    w = synth.Workload(100_000, 1_000_000, 1.0, seed=0, width=4)
    fk, m, dim = w.fk(), w.measure(), w.dim()
    d_fk = dev(fk)
    idx = skx.skx_build_index(d_fk, w.n)
    fk2 = torch.empty_like(d_fk)
    skx.skx_remap(idx, d_fk, fk2)
    dim2 = torch.empty((w.n, 4), dtype=torch.int32, device=DEV)
    skx.skx_reorder(idx, dev(dim), dim2)
    got = skx.skx_probe_aggregate(dim2, fk2, dev(m), skx.Query.groupby_sum())
    plain = skx.skx_probe_aggregate(dev(dim), d_fk, dev(m), skx.Query.groupby_sum(), tuning=skx.Tuning.plain())
    want = oracle.probe(dim, fk, m, nthreads=8)
    assert np.array_equal(got.cpu().numpy(), want)
    assert np.array_equal(plain.cpu().numpy(), want)
    assert status() == skx.SKX_OK


def test_join_aggregate_host_api():
    w = synth.Workload(30_000, 400_001, 1.0, seed=8, width=16)
    fk, m, dim = w.fk(), w.measure(), w.dim()
    for qname in ("groupby", "sum", "count"):
        d = QUERIES[qname]
        got = skx.skx_join_aggregate_host(dim, fk, m, _q(d))
        assert np.array_equal(got, _oracle(dim, fk, m, d))


@pytest.mark.parametrize("f", [0, 1, 3, 7, 33, 4099, 1_000_003])
def test_join_aggregate_host_chunked_copies(f):
    """The host path copies the measure column in chunks cut on 16-byte
    boundaries and probes each as it lands: ragged and tiny columns, pinned
    host tensors, and a second call reusing the copy stream."""
    w = synth.Workload(5_000, f, 1.2, seed=19, width=16)
    fk, m, dim = w.fk(), w.measure(), w.dim()
    hfk = torch.from_numpy(fk).pin_memory()
    hm = torch.from_numpy(m).pin_memory()
    hdim = torch.from_numpy(dim).pin_memory()
    for qname in ("groupby", "count"):
        d = QUERIES[qname]
        want = _oracle(dim, fk, m, d)
        for _ in range(2):
            assert np.array_equal(skx.skx_join_aggregate_host(hdim, hfk, hm, _q(d)), want)


def test_autotune_choice_is_exact_and_cached(probe_data):
    d = QUERIES["groupby"]
    want = _oracle(probe_data["dim"], probe_data["fk"], probe_data["m"], d)
    q = _q(d)
    for remapped, rows, fk in [(True, probe_data["d_dim2"], probe_data["d_fk2"]),
                               (False, probe_data["d_dim"], probe_data["d_fk"])]:
        t, ms = skx.skx_probe_autotune(rows, fk, probe_data["d_m"], q, remapped=remapped)
        assert ms > 0
        if not remapped:
            assert t.hot_keys == -1
        got = skx.skx_probe_aggregate(rows, fk, probe_data["d_m"], q, tuning=t)
        assert np.array_equal(got.cpu().numpy(), want)
    # tuning = NULL picks up the cached remapped choice for this shape
    dflt = skx.skx_probe_default_tuning(probe_data["d_dim2"].shape[0], 64, probe_data["d_fk2"].numel(), q)
    t, _ = skx.skx_probe_autotune(probe_data["d_dim2"], probe_data["d_fk2"], probe_data["d_m"], q, remapped=True)
    dflt = skx.skx_probe_default_tuning(probe_data["d_dim2"].shape[0], 64, probe_data["d_fk2"].numel(), q)
    assert dflt.as_dict() == t.as_dict()
    got = skx.skx_probe_aggregate(probe_data["d_dim2"], probe_data["d_fk2"], probe_data["d_m"], q)
    assert np.array_equal(got.cpu().numpy(), want)
