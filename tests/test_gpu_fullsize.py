"""Parity at the full configured sizes, with the launch configurations bench.py
times (autotuned probe, whole-row reorder, batched plan, serving loop).

* 20M x 64-byte rows, 500M-row FK column: counts (both count algorithms), perm, rank, remap and
  reorder compared with the oracle element by element, and the probe result at
  Zipf s in {0, 0.5, 1.0, 1.5} on the remapped layout compared with the oracle
  on the original layout.
* 200M x 64-byte rows, 1B-row FK column (the largest cache-fit size): counts,
  perm, rank, remap, reorder and COUNT / SUM / GROUP BY SUM compared with the
  oracle element by element, with the size-free properties (bijection,
  inverse, non-increasing counts, ascending ids among ties, layout invariance)
  checked beside them.
* The drift variant (64M rows, 1B FK rows, 10 % of the ranks re-shuffled): the
  stale index's probe and the rebuilt index against the oracle.
* 512 batched queries and 256 served requests against the resident index,
  each compared with the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1910_10063_gb300 import synth  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1910_10063_gb300 as skx  # noqa: E402

DEV = torch.device("cuda:0")
N1, F1 = 20_000_000, 500_000_000
THREADS = 16


@pytest.fixture(scope="module")
def large():
    w = synth.DeviceWorkload(N1, F1, 1.0, seed=0, width=16, device=DEV)
    yield w
    del w
    torch.cuda.empty_cache()


def test_large_build_remap_reorder_exact(large):
    w = large
    idx = skx.skx_build_index(w.fk, N1)
    fk2 = torch.empty_like(w.fk)
    skx.skx_remap(idx, w.fk, fk2)
    dim2 = torch.empty_like(w.dim)
    skx.skx_reorder(idx, w.dim, dim2)
    assert skx.skx_stream_status() == skx.SKX_OK
    fk = w.fk.cpu().numpy()
    cnt, perm, rank = oracle.build_index(fk, N1)
    assert np.array_equal(idx.counts.cpu().numpy().view(np.uint32).astype(np.uint64), cnt)
    assert np.array_equal(idx.perm.cpu().numpy(), perm)
    assert np.array_equal(idx.rank.cpu().numpy(), rank)
    for method in (skx.SKX_COUNT_SINGLE_PASS, skx.SKX_COUNT_PARTITIONED):  # both count algorithms
        c = skx.skx_count_ex(w.fk, N1, method)
        assert np.array_equal(c.cpu().numpy().view(np.uint32).astype(np.uint64), cnt)
        del c
    assert np.array_equal(fk2.cpu().numpy(), oracle.remap(rank, fk))
    assert np.array_equal(dim2.cpu().numpy(), oracle.reorder(perm, w.dim.cpu().numpy()))
    idx.close()


def test_partitioned_count_at_its_size_limit():
    """The partitioned count at N = 2^28 ids (8192 buckets: the partition phase's shared memory
    just under the per-block limit) and 2^28 + 3 keys, exact against the oracle; one id more and
    the partitioned count is refused while the automatic count still answers (single pass)."""
    n, f = 1 << 28, (1 << 28) + 3
    w = synth.DeviceWorkload(n, f, 1.0, seed=14, width=1, device=DEV, with_measure=False, with_dim=False)
    want = oracle.histogram(w.fk.cpu().numpy(), n)
    c = skx.skx_count_ex(w.fk, n, skx.SKX_COUNT_PARTITIONED)
    assert skx.skx_stream_status() == skx.SKX_OK
    assert np.array_equal(c.cpu().numpy().view(np.uint32).astype(np.uint64), want)
    del c
    c = torch.empty(n + 1, dtype=torch.int32, device=DEV)
    with pytest.raises(skx.SkxError) as e:
        skx.skx_count_ex(w.fk, n + 1, skx.SKX_COUNT_PARTITIONED, counts=c)
    assert e.value.status == skx.SKX_ENOTSUP
    skx.skx_count(w.fk, n + 1, counts=c)
    got = c.cpu().numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(got[:n], want) and got[n] == 0
    del w, c
    torch.cuda.empty_cache()


@pytest.mark.parametrize("s", [0.0, 0.5, 1.0, 1.5])
def test_large_probe_exact(large, s):
    w = large
    fk = w.fk if s == 1.0 else synth.DeviceWorkload(N1, F1, s, seed=0, width=16, device=DEV, r2id=w.r2id_host,
                                                     with_measure=False, with_dim=False).fk
    idx = skx.skx_build_index(fk, N1)
    fk2 = torch.empty_like(fk)
    skx.skx_remap(idx, fk, fk2)
    dim2 = torch.empty_like(w.dim)
    skx.skx_reorder(idx, w.dim, dim2)
    q = skx.Query.groupby_sum()
    t, _ = skx.skx_probe_autotune(dim2, fk2, w.measure, q, remapped=True)
    got = skx.skx_probe_aggregate(dim2, fk2, w.measure, q, tuning=t).cpu().numpy()
    want = oracle.probe(w.dim.cpu().numpy(), fk.cpu().numpy(), w.measure.cpu().numpy(), nthreads=THREADS)
    assert np.array_equal(got, want)
    # the query copy path gives the same result: 8-byte rows (the lean kernel's launch, no hot
    # prefix), and the packed copy with the bench's launch (512 threads, as many CTAs as fit)
    q8 = skx.skx_reorder_query(idx, w.dim, q)
    got8 = skx.skx_probe_aggregate(q8, fk2, w.measure, skx.skx_query_prefiltered(q),
                                   tuning=skx.Tuning.plain()).cpu().numpy()
    assert np.array_equal(got8, want)
    p8, p4 = skx.skx_reorder_query_packed(idx, w.dim, q)
    assert torch.equal(p8, q8)
    gotp = skx.skx_probe_packed(p4, p8, fk2, w.measure, q).cpu().numpy()
    assert np.array_equal(gotp, want)
    idx.close()
    assert skx.skx_stream_status() == skx.SKX_OK


def _host_equal_chunked(dev_t, host_a, chunk=1 << 28):
    """dev_t (device tensor) equals host_a (numpy), compared in slices of the first axis."""
    n = dev_t.shape[0]
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        if not np.array_equal(dev_t[a:b].cpu().numpy(), host_a[a:b]):
            return False
    return True


def _index_properties(idx, fk, n, f):
    """Properties that hold at any size, checked on the device beside the exact comparison."""
    perm, rank = idx.perm, idx.rank
    cnt = idx.counts.view(torch.int32).to(torch.int64)
    ar = torch.arange(n, device=DEV, dtype=torch.int32)
    assert torch.equal(torch.sort(perm).values, ar)                         # bijection
    assert torch.equal(rank[perm.long()], ar)                               # rank is the inverse
    assert int(cnt.sum()) == f
    c_by_rank = cnt[perm.long()]
    assert bool((c_by_rank[1:] <= c_by_rank[:-1]).all())                    # decreasing frequency
    ties = c_by_rank[1:] == c_by_rank[:-1]
    assert bool((perm[1:][ties] > perm[:-1][ties]).all())                   # ascending ids among ties


QUERIES = {"groupby_sum": (oracle.AGG_GROUPBY_SUM, 1000), "count": (oracle.AGG_COUNT, 1),
           "sum": (oracle.AGG_SUM, 1)}


def _query(name):
    return {"groupby_sum": skx.Query.groupby_sum(), "count": skx.Query.count(), "sum": skx.Query.sum()}[name]


def test_cachefit_largest_exact():
    """The largest cache-fit point, 200M x 64-byte rows and 1B FK rows at Zipf s = 1.0, element by
    element against the oracle: counts, perm, rank, the remapped column, the reordered table, and
    COUNT / SUM / GROUP BY SUM on the remapped layout (autotuned, as the sweep times it) against the
    oracle's join over the original layout."""
    n, f = 200_000_000, 1_000_000_000
    w = synth.DeviceWorkload(n, f, 1.0, seed=2, width=16, device=DEV)
    idx = skx.skx_build_index(w.fk, n)
    fk2 = torch.empty_like(w.fk)
    skx.skx_remap(idx, w.fk, fk2)
    dim2 = torch.empty_like(w.dim)
    skx.skx_reorder(idx, w.dim, dim2)
    assert skx.skx_stream_status() == skx.SKX_OK
    _index_properties(idx, w.fk, n, f)
    got = {}
    for name in QUERIES:
        q = _query(name)
        t, _ = skx.skx_probe_autotune(dim2, fk2, w.measure, q, remapped=True)
        got[name] = skx.skx_probe_aggregate(dim2, fk2, w.measure, q, tuning=t).cpu().numpy()
        plain = skx.skx_probe_aggregate(w.dim, w.fk, w.measure, q, tuning=skx.Tuning.plain()).cpu().numpy()
        assert np.array_equal(plain, got[name])                             # layout invariance
    assert skx.skx_stream_status() == skx.SKX_OK

    fk_h = w.fk.cpu().numpy()
    cnt, perm, rank = oracle.build_index(fk_h, n)
    assert np.array_equal(idx.counts.cpu().numpy().view(np.uint32).astype(np.uint64), cnt)
    assert np.array_equal(idx.perm.cpu().numpy(), perm)
    assert np.array_equal(idx.rank.cpu().numpy(), rank)
    del cnt
    assert _host_equal_chunked(fk2, oracle.remap(rank, fk_h))
    dim_h = w.dim.cpu().numpy()
    assert _host_equal_chunked(dim2, oracle.reorder(perm, dim_h))
    m_h = w.measure.cpu().numpy()
    for name, (agg, g) in QUERIES.items():
        want = oracle.probe(dim_h, fk_h, m_h, agg, 1, 50, 0, g, 2 if agg != oracle.AGG_COUNT else -1,
                            nthreads=THREADS)
        assert np.array_equal(got[name], want), name
    idx.close()
    del w, fk2, dim2
    torch.cuda.empty_cache()


def test_cachefit_drift_exact():
    """The drift variant of the cache-fit sweep (64M x 64-byte rows, 1B FK rows; 10 % of the ranks
    re-shuffled): the stale index's probe of the drifted column and the rebuilt index, both against
    the oracle on the original keys."""
    n, f = 64_000_000, 1_000_000_000
    w = synth.DeviceWorkload(n, f, 1.0, seed=0, width=16, device=DEV)
    idx = skx.skx_build_index(w.fk, n)
    dim2 = torch.empty_like(w.dim)
    skx.skx_reorder(idx, w.dim, dim2)
    r2d = synth.drift_rank_to_id(w.r2id_host, 0, 0.1)
    wd = synth.DeviceWorkload(n, f, 1.0, seed=1, width=16, device=DEV, r2id=r2d, with_measure=False,
                              with_dim=False)
    q = skx.Query.groupby_sum()
    fks = torch.empty_like(wd.fk)
    skx.skx_remap(idx, wd.fk, fks)  # recode through the stale index
    t, _ = skx.skx_probe_autotune(dim2, fks, w.measure, q, remapped=True)
    stale = skx.skx_probe_aggregate(dim2, fks, w.measure, q, tuning=t).cpu().numpy()
    idx2 = skx.skx_build_index(wd.fk, n)
    skx.skx_remap(idx2, wd.fk, fks)
    dim3 = torch.empty_like(dim2)
    skx.skx_reorder(idx2, w.dim, dim3)
    fresh = skx.skx_probe_aggregate(dim3, fks, w.measure, q, tuning=t).cpu().numpy()
    assert skx.skx_stream_status() == skx.SKX_OK
    _index_properties(idx2, wd.fk, n, f)

    fkd_h = wd.fk.cpu().numpy()
    cnt, perm, rank = oracle.build_index(fkd_h, n)
    assert np.array_equal(idx2.counts.cpu().numpy().view(np.uint32).astype(np.uint64), cnt)
    assert np.array_equal(idx2.perm.cpu().numpy(), perm)
    assert np.array_equal(idx2.rank.cpu().numpy(), rank)
    dim_h = w.dim.cpu().numpy()
    assert _host_equal_chunked(fks, oracle.remap(rank, fkd_h))
    assert _host_equal_chunked(dim3, oracle.reorder(perm, dim_h))
    want = oracle.probe(dim_h, fkd_h, w.measure.cpu().numpy(), nthreads=THREADS)
    assert np.array_equal(stale, want)
    assert np.array_equal(fresh, want)
    idx.close()
    idx2.close()
    del w, wd, fks, dim2, dim3
    torch.cuda.empty_cache()


def test_batched_queries_exact(large):
    import bench
    w = large

    class A:
        n = N1
    queries = bench.batch_workload(A, w, DEV, 512)
    idx = skx.skx_build_index(w.fk, N1)
    dim2 = torch.empty_like(w.dim)
    skx.skx_reorder(idx, w.dim, dim2)
    items = []
    for fk, m, q, _ in queries:
        fk2 = torch.empty_like(fk)
        skx.skx_remap(idx, fk, fk2)
        items.append((fk2, m, q, torch.empty(q.nout, dtype=torch.int64, device=DEV)))
    plan = skx.BatchPlan(dim2, items)
    plan.autotune()
    plan.launch(use_graph=True)
    torch.cuda.synchronize()
    dim_h = w.dim.cpu().numpy()
    for (fk, m, q, _), (_, _, _, out) in zip(queries, items):
        want = oracle.probe(dim_h, fk.cpu().numpy(), m.cpu().numpy(), q.agg, q.filter_col, q.filter_lt, q.group_col,
                            q.num_groups, q.payload_col, nthreads=THREADS)
        assert np.array_equal(out.cpu().numpy(), want)
    plan.close()
    idx.close()


def test_served_requests_exact():
    n = 50_000_000
    ws = synth.DeviceWorkload(n, 25 * n, 1.0, seed=7, width=16, device=DEV, with_measure=False)
    idx = skx.skx_build_index(ws.fk, n)
    dim2 = torch.empty_like(ws.dim)
    skx.skx_reorder(idx, ws.dim, dim2)
    dim_h = ws.dim.cpu().numpy()
    r2id = ws.r2id_host
    del ws
    torch.cuda.empty_cache()
    rng = np.random.default_rng(9)
    sizes = synth.lognormal_sizes(256, 11)
    qdefs = [skx.Query.count(), skx.Query.sum(), skx.Query.groupby_sum()]
    cdf = {s: torch.from_numpy(synth.zipf_cdf(n, s)).to(DEV) for s in (0.8, 1.0, 1.2)}
    d_r2id = torch.from_numpy(r2id).to(DEV)
    reqs = []
    for i in range(256):
        s = float(rng.choice([0.8, 1.0, 1.2]))
        fk = synth.zipf_fk_device(cdf[s], d_r2id, 5000 + i, int(sizes[i])).cpu().pin_memory()
        m = synth.measure_device(5000 + i, int(sizes[i]), device=DEV).cpu().pin_memory()
        reqs.append((fk, m, qdefs[i % 3]))
    srv = skx.Server(dim2, idx.rank, skx.ServerConfig(max_inflight=64))
    tickets = [srv.submit(*r) for r in reqs]
    for t, (fk, m, q) in zip(tickets, reqs):
        want = oracle.probe(dim_h, fk.numpy(), m.numpy(), q.agg, q.filter_col, q.filter_lt, q.group_col,
                            q.num_groups, q.payload_col, nthreads=THREADS)
        assert np.array_equal(srv.wait(t), want)
    srv.close()
    idx.close()
