"""Serving loop (continuous batching) through the C ABI: every result equals
the oracle, alone and in a concurrent mix; admission bounded by memory; bounded
waits."""
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
Q = {
    "groupby": (skx.Query.groupby_sum(), dict(agg=2, filter_col=1, filter_lt=50, group_col=0, num_groups=1000, payload_col=2)),
    "sum": (skx.Query.sum(), dict(agg=1, filter_col=1, filter_lt=50, group_col=0, num_groups=1, payload_col=2)),
    "count": (skx.Query.count(), dict(agg=0, filter_col=1, filter_lt=50, group_col=0, num_groups=1, payload_col=-1)),
    "groupby_attr1": (skx.Query.groupby_sum(num_groups=100, filter_col=1, filter_lt=90, group_col=1, payload_col=3),
                      dict(agg=2, filter_col=1, filter_lt=90, group_col=1, num_groups=100, payload_col=3)),
}


@pytest.fixture(scope="module")
def served():
    n = 300_000
    w = synth.Workload(n, 3_000_000, 1.0, seed=41, width=16)
    build_fk, dim = w.fk(), w.dim()
    idx = skx.skx_build_index(torch.from_numpy(build_fk).to(DEV), n)
    d_dim = torch.from_numpy(dim).to(DEV)
    dim2 = torch.empty_like(d_dim)
    skx.skx_reorder(idx, d_dim, dim2)
    rng = np.random.default_rng(3)
    reqs = []
    sizes = [0, 1, 7, 4096, 65537, 200_000, 1_500_000, 33, 250_001, 10_000, 3, 999_999]
    names = list(Q)
    for i, f in enumerate(sizes * 2):
        wr = synth.Workload(n, f, float(rng.choice([0.8, 1.0, 1.2])), seed=100 + i, width=16, r2id=w.r2id)
        fk = torch.from_numpy(wr.fk()).pin_memory() if f else torch.zeros(0, dtype=torch.int32)
        m = torch.from_numpy(wr.measure()).pin_memory() if f else torch.zeros(0, dtype=torch.int32)
        name = names[i % len(names)]
        want = oracle.probe(dim, fk.numpy(), m.numpy(), nthreads=8, **{k: v for k, v in Q[name][1].items()})
        reqs.append((fk, m, Q[name][0], want))
    return dict(idx=idx, dim2=dim2, rank=idx.rank, reqs=reqs, n=n, dim=dim)


def test_server_results_alone_and_in_mix(served):
    alone = skx.Server(served["dim2"], served["rank"], skx.ServerConfig(max_inflight=1))
    solo = [alone.wait(alone.submit(fk, m, q)) for fk, m, q, _ in served["reqs"]]
    alone.close()
    mix = skx.Server(served["dim2"], served["rank"], skx.ServerConfig(max_inflight=16, tile_rows=8192,
                                                                      round_rows=300_000))
    tickets = [mix.submit(fk, m, q) for fk, m, q, _ in served["reqs"]]
    together = [mix.wait(t) for t in tickets]
    st = mix.stats()
    mix.close()
    assert st["rounds"] > 1 and st["max_active"] > 1  # requests really shared rounds
    for (fk, m, q, want), a, b in zip(served["reqs"], solo, together):
        assert np.array_equal(a, want)
        assert np.array_equal(b, want)
    assert skx.skx_stream_status() == skx.SKX_OK


def test_server_replay_poisson(served):
    srv = skx.Server(served["dim2"], served["rank"], skx.ServerConfig(max_inflight=8))
    reqs = [srv.make_request(fk, m, q) for fk, m, q, _ in served["reqs"]]
    arrivals = np.cumsum(np.random.default_rng(0).exponential(200e-6, size=len(reqs)))
    lat = srv.replay(reqs, arrivals)
    srv.close()
    assert np.all(lat > 0)
    for (req, keep), (_, _, _, want) in zip(reqs, served["reqs"]):
        assert np.array_equal(keep[2], want)


def test_server_admission_by_memory(served):
    # an arena that holds about one mid-size request at a time; never more in flight than fit
    big = max(fk.numel() for fk, _, _, _ in served["reqs"])
    cfg = skx.ServerConfig(max_inflight=8, memory_budget=8 * big + (1 << 20))
    srv = skx.Server(served["dim2"], served["rank"], cfg)
    tickets = [srv.submit(fk, m, q) for fk, m, q, _ in served["reqs"]]
    for t, (_, _, _, want) in zip(tickets, served["reqs"]):
        assert np.array_equal(srv.wait(t), want)
    need = sorted(2 * ((fk.numel() * 4 + 255) // 256 * 256) + (q.nout * 8 + 255) // 256 * 256
                  for fk, _, q, _ in served["reqs"])
    fit = int(np.searchsorted(np.cumsum(need), cfg.memory_budget, side="right"))  # the most that fit at once
    assert 1 <= srv.stats()["max_active"] <= min(fit, cfg.max_inflight)
    # a request that can never fit the arena is refused at submit
    huge = torch.zeros(cfg.memory_budget // 4, dtype=torch.int32)
    with pytest.raises(skx.SkxError) as e:
        srv.submit(huge, huge, skx.Query.sum())
    assert e.value.status == skx.SKX_ENOMEM
    srv.close()


def test_server_bounded_wait(served):
    """A wait of 0 ms right after submitting a 100M-row request cannot see it finished (its keys
    alone take milliseconds to copy): SKX_ETIMEOUT, deterministically; a patient wait then gets
    the exact result."""
    n = served["n"]
    keys = synth.DeviceWorkload(n, 100_000_000, 1.0, seed=44, width=16, device=DEV, r2id=None,
                                with_measure=False, with_dim=False).fk
    fk = torch.empty(keys.numel(), dtype=torch.int32, pin_memory=True)
    fk.copy_(keys)
    del keys
    srv = skx.Server(served["dim2"], served["rank"])
    t = srv.submit(fk, None, skx.Query.count())
    assert skx.lib().skx_server_wait(srv._h, t, 0) == skx.SKX_ETIMEOUT
    want = oracle.probe(served["dim"], fk.numpy(), None, agg=0, filter_col=1, filter_lt=50, group_col=0,
                        num_groups=1, payload_col=-1, nthreads=16)
    assert np.array_equal(srv.wait(t), want)
    assert skx.lib().skx_server_wait(srv._h, 123456789, 10) == skx.SKX_EINVAL
    srv.close()


def test_server_admission_limited_by_the_arena(served):
    """Six 1M-row requests against an arena that holds two of them: never more than two are in
    flight, two are, and every result is exact."""
    n = served["n"]
    reqs = []
    for i in range(6):
        wr = synth.Workload(n, 1_000_000, 1.0, seed=300 + i, width=16)
        fk = torch.from_numpy(wr.fk()).pin_memory()
        m = torch.from_numpy(wr.measure()).pin_memory()
        want = oracle.probe(served["dim"], fk.numpy(), m.numpy(), nthreads=8)
        reqs.append((fk, m, want))
    one = 2 * ((1_000_000 * 4 + 255) // 256 * 256) + 4096 * 8  # keys, measures and an output slot
    cfg = skx.ServerConfig(max_inflight=8, memory_budget=int(2.5 * one))
    srv = skx.Server(served["dim2"], served["rank"], cfg)
    tickets = [srv.submit(fk, m, skx.Query.groupby_sum()) for fk, m, _ in reqs]
    for t, (_, _, want) in zip(tickets, reqs):
        assert np.array_equal(srv.wait(t), want)
    st = srv.stats()
    srv.close()
    assert st["max_active"] == 2, st


def test_server_round_deadline_expires():
    """A round that outlives the server's bound on waits for the device (timeout_ms = 1) fails its
    requests with SKX_ETIMEOUT instead of waiting on; the server is then closed cleanly and the
    device is unaffected.  The rounds are made slow on purpose: 100M uniform keys per round over a
    20M x 64-byte table (every gather a DRAM miss, about 2 ms a round)."""
    n = 20_000_000
    w = synth.DeviceWorkload(n, 300_000_000, 0.0, seed=45, width=16, device=DEV, with_measure=False)
    fk = torch.empty(w.fk.numel(), dtype=torch.int32, pin_memory=True)
    fk.copy_(w.fk)
    cfg = skx.ServerConfig(round_rows=100_000_000, timeout_ms=1)
    srv = skx.Server(w.dim, None, cfg)  # keys already in table order: no recode
    t = srv.submit(fk, None, skx.Query.count())
    st = skx.lib().skx_server_wait(srv._h, t, 60_000)
    assert st == skx.SKX_ETIMEOUT
    srv.close()
    assert skx.skx_stream_status() == skx.SKX_OK
    del w, fk
    torch.cuda.empty_cache()
