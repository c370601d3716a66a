"""Multi-rank host logic on CPU with gloo (world_size 2): the bench's
max-over-ranks timing, rank-0-only reference arm, and the sharded form of the
path (per-rank counts and partial results over fact-row shards, summed by one
all-reduce each) checked against the unsharded oracle."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        from paper_1910_10063_gb300 import synth
        out = {}
        # max over ranks
        out["max"] = bench.max_over_ranks(10.0 + rank, dist, "cpu")
        # reference arm prints on rank 0 only
        out["ref_is_none"] = bench.run_reference(None, rank, world) is None if rank != 0 else None
        # sharded path: each rank owns a contiguous slice of the fact rows
        w = synth.Workload(5000, 200_003, 1.1, seed=3, width=4)
        fk, m, dim = w.fk(), w.measure(), w.dim()
        lo, hi = fk.size * rank // world, fk.size * (rank + 1) // world
        cnt = torch.from_numpy(oracle.histogram(fk[lo:hi], w.n).astype(np.int64))
        dist.all_reduce(cnt)  # the one integer all-reduce of the build
        part = torch.from_numpy(oracle.probe(dim, fk[lo:hi], m[lo:hi], num_groups=1000))
        dist.all_reduce(part)  # the one G-entry reduce of the probe (sums mod 2^64)
        out["cnt_ok"] = np.array_equal(cnt.numpy().astype(np.uint64), oracle.histogram(fk, w.n))
        out["probe_ok"] = np.array_equal(part.numpy(), oracle.probe(dim, fk, m, num_groups=1000))
        # every rank derives the same order from the reduced counts
        perm = oracle.sort_by_frequency(cnt.numpy().astype(np.uint64))
        g = [torch.zeros(w.n, dtype=torch.int32) for _ in range(world)]
        dist.all_gather(g, torch.from_numpy(perm))
        out["same_perm"] = all(torch.equal(g[0], x) for x in g)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r]["max"] == 11.0
        assert res[r]["cnt_ok"] and res[r]["probe_ok"] and res[r]["same_perm"]
    assert res[1]["ref_is_none"] is True
