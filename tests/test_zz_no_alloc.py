"""The allocation-free sort entry point, called through the C ABI.

skx_sort_by_count_noalloc serves callers that may not allocate device memory
when they order ids by frequency: a framework whose caching allocator already
holds nearly all of HBM, a latency-critical loop where an allocation could
synchronise the device or fail, or a plug-in that is handed fixed buffers.
Its scratch is a fixed array inside the library, shared by all calls and left
holding the previous call's data.  So the tests make calls in a row with
different sizes and both sort paths (the heavy/light split when F <= 64 N, the
plain LSD passes above), and check each result bit for bit against the oracle
and against the allocating skx_build_index_from_counts.  After a set-up call
(N = 0) has made the array resident, a call at the largest size must leave the
device's free memory unchanged.  This file sorts last so that a run stopping
at its first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_1910_10063_gb300 as skx  # noqa: E402
from paper_1910_10063_gb300 import synth  # noqa: E402


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_noalloc_sort_matches_oracle_and_allocating_sort_on_consecutive_calls():
    L = skx.lib()
    max_n = L.skx_sort_by_count_noalloc_max_n()
    assert max_n == 1 << 20
    assert L.skx_sort_by_count_noalloc(None, 0, 0, None, None, _stream()) == skx.SKX_OK  # set-up only
    # large then small (stale scratch), the split path and the plain LSD path (F > 64 N)
    cases = [(max_n, 5_000_000, 1.3, 1), (100_000, 1_000_000, 1.0, 0), (5_000, 2_000_000, 0.6, 3),
             (max_n, 3_000_000, 0.0, 4)]
    for n, f, s, seed in cases:
        w = synth.Workload(n, f, s, seed=seed)
        fk_h = w.fk()
        fk = torch.from_numpy(fk_h).cuda()
        counts = skx.skx_count(fk, n)
        ref = skx.skx_build_index_from_counts(counts, f)
        cnt_o = oracle.histogram(fk_h, n)
        perm_o = oracle.sort_by_frequency(cnt_o)
        rank_o = oracle.invert(perm_o)
        perm = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        rank = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        st = L.skx_sort_by_count_noalloc(_p(counts), n, f, _p(perm), _p(rank), _stream())
        assert st == skx.SKX_OK, L.skx_strerror(st)
        torch.cuda.synchronize()
        assert np.array_equal(perm.cpu().numpy(), perm_o)
        assert np.array_equal(rank.cpu().numpy(), rank_o)
        assert torch.equal(perm, ref.perm)
        assert torch.equal(rank, ref.rank)
        ref.close()
    assert skx.skx_stream_status() == skx.SKX_OK


def test_noalloc_sort_allocates_nothing():
    L = skx.lib()
    n, f = L.skx_sort_by_count_noalloc_max_n(), 4_000_000
    w = synth.Workload(n, f, 1.1, seed=5)
    fk = torch.from_numpy(w.fk()).cuda()
    counts = skx.skx_count(fk, n)
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    rank = torch.empty(n, dtype=torch.int32, device="cuda")
    assert L.skx_sort_by_count_noalloc(None, 0, 0, None, None, _stream()) == skx.SKX_OK
    assert L.skx_sort_by_count_noalloc(_p(counts), n, f, _p(perm), _p(rank), _stream()) == skx.SKX_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert L.skx_sort_by_count_noalloc(_p(counts), n, f, _p(perm), _p(rank), _stream()) == skx.SKX_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    perm_o = oracle.sort_by_frequency(oracle.histogram(fk.cpu().numpy(), n))
    assert np.array_equal(perm.cpu().numpy(), perm_o)
    assert skx.skx_stream_status() == skx.SKX_OK


def test_noalloc_sort_rejects_domain_beyond_its_array():
    L = skx.lib()
    n = L.skx_sort_by_count_noalloc_max_n() + 1
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    rank = torch.empty(n, dtype=torch.int32, device="cuda")
    st = L.skx_sort_by_count_noalloc(_p(counts), n, 10, _p(perm), _p(rank), None)
    assert st == skx.SKX_EINVAL


def test_noalloc_sort_reports_counts_beyond_the_bound():
    """Counts that break the bound F are data errors: reported, not silently truncated."""
    L = skx.lib()
    n = 8192  # two 4096-id tiles
    for f, fill in ((1000, 2000), (255 * 4, 300)):  # one count above F; more heavy ids than F / 255
        counts = torch.full((n,), fill, dtype=torch.int32, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        rank = torch.empty(n, dtype=torch.int32, device="cuda")
        assert L.skx_sort_by_count_noalloc(_p(counts), n, f, _p(perm), _p(rank), _stream()) == skx.SKX_OK
        assert skx.skx_stream_status() == skx.SKX_EINVAL
    assert skx.skx_stream_status() == skx.SKX_OK
