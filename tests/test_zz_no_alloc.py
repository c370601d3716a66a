"""The allocation-free sort entry point, called through the C ABI, against the
allocating one.

skx_sort_by_count_noalloc serves callers that may not allocate device memory
when they order ids by frequency (a framework that already reserved HBM, a
latency-critical loop, a plug-in handed fixed buffers).  Its scratch is a fixed
array inside the library, shared by all calls and left holding the previous
call's data, so the test makes two calls in a row with different sizes and
checks each result bit for bit against skx_build_index_from_counts.  This file
sorts last so that a run stopping at its first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1910_10063_gb300 as skx  # noqa: E402
from paper_1910_10063_gb300 import synth  # noqa: E402


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_sort_matches_allocating_sort_on_consecutive_calls():
    L = skx.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    max_n = L.skx_sort_by_count_noalloc_max_n()
    assert max_n == 1 << 20
    cases = [(max_n, 5_000_000, 1.3, 1), (100_000, 1_000_000, 1.0, 0)]  # large then small: stale scratch
    for n, f, s, seed in cases:
        w = synth.Workload(n, f, s, seed=seed)
        fk = torch.from_numpy(w.fk()).cuda()
        counts = skx.skx_count(fk, n)
        ref = skx.skx_build_index_from_counts(counts, f)
        perm = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        rank = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        st = L.skx_sort_by_count_noalloc(_p(counts), n, f, _p(perm), _p(rank), stream)
        assert st == skx.SKX_OK, skx.lib().skx_strerror(st)
        torch.cuda.synchronize()
        assert torch.equal(perm, ref.perm)
        assert torch.equal(rank, ref.rank)
        ref.close()
    assert skx.skx_stream_status() == skx.SKX_OK


def test_noalloc_sort_rejects_domain_beyond_its_array():
    L = skx.lib()
    n = L.skx_sort_by_count_noalloc_max_n() + 1
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    rank = torch.empty(n, dtype=torch.int32, device="cuda")
    st = L.skx_sort_by_count_noalloc(_p(counts), n, 10, _p(perm), _p(rank), None)
    assert st == skx.SKX_EINVAL
