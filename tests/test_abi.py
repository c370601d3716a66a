"""The C-ABI libraries load and export every symbol their headers declare
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1910_10063_gb300")

HEADERS = {
    "skx.h": os.path.join(PKG, "libskx.so"),
    "skx_synth.h": os.path.join(PKG, "libskx_synth.so"),
}


def declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(skx_\w+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_t")))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1910_10063_gb300 import build
    build.build()


@pytest.mark.parametrize("header", list(HEADERS))
def test_exports_every_declared_symbol(header):
    lib = ctypes.CDLL(HEADERS[header])
    names = declared(header)
    assert names, header
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"{header}: not exported: {missing}"


def test_host_only_entry_points():
    lib = ctypes.CDLL(HEADERS["skx.h"])
    lib.skx_strerror.restype = ctypes.c_char_p
    lib.skx_strerror.argtypes = [ctypes.c_int]
    assert lib.skx_strerror(0) == b"SKX_OK"
    assert b"SKX_EKEYRANGE" in lib.skx_strerror(3)
    assert lib.skx_version() == (1 << 16)


def test_argument_errors_without_gpu():
    """Invalid arguments are rejected before any CUDA call."""
    import paper_1910_10063_gb300 as skx
    L = skx.lib()
    out = ctypes.c_void_p()
    assert L.skx_build_index(None, 10, 5, None, None) == skx.SKX_EINVAL
    assert L.skx_build_index(None, 10, 5, None, ctypes.byref(out)) == skx.SKX_EINVAL
    assert L.skx_build_index(None, 0, 0, None, ctypes.byref(out)) == skx.SKX_EINVAL
    q = skx.Query.groupby_sum(num_groups=0)
    assert L.skx_probe_aggregate(ctypes.c_void_p(16), 10, 16, ctypes.c_void_p(16), ctypes.c_void_p(16), 10,
                                 ctypes.byref(q), ctypes.c_void_p(16), None, None) == skx.SKX_EINVAL
    q = skx.Query.groupby_sum()
    assert L.skx_probe_aggregate(ctypes.c_void_p(16), 10, 18, ctypes.c_void_p(16), ctypes.c_void_p(16), 10,
                                 ctypes.byref(q), ctypes.c_void_p(16), None, None) == skx.SKX_EINVAL
    q.filter_col = 7
    assert L.skx_probe_aggregate(ctypes.c_void_p(16), 10, 16, ctypes.c_void_p(16), ctypes.c_void_p(16), 10,
                                 ctypes.byref(q), ctypes.c_void_p(16), None, None) == skx.SKX_EINVAL
    assert L.skx_remap(None, None, None, 5, None) == skx.SKX_EINVAL
    P = ctypes.c_void_p
    assert L.skx_count_ex(P(16), 10, 5, P(16), 7, None) == skx.SKX_EINVAL
    assert L.skx_count_ex(P(16), 10, 5, P(16), -1, None) == skx.SKX_EINVAL
    assert L.skx_count_ex(P(16), 1 << 32, 5, P(16), skx.SKX_COUNT_AUTO, None) == skx.SKX_EINVAL
    assert L.skx_count_ex(P(16), 10, (1 << 28) + 1, P(16), skx.SKX_COUNT_PARTITIONED, None) == skx.SKX_ENOTSUP
    # the packed query copy: key bits b with 2^b >= G + 2, G = num_groups (GROUP BY) or 1
    for g, bits in ((1, 2), (2, 2), (3, 3), (1000, 10), (1022, 10), (1023, 11), (1 << 24, 25)):
        assert L.skx_query_packed_key_bits(ctypes.byref(skx.Query(skx.SKX_AGG_GROUPBY_SUM, 1, 50, 0, g, 2))) == bits
    assert L.skx_query_packed_key_bits(ctypes.byref(skx.Query(skx.SKX_AGG_SUM, 1, 50, 0, 1, 2))) == 2
    assert L.skx_query_packed_key_bits(ctypes.byref(skx.Query(skx.SKX_AGG_COUNT, 1, 50, 0, 1, -1))) == 2
    assert L.skx_query_packed_key_bits(ctypes.byref(skx.Query(7, 1, 50, 0, 1, 2))) == -1
    assert L.skx_query_packed_key_bits(ctypes.byref(skx.Query(skx.SKX_AGG_GROUPBY_SUM, 1, 50, 0, 0, 2))) == -1
    q = skx.Query.groupby_sum()
    assert L.skx_reorder_query_packed(None, P(16), 10, 64, ctypes.byref(q), P(16), None, None) == skx.SKX_EINVAL
    assert L.skx_reorder_query_packed(None, P(16), 10, 64, ctypes.byref(q), P(4096), P(4098), None) == skx.SKX_EINVAL
    assert L.skx_probe_packed(None, P(16), 10, P(16), P(16), 10, ctypes.byref(q), P(16), None, None) == skx.SKX_EINVAL
    assert L.skx_probe_packed(P(16), P(16), 10, P(16), P(16), 1 << 32, ctypes.byref(q), P(16), None,
                              None) == skx.SKX_EINVAL


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1910_10063_gb300 as skx
    monkeypatch.setattr(skx, "_lib", None)
    monkeypatch.setattr(skx, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        skx.lib()
