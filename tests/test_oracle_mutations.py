"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch every one of them (no GPU; the real oracle source is never touched)."""
import os

import pytest

import oracle
from oracle_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(oracle.__file__), "skx_oracle.c")

# (name, exact text in skx_oracle.c, replacement)
MUTATIONS = [
    ("ascending_frequency", "return a->count > b->count ? -1 : 1;", "return a->count < b->count ? -1 : 1;"),
    ("tie_break_descending_id", "return a->id < b->id ? -1 : (a->id > b->id ? 1 : 0);",
     "return a->id > b->id ? -1 : (a->id < b->id ? 1 : 0);"),
    ("invert_transposed", "rank[v] = r;", "rank[r] = v;"),
    ("remap_dropped_rank", "fk_out[i] = rank[v];", "fk_out[i] = v;"),
    ("reorder_scatter_not_gather",
     "memcpy(dst + (size_t)r * (size_t)row_bytes,\n               src + (size_t)v * (size_t)row_bytes",
     "memcpy(dst + (size_t)v * (size_t)row_bytes,\n               src + (size_t)r * (size_t)row_bytes"),
    ("filter_not_strict", "!(row[j->filter_col] < j->filter_lt)", "!(row[j->filter_col] <= j->filter_lt)"),
    ("payload_wrong_column", "(int64_t)row[j->payload_col] : 1", "(int64_t)row[j->group_col] : 1"),
    ("dropped_measure", "(uint64_t)((int64_t)j->measure[i] * p)", "(uint64_t)(p)"),
    ("product_in_32_bits", "(uint64_t)((int64_t)j->measure[i] * p)", "(uint64_t)(int64_t)(int32_t)((int64_t)j->measure[i] * p)"),
    ("histogram_double_count", "cnt[v] += 1;", "cnt[v] += 1 + (v == 0);"),
    ("group_from_filter_column", "int32_t g = row[j->group_col];", "int32_t g = row[j->filter_col] % j->G;"),
    ("topk_drops_rank_zero", "if (r >= 0 && r < k)", "if (r > 0 && r < k)"),
    ("topk_off_by_one", "out[r] += 1;", "out[r > 0 ? r - 1 : 0] += 1;"),
    ("select_not_strict", "+ (size_t)filter_col] < filter_lt)", "+ (size_t)filter_col] <= filter_lt)"),
    ("select_wrong_offset", "offsets[c++] = (uint32_t)i;", "offsets[c++] = (uint32_t)v;"),
    ("append_new_ids_first", "perm_out[N + j] = N + j;", "perm_out[N + j] = j;"),
    ("cache_model_no_normalisation", "double n = k * f[j] / (1.0 - fi);", "double n = k * f[j];"),
    ("cache_model_cdf_exponent", "c = 1.0 - pow(1.0 - f[i], K);", "c = 1.0 - pow(1.0 - f[i], K + 1.0);"),
    ("threshold_counts_misses", "while (j < L && cdf[j] >= p)", "while (j < L && cdf[j] < p)"),
    ("threshold_ignores_rows_per_line", "*t = j * (int64_t)rows_per_line;", "*t = j;"),
    ("fit_no_log_of_x", "long double u = logl((long double)x[k])", "long double u = (long double)x[k]"),
    ("fit_slope_sign", "long double b = ((long double)m * suv - su * sv) / den;",
     "long double b = (su * sv - (long double)m * suv) / den;"),
    ("fit_intercept_plus", "*intercept = (double)((sv - b * su) / (long double)m);",
     "*intercept = (double)((sv + b * su) / (long double)m);"),
    ("materialize_wrong_stride", "out[i] = rows[(int64_t)v * row_words + col];", "out[i] = rows[(int64_t)v + col];"),
    ("materialize_no_recode_of_key", "int32_t v = fk[i];\n        if (v < 0 || v >= N)\n            return ORC_EKEY;\n        out[i]",
     "int32_t v = (int32_t)(i % N);\n        if (v < 0 || v >= N)\n            return ORC_EKEY;\n        out[i]"),
    ("thread_merge_drops_last", "for (int t = 0; t < nthreads; t++) {\n        if (jobs[t].status",
     "for (int t = 0; t < nthreads - (nthreads > 1); t++) {\n        if (jobs[t].status"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique/present"
    mutant_src = tmp_path / "mutant.c"
    mutant_src.write_text(src.replace(old, new))
    lib = oracle.load(oracle.build(str(mutant_src), str(tmp_path / "libmutant.so"), force=True))
    failures = 0
    for pin in ALL_PINS:
        try:
            pin(lib)
        except (AssertionError, oracle.OracleError):
            failures += 1
    assert failures > 0, f"no pin detects mutation {name}"
