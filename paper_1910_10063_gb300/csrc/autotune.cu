// autotune.cu -- picks the probe's launch shape, hot-prefix threshold and
// split threshold by timing candidates on the caller's own data, and caches
// the choice.
//
// The threshold t of threshold-based processing (Section IV-B) depends on
// the skew and on the cache sizes; the paper derives it from a cost model or
// experimentally.  Here it is chosen experimentally per workload shape: each
// candidate (block size, 16-byte vectors per thread, CTAs per SM, t, lane
// copies) runs the probe on a prefix of the real fact column and the fastest
// wins.  The plain layout (no permutation index) is searched without a hot
// prefix, because its ids carry no frequency information.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "skx_internal.cuh"

namespace skx {
namespace {

using Key = std::tuple<int, int32_t, int32_t, int32_t, int, int>;  // device, N, row_bytes, agg, log2 F, remapped
std::mutex g_tune_mu;
std::map<Key, skx_tuning> g_tune_cache;

int log2_bucket(int64_t F) {
    int b = 0;
    while (b < 62 && (int64_t(1) << (b + 1)) <= F) ++b;
    return b;
}

Key key_of(int32_t N, int32_t row_bytes, const skx_query &q, int64_t F, int remapped) {
    int d = 0;
    cudaGetDevice(&d);
    return Key(d, N, row_bytes, q.agg, log2_bucket(F), remapped ? 1 : 0);
}

// Candidates of the split probe around the model's threshold t_model (Section
// IV-B): half, equal and twice t, with and without a shared-memory hot prefix,
// at the split kernels' 512 threads with one or as many CTAs per SM as fit.
void split_candidates(int32_t N, int32_t t_model, std::vector<skx_tuning> &c) {
    if (t_model <= 0) return;
    for (int64_t tm : {int64_t(t_model) / 2, int64_t(t_model), int64_t(t_model) * 2})
        for (int h : {-1, 2048, 8192})
            for (int cps : {-1, 1}) {
                if (tm <= (h > 0 ? h : 0) || tm >= N) continue;
                skx_tuning t{};
                t.block_threads = 512;
                t.unroll = 1;
                t.ctas_per_sm = cps;
                t.hot_keys = h;
                t.lane_keys = h == -1 ? -1 : 0;
                t.split_keys = (int32_t)tm;
                c.push_back(t);
            }
}

std::vector<skx_tuning> candidates(int remapped, int32_t N) {
    std::vector<skx_tuning> c;
    const int blocks[] = {256, 512};
    const int unrolls[] = {1, 2};
    const int hots_remapped[] = {-1, 1024, 4096, 16384, 0};
    for (int b : blocks)
        for (int u : unrolls)
            for (int cps : {0, 1024 / b, 2048 / b}) {
                if (remapped) {
                    for (int h : hots_remapped) {
                        if (h > N) continue;
                        skx_tuning t{};
                        t.block_threads = b;
                        t.unroll = u;
                        t.ctas_per_sm = cps == 0 ? -1 : cps;
                        t.hot_keys = h;
                        t.lane_keys = h == -1 ? -1 : 0;
                        c.push_back(t);
                    }
                } else {
                    skx_tuning t{};
                    t.block_threads = b;
                    t.unroll = u;
                    t.ctas_per_sm = cps == 0 ? -1 : cps;
                    t.hot_keys = -1;
                    t.lane_keys = -1;
                    c.push_back(t);
                }
            }
    return c;
}

}  // namespace

bool cached_probe_tuning(int32_t N, int32_t row_bytes, const skx_query &q, int64_t F, int remapped, skx_tuning *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key_of(N, row_bytes, q, F, remapped));
    if (it == g_tune_cache.end()) return false;
    *out = it->second;
    return true;
}

}  // namespace skx

using namespace skx;

extern "C" skx_status skx_probe_autotune_ex(const void *d_rows, int32_t N, int32_t row_bytes, const int32_t *d_fk,
                                            const int32_t *d_measure, int64_t F, const skx_query *q, int remapped,
                                            const skx_tuning *hint, int64_t *d_out, void *stream, skx_tuning *out,
                                            float *best_ms) {
    if (!out) return SKX_EINVAL;
    skx_status s = validate_query(q, row_bytes);
    if (s != SKX_OK) return s;
    if (N < 1 || F < 1 || F >= (int64_t(1) << 32) || !d_rows || !d_fk || !d_out ||
        (q->agg != SKX_AGG_COUNT && !d_measure))
        return SKX_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned *err = device_error_word();
    if (!err) return SKX_ENOMEM;
    const int64_t sample = std::min<int64_t>(F, int64_t(1) << 26);  // 64M rows is plenty to rank shapes
    ProbeArgs a{};
    a.rows = d_rows;
    a.N = N;
    a.row_bytes = row_bytes;
    a.fk = d_fk;
    a.measure = d_measure;
    a.F = sample;
    a.q = *q;
    a.out = d_out;
    a.err = err;
    cudaEvent_t e0, e1;
    SKX_CUDA_TRY(cudaEventCreate(&e0));
    SKX_CUDA_TRY(cudaEventCreate(&e1));
    // best of two runs of candidate t on the first `rows` fact rows (1e30 if it cannot launch)
    auto time_of = [&](skx_tuning t, int64_t rows) {
        ProbeArgs b = a;
        b.F = rows;
        resolve_probe_tuning(b, t);
        float ms_min = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {
            cudaEventRecord(e0, st);
            if (launch_probe(b, t, st) != cudaSuccess) ok = false;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_min = std::min(ms_min, ms);
        }
        cudaGetLastError();  // a candidate that cannot launch (resources) is skipped
        return std::make_pair(ok ? ms_min : 1e30f, t);
    };
    float best = 1e30f;
    skx_tuning best_t{};
    bool any = false;
    for (const skx_tuning &c : candidates(remapped, N)) {
        const auto r = time_of(c, sample);
        if (r.first < best) {
            best = r.first;
            best_t = r.second;
            any = true;
        }
    }
    // The split pays through cold rows that the whole column references several times, so a
    // short prefix understates it: its candidates and the best unsplit shape are timed again on
    // a longer prefix of up to 2^28 rows.
    std::vector<skx_tuning> sc;
    if (remapped && hint && hint->split_keys > 0) split_candidates(N, hint->split_keys, sc);
    int64_t rows_used = sample;
    if (!sc.empty() && any) {
        rows_used = std::min<int64_t>(F, int64_t(1) << 28);
        const auto base = time_of(best_t, rows_used);
        best = base.first;
        for (const skx_tuning &c : sc) {
            const auto r = time_of(c, rows_used);
            if (r.first < best) {
                best = r.first;
                best_t = r.second;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!any) return SKX_ECUDA;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key_of(N, row_bytes, *q, F, remapped)] = best_t;
    }
    *out = best_t;
    if (best_ms) *best_ms = best * float(F) / float(rows_used);
    return SKX_OK;
}

extern "C" skx_status skx_probe_autotune(const void *d_rows, int32_t N, int32_t row_bytes, const int32_t *d_fk,
                                         const int32_t *d_measure, int64_t F, const skx_query *q, int remapped,
                                         int64_t *d_out, void *stream, skx_tuning *out, float *best_ms) {
    return skx_probe_autotune_ex(d_rows, N, row_bytes, d_fk, d_measure, F, q, remapped, nullptr, d_out, stream, out,
                                 best_ms);
}
