// cache_model.cu -- the stack-distance cache model of Section III-C (host code).
//
// For L cache lines with access frequencies f_i and an LRU cache of S lines,
// line i's next reference is modelled as geometric with p = f_i.  Within k
// trials every other line j is expected n_j = k f_j / (1 - f_i) times, so the
// number of distinct lines seen is d(k) = k - sum_{j != i} max(0, n_j - 1).
// K_i is the smallest k >= S with d(k) >= S, equality taken up to rounding
// (relative 1e-9), found by binary search (infinite when fewer than S other
// lines are ever used), cdf_i = 1 - (1 - f_i)^K_i, and
// the estimated hit rate is sum_i f_i cdf_i.
//
// Fast evaluation: with the frequencies sorted in decreasing order g and
// prefix sums P, the lines with n_j > 1 are the prefix g_j > (1 - f_i) / k,
// so d(k) costs one binary search.  Lines are visited hottest first; past the
// hot lines that count among their own repeats, K_i can only fall as f_i
// falls and never below its value at f = 0, so once it reaches that value
// every colder line shares it.
#include <algorithm>
#include <cmath>
#include <vector>

#include "skx_internal.cuh"

namespace {

struct Model {
    std::vector<double> g;  // frequencies, decreasing
    std::vector<double> P;  // P[m] = g[0] + ... + g[m-1]
    int64_t used = 0;       // lines with f > 0

    // d(k) for a line of frequency fi that sits in g (self = true) or not.
    double d(double k, double fi, bool self) const {
        const double thr = (1.0 - fi) / k;  // n_j > 1  <=>  g_j > thr
        const int64_t m = std::upper_bound(g.begin(), g.end(), thr, std::greater<double>()) - g.begin();
        const bool self_in = self && fi > thr;
        const int64_t others = used - (self ? 1 : 0);
        // once every other used line repeats, sum_{j != i} n_j = k exactly and d = others
        if (m - (self_in ? 1 : 0) >= others) return double(others);
        double rep = (k / (1.0 - fi)) * P[m] - double(m);
        if (self_in) rep -= k * fi / (1.0 - fi) - 1.0;  // line i is not one of "the others"
        return k - rep;
    }

    // smallest integer k >= S with d(k) >= S (up to rounding), or infinity when it
    // is not reached before 64 / f (where 1 - (1 - f)^k is 1 to within e^-64)
    double K(double fi, bool self, int64_t S, double hi_hint, double fpos_min) const {
        const int64_t others = used - (self ? 1 : 0);
        if (others < S) return INFINITY;
        const double target = double(S) * (1.0 - 1e-9);
        const double kmax = std::ceil(64.0 / (fi > 0.0 ? fi : fpos_min)) + double(S);
        double lo = double(S), hi = std::min(kmax, std::max(double(S), hi_hint));
        while (hi < kmax && d(hi, fi, self) < target) hi = std::min(kmax, hi * 2.0 + 1.0);
        if (d(hi, fi, self) < target) return INFINITY;
        while (hi - lo >= 1.0) {
            const double mid = lo + std::floor((hi - lo) / 2.0);
            if (d(mid, fi, self) >= target) hi = mid;
            else lo = mid + 1.0;
        }
        return lo;
    }
};

// Evaluates the model: the hit rate and, when cdf is given, each line's hit
// probability in the order of f.
skx_status eval_model(const double *h_f, int64_t L, int64_t S, double *hit, double *cdf) {
    if (!h_f || L < 1 || S < 1) return SKX_EINVAL;
    Model m;
    std::vector<int64_t> order(L);
    for (int64_t j = 0; j < L; ++j) {
        if (!(h_f[j] >= 0.0)) return SKX_EINVAL;
        order[j] = j;
    }
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return h_f[x] > h_f[y]; });
    m.g.resize(L);
    for (int64_t j = 0; j < L; ++j) m.g[j] = h_f[order[j]];
    m.P.assign(L + 1, 0.0);
    for (int64_t j = 0; j < L; ++j) m.P[j + 1] = m.P[j] + m.g[j];
    m.used = std::lower_bound(m.g.begin(), m.g.end(), 0.0, std::greater<double>()) - m.g.begin();  // g > 0
    // K at the limit f_i -> 0.  Every line i that is not among its own repeated
    // lines (f_i K_i <= 1 - f_i) has d_i(k) <= d_floor(k), so K_i >= k_floor, and
    // for such lines K_i does not increase as f_i decreases; colder lines then
    // satisfy the same condition.  So once such a line has K_i == k_floor,
    // every colder line has K = k_floor too.
    const double fpos_min = m.used ? m.g[m.used - 1] : 1.0;  // smallest positive frequency
    const double k_floor = m.K(0.0, false, S, double(S), fpos_min);
    double h = 0.0, k_prev = INFINITY;
    bool at_floor = false, monotone = false;
    for (int64_t i = 0; i < m.used; ++i) {  // hottest first
        const double fi = m.g[i];
        double c;
        if (fi >= 1.0) {
            c = 1.0;
        } else {
            double Ki;
            if (at_floor) {
                Ki = k_floor;
            } else {
                Ki = m.K(fi, true, S, (monotone && !std::isinf(k_prev)) ? k_prev : double(S), fpos_min);
                monotone = !std::isinf(Ki) && fi * Ki <= 1.0 - fi;
                if (monotone && Ki == k_floor) at_floor = true;
            }
            k_prev = Ki;
            c = std::isinf(Ki) ? 1.0 : 1.0 - std::pow(1.0 - fi, Ki);
        }
        if (cdf) cdf[order[i]] = c;
        h += fi * c;
    }
    if (cdf)
        for (int64_t i = m.used; i < L; ++i) cdf[order[i]] = 0.0;  // never referenced
    if (hit) *hit = h;
    return SKX_OK;
}

}  // namespace

extern "C" {

skx_status skx_cache_hit_rate(const double *h_f, int64_t L, int64_t S, double *hit) {
    if (!hit) return SKX_EINVAL;
    return eval_model(h_f, L, S, hit, nullptr);
}

skx_status skx_cache_line_cdf(const double *h_f, int64_t L, int64_t S, double *h_cdf) {
    if (!h_cdf) return SKX_EINVAL;
    return eval_model(h_f, L, S, nullptr, h_cdf);
}

skx_status skx_cache_threshold(const double *h_f, int64_t L, int64_t S, double p, int32_t rows_per_line,
                               int64_t *t) {
    if (!t || rows_per_line < 1 || !(p > 0.0 && p <= 1.0)) return SKX_EINVAL;
    std::vector<double> cdf(L > 0 ? L : 1);
    const skx_status s = eval_model(h_f, L, S, nullptr, cdf.data());
    if (s != SKX_OK) return s;
    int64_t j = 0;
    while (j < L && cdf[j] >= p) ++j;
    *t = j * int64_t(rows_per_line);
    return SKX_OK;
}

skx_status skx_drift_from_counts(const uint32_t *h_counts_by_rank, int32_t N, int64_t t, double max_loss,
                                 skx_drift *out) {
    if (!h_counts_by_rank || !out || N < 1 || t < 1 || t > N || !(max_loss >= 0.0)) return SKX_EINVAL;
    uint64_t total = 0, stale = 0;
    for (int32_t r = 0; r < N; ++r) {
        total += h_counts_by_rank[r];
        if (r < t) stale += h_counts_by_rank[r];
    }
    if (total == 0) return SKX_EINVAL;
    // the t largest counts: what a rebuilt index would rank below t
    std::vector<uint32_t> c(h_counts_by_rank, h_counts_by_rank + N);
    std::nth_element(c.begin(), c.begin() + (t - 1), c.end(), std::greater<uint32_t>());
    uint64_t fresh = 0;
    for (int64_t r = 0; r < t; ++r) fresh += c[r];
    skx_drift d{};
    d.sample = int64_t(total);
    d.t = t;
    d.share_stale = double(stale) / double(total);
    d.share_fresh = double(fresh) / double(total);
    d.loss = d.share_fresh - d.share_stale;
    d.rebuild = d.loss > max_loss ? 1 : 0;
    *out = d;
    return SKX_OK;
}

skx_status skx_powerlaw_fit(const double *h_x, const double *h_y, int64_t n, double *slope, double *intercept) {
    if (!h_x || !h_y || n < 0 || !slope || !intercept) return SKX_EINVAL;
    // centred sums for the least-squares line through (log x, log y)
    int64_t m = 0;
    double sx = 0.0, sy = 0.0;
    for (int64_t k = 0; k < n; ++k)
        if (h_x[k] > 0.0 && h_y[k] > 0.0) {
            sx += std::log(h_x[k]);
            sy += std::log(h_y[k]);
            ++m;
        }
    if (m < 2) return SKX_EINVAL;
    const double mx = sx / double(m), my = sy / double(m);
    double sxx = 0.0, sxy = 0.0;
    for (int64_t k = 0; k < n; ++k)
        if (h_x[k] > 0.0 && h_y[k] > 0.0) {
            const double u = std::log(h_x[k]) - mx, v = std::log(h_y[k]) - my;
            sxx += u * u;
            sxy += u * v;
        }
    if (!(sxx > 0.0)) return SKX_EINVAL;  // all x equal: no line
    *slope = sxy / sxx;
    *intercept = my - *slope * mx;
    return SKX_OK;
}

// The split threshold of Section IV-B from the index, the paper's way: sample
// the value-frequency distribution (the index's counts at log-spaced ranks),
// fit it to a power law (a line in a log-log plot), and run the cache model
// on the fitted frequencies of the remapped table's lines.
skx_status skx_split_threshold(const skx_index *idx, int32_t row_bytes, int64_t cache_bytes, double p, int64_t *t,
                               void *stream) {
    if (!idx || !t || row_bytes < 4 || row_bytes % 4 != 0 || cache_bytes < 0 || !(p > 0.0 && p <= 1.0))
        return SKX_EINVAL;
    const int32_t N = skx_index_size(idx);
    if (N < 2) return SKX_EINVAL;
    constexpr int64_t kLine = 128;
    if (cache_bytes > 0 && cache_bytes < kLine) return SKX_EINVAL;
    if (cache_bytes == 0) {
        int dev = 0, l2 = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess ||
            l2 <= 0)
            return SKX_ECUDA;
        // the share of the L2 that a probe's dimension lines keep while the fact
        // columns stream past (measured with uniform keys: about two thirds)
        cache_bytes = int64_t(l2) * 2 / 3;
    }
    const int64_t S = std::max<int64_t>(1, cache_bytes / kLine);
    std::vector<int64_t> ranks;
    for (int k = 0; k < 48; ++k) {
        const int64_t r = int64_t(std::floor(std::exp(std::log(double(N)) * k / 47.0))) - 1;
        const int64_t rr = std::min<int64_t>(N - 1, std::max<int64_t>(0, r));
        if (ranks.empty() || rr > ranks.back()) ranks.push_back(rr);
    }
    std::vector<uint32_t> cnt(ranks.size());
    skx_status st = skx_index_counts_at_ranks(idx, ranks.data(), int64_t(ranks.size()), cnt.data(), stream);
    if (st != SKX_OK) return st;
    std::vector<double> x(ranks.size()), y(ranks.size());
    for (size_t k = 0; k < ranks.size(); ++k) {
        x[k] = double(ranks[k] + 1);
        y[k] = double(cnt[k]);
    }
    double slope = 0.0, icpt = 0.0;
    st = skx_powerlaw_fit(x.data(), y.data(), int64_t(x.size()), &slope, &icpt);
    if (st != SKX_OK) return st;
    return skx_split_threshold_from_fit(slope, N, row_bytes, S * kLine, p, t);
}

// The host half of skx_split_threshold: frequencies proportional to
// (r + 1)^slope over ranks r < N, summed per 128-byte line of the remapped
// table, and the model's threshold over S = cache_bytes / 128 lines.
skx_status skx_split_threshold_from_fit(double slope, int32_t N, int32_t row_bytes, int64_t cache_bytes, double p,
                                        int64_t *t) {
    constexpr int64_t kLine = 128;
    if (!t || N < 1 || row_bytes < 4 || row_bytes % 4 != 0 || cache_bytes < kLine || !(p > 0.0 && p <= 1.0) ||
        !std::isfinite(slope))
        return SKX_EINVAL;
    const int64_t S = cache_bytes / kLine;
    const int32_t rows_per_line = std::max<int32_t>(1, int32_t(kLine / row_bytes));
    const int64_t L = (int64_t(N) + rows_per_line - 1) / rows_per_line;
    std::vector<double> f(L, 0.0);
    double total = 0.0;
    for (int64_t r = 0; r < N; ++r) {
        const double w = std::pow(double(r + 1), slope);
        f[r / rows_per_line] += w;
        total += w;
    }
    if (!(total > 0.0)) return SKX_EINVAL;
    for (double &v : f) v /= total;
    const skx_status st = skx_cache_threshold(f.data(), L, S, p, rows_per_line, t);
    if (st == SKX_OK && *t > N) *t = N;
    return st;
}

}  // extern "C"
