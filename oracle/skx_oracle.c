/*
 * skx_oracle.c -- CPU oracle for the permutation index.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of what the GPU path computes, used by the tests, by the
 * smoke check and by the benchmark's CPU-baseline leg.  The product path
 * never calls it, and it shares no code with the CUDA sources.
 *
 * Source: W. Zhang and K. A. Ross, "Exploiting Data Skew for Improved Query
 * Performance", ICDE 2020 (extended version, arXiv 1910.10063).
 *
 *   Section III      the permutation index: the values of column C in
 *                    decreasing frequency order (offset representation),
 *                    and the popularity rank of each dimension row (rank
 *                    representation); both are kept so lookups in either
 *                    direction are O(1).
 *   Section III-A    building = a Q3 count of each value + a sort of the
 *                    values by frequency + a Q1-style recode C'[i] = Rank(C[i]).
 *   Section III-B    a query works on a copy of the needed dimension rows
 *                    permuted by the index (offset order).
 *   Section I, IV-A  Q1 gather through the FK, Q2 filter on a dimension
 *                    attribute, aggregation over the result.
 *   Section IV-C     intra-query parallelism: non-overlapping fact chunks
 *                    per thread, each with its own independent result
 *                    buffer, combined at the end.
 *
 * Readings where the paper is silent (each one is also listed in the design
 * notes): ids are 0-based; equal counts are ordered by ascending id; ids that
 * never occur get count 0 and follow all occurring ids (ascending id), so the
 * permutation is a bijection on [0, N); counts are uint64; the aggregate
 * product measure*payload is formed in int64 and summed with wrap-around
 * modulo 2^64 (reported as int64); the filter is a strict "<".
 *
 * Every entry point returns 0 on success, ORC_EKEY when an FK is outside
 * [0, N), ORC_EGROUP when a group key is outside [0, G), ORC_EINVAL on bad
 * arguments.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <math.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_EKEY 3
#define ORC_EGROUP 4

#define ORC_AGG_COUNT 0
#define ORC_AGG_SUM 1
#define ORC_AGG_GROUPBY_SUM 2

/* ------------------------------------------------------------------------
 * Q3 (Section I; first step of the build, Section III-A):
 * cnt[v] = number of rows i with fk[i] == v.
 */
int orc_histogram(const int32_t *fk, int64_t F, int32_t N, uint64_t *cnt)
{
    if (F < 0 || N < 0 || (F > 0 && (!fk || N == 0)) || (N > 0 && !cnt))
        return ORC_EINVAL;
    for (int32_t v = 0; v < N; v++)
        cnt[v] = 0;
    for (int64_t i = 0; i < F; i++) {
        int32_t v = fk[i];
        if (v < 0 || v >= N)
            return ORC_EKEY;
        cnt[v] += 1;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Sort by frequency (Section III, offset representation; Section III-A):
 * perm[r] = the id with the r-th largest count; ties by ascending id.
 */
typedef struct {
    uint64_t count;
    int32_t id;
} orc_item;

static int orc_cmp_item(const void *pa, const void *pb)
{
    const orc_item *a = (const orc_item *)pa, *b = (const orc_item *)pb;
    if (a->count != b->count)
        return a->count > b->count ? -1 : 1; /* decreasing frequency */
    return a->id < b->id ? -1 : (a->id > b->id ? 1 : 0);
}

int orc_sort_by_frequency(const uint64_t *cnt, int32_t N, int32_t *perm)
{
    if (N < 0 || (N > 0 && (!cnt || !perm)))
        return ORC_EINVAL;
    if (N == 0)
        return ORC_OK;
    orc_item *items = (orc_item *)malloc(sizeof(orc_item) * (size_t)N);
    if (!items)
        return ORC_EINVAL;
    for (int32_t v = 0; v < N; v++) {
        items[v].count = cnt[v];
        items[v].id = v;
    }
    qsort(items, (size_t)N, sizeof(orc_item), orc_cmp_item);
    for (int32_t r = 0; r < N; r++)
        perm[r] = items[r].id;
    free(items);
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Rank representation (Section III): rank[perm[r]] = r.
 */
int orc_invert(const int32_t *perm, int32_t N, int32_t *rank)
{
    if (N < 0 || (N > 0 && (!perm || !rank)))
        return ORC_EINVAL;
    for (int32_t r = 0; r < N; r++) {
        int32_t v = perm[r];
        if (v < 0 || v >= N)
            return ORC_EKEY;
        rank[v] = r;
    }
    return ORC_OK;
}

/* Whole build (Section III-A): count, sort by frequency, invert. */
int orc_build_index(const int32_t *fk, int64_t F, int32_t N, uint64_t *cnt,
                    int32_t *perm, int32_t *rank)
{
    int st = orc_histogram(fk, F, N, cnt);
    if (st)
        return st;
    st = orc_sort_by_frequency(cnt, N, perm);
    if (st)
        return st;
    return orc_invert(perm, N, rank);
}

/* ------------------------------------------------------------------------
 * Recode of the fact column (Section III-A): fk_out[i] = rank[fk[i]].
 */
int orc_remap(const int32_t *rank, int32_t N, const int32_t *fk, int64_t F,
              int32_t *fk_out)
{
    if (F < 0 || N < 0 || (F > 0 && (!rank || !fk || !fk_out)))
        return ORC_EINVAL;
    for (int64_t i = 0; i < F; i++) {
        int32_t v = fk[i];
        if (v < 0 || v >= N)
            return ORC_EKEY;
        fk_out[i] = rank[v];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Permuted copy of the dimension rows (Section III-B):
 * rows_out[r] = rows[perm[r]], row_bytes bytes each.
 */
int orc_reorder(const int32_t *perm, int32_t N, const void *rows,
                int32_t row_bytes, void *rows_out)
{
    if (N < 0 || row_bytes <= 0 || (N > 0 && (!perm || !rows || !rows_out)))
        return ORC_EINVAL;
    const unsigned char *src = (const unsigned char *)rows;
    unsigned char *dst = (unsigned char *)rows_out;
    for (int32_t r = 0; r < N; r++) {
        int32_t v = perm[r];
        if (v < 0 || v >= N)
            return ORC_EKEY;
        memcpy(dst + (size_t)r * (size_t)row_bytes,
               src + (size_t)v * (size_t)row_bytes, (size_t)row_bytes);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * FK-join probe + filter + aggregate (Sections I and IV-A: Q1 gathers the
 * dimension row through the FK used as an array offset, Q2 keeps rows whose
 * dimension attribute passes "col < c", the aggregation sums per group).
 *
 *   COUNT        out[0] = #{i : dim[fk[i]].filter < c}
 *   SUM          out[0] = sum_i measure[i] * dim[fk[i]].payload   (filtered)
 *   GROUPBY_SUM  out[g] = same sum restricted to dim[fk[i]].group == g
 *
 * filter_col < 0 means "no filter"; payload_col < 0 means payload 1.
 * Rows are int32[row_words] records; column c is word c of the row.
 */
typedef struct {
    const int32_t *rows;
    int32_t N, row_words;
    const int32_t *fk, *measure;
    int64_t begin, end;
    int agg, filter_col, group_col, payload_col;
    int32_t filter_lt, G;
    uint64_t *out; /* private buffer, G entries (1 for COUNT/SUM) */
    int status;
} orc_probe_job;

static void orc_probe_range(orc_probe_job *j)
{
    j->status = ORC_OK;
    for (int64_t i = j->begin; i < j->end; i++) {
        int32_t v = j->fk[i];
        if (v < 0 || v >= j->N) {
            j->status = ORC_EKEY;
            return;
        }
        const int32_t *row = j->rows + (size_t)v * (size_t)j->row_words;
        if (j->filter_col >= 0 && !(row[j->filter_col] < j->filter_lt))
            continue;
        if (j->agg == ORC_AGG_COUNT) {
            j->out[0] += 1;
            continue;
        }
        int64_t p = j->payload_col >= 0 ? (int64_t)row[j->payload_col] : 1;
        uint64_t prod = (uint64_t)((int64_t)j->measure[i] * p);
        if (j->agg == ORC_AGG_SUM) {
            j->out[0] += prod;
        } else {
            int32_t g = row[j->group_col];
            if (g < 0 || g >= j->G) {
                j->status = ORC_EGROUP;
                return;
            }
            j->out[g] += prod;
        }
    }
}

static void *orc_probe_thread(void *arg)
{
    orc_probe_range((orc_probe_job *)arg);
    return NULL;
}

int orc_probe(const int32_t *rows, int32_t N, int32_t row_words,
              const int32_t *fk, const int32_t *measure, int64_t F, int agg,
              int filter_col, int32_t filter_lt, int group_col, int32_t G,
              int payload_col, uint64_t *out, int nthreads)
{
    if (F < 0 || N < 0 || row_words <= 0 || !out)
        return ORC_EINVAL;
    if (agg < ORC_AGG_COUNT || agg > ORC_AGG_GROUPBY_SUM)
        return ORC_EINVAL;
    if (filter_col >= row_words || payload_col >= row_words)
        return ORC_EINVAL;
    if (agg == ORC_AGG_GROUPBY_SUM && (G <= 0 || group_col < 0 || group_col >= row_words))
        return ORC_EINVAL;
    if (F > 0 && (!rows || !fk || (agg != ORC_AGG_COUNT && !measure)))
        return ORC_EINVAL;
    int32_t nout = agg == ORC_AGG_GROUPBY_SUM ? G : 1;
    if (nthreads < 1)
        nthreads = 1;
    if ((int64_t)nthreads > F)
        nthreads = F > 0 ? (int)F : 1;

    orc_probe_job *jobs = (orc_probe_job *)calloc((size_t)nthreads, sizeof(orc_probe_job));
    uint64_t *bufs = (uint64_t *)calloc((size_t)nthreads * (size_t)nout, sizeof(uint64_t));
    pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !bufs || !tids) {
        free(jobs); free(bufs); free(tids);
        return ORC_EINVAL;
    }
    for (int t = 0; t < nthreads; t++) {
        orc_probe_job *j = &jobs[t];
        j->rows = rows; j->N = N; j->row_words = row_words;
        j->fk = fk; j->measure = measure;
        j->begin = F * t / nthreads;
        j->end = F * (t + 1) / nthreads;
        j->agg = agg; j->filter_col = filter_col; j->group_col = group_col;
        j->payload_col = payload_col; j->filter_lt = filter_lt; j->G = G;
        j->out = bufs + (size_t)t * (size_t)nout;
    }
    int spawned = 0;
    for (int t = 1; t < nthreads; t++) {
        if (pthread_create(&tids[t], NULL, orc_probe_thread, &jobs[t]) != 0)
            break;
        spawned = t;
    }
    orc_probe_range(&jobs[0]);
    for (int t = 1; t <= spawned; t++)
        pthread_join(tids[t], NULL);
    for (int t = spawned + 1; t < nthreads; t++) /* threads that failed to start */
        orc_probe_range(&jobs[t]);

    int status = ORC_OK;
    for (int32_t g = 0; g < nout; g++)
        out[g] = 0;
    for (int t = 0; t < nthreads; t++) {
        if (jobs[t].status && !status)
            status = jobs[t].status;
        for (int32_t g = 0; g < nout; g++)
            out[g] += jobs[t].out[(size_t)g];
    }
    free(jobs); free(bufs); free(tids);
    return status;
}

/* ------------------------------------------------------------------------
 * Heavy-hitter counts (Section I, query Q3a; Section IV-B): with an up-to-date
 * index the k most frequent values are the transformed ids 0..k-1, so the
 * query counts only those: out[r] = #{i : fk_remapped[i] == r}, r < k.  Keys
 * outside [0, k) are ignored.
 */
int orc_topk_counts(const int32_t *fk_remapped, int64_t F, int32_t k, uint64_t *out)
{
    if (F < 0 || k < 1 || !out || (F > 0 && !fk_remapped))
        return ORC_EINVAL;
    for (int32_t r = 0; r < k; r++)
        out[r] = 0;
    for (int64_t i = 0; i < F; i++) {
        int32_t r = fk_remapped[i];
        if (r >= 0 && r < k)
            out[r] += 1;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Selection (Section I, query Q2; Section IV-A): the offsets i, in increasing
 * order, of the fact rows whose dimension row passes "col < c"; *count is
 * their number.  offsets must hold F entries.
 */
int orc_select(const int32_t *rows, int32_t N, int32_t row_words, const int32_t *fk, int64_t F,
               int filter_col, int32_t filter_lt, uint32_t *offsets, int64_t *count)
{
    if (F < 0 || N < 0 || row_words <= 0 || filter_col < 0 || filter_col >= row_words || !count ||
        (F > 0 && (!rows || !fk || !offsets)))
        return ORC_EINVAL;
    int64_t c = 0;
    for (int64_t i = 0; i < F; i++) {
        int32_t v = fk[i];
        if (v < 0 || v >= N)
            return ORC_EKEY;
        if (rows[(size_t)v * (size_t)row_words + (size_t)filter_col] < filter_lt)
            offsets[c++] = (uint32_t)i;
    }
    *count = c;
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Index maintenance (Section III-A): n_new dimension rows appended to a
 * table of N rows get the ids N..N+n_new-1 and enter the permutation index at
 * its end as the new least frequent items; existing ranks are unchanged.
 */
int orc_index_append(const int32_t *perm, const int32_t *rank, int32_t N, int32_t n_new,
                     int32_t *perm_out, int32_t *rank_out)
{
    if (N < 0 || n_new < 0 || (N > 0 && (!perm || !rank)) || !perm_out || !rank_out)
        return ORC_EINVAL;
    for (int32_t r = 0; r < N; r++) {
        perm_out[r] = perm[r];
        rank_out[r] = rank[r];
    }
    for (int32_t j = 0; j < n_new; j++) {
        perm_out[N + j] = N + j;
        rank_out[N + j] = N + j;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Cache model (Section III-C).  f[0..L) are the access frequencies of L cache
 * lines (sum 1), S the cache size in lines.  For line i and k trials, each
 * other line j is expected n_j = k f_j / (1 - f_i) times; the number of
 * distinct lines is d(k) = k - sum_{j != i} max(0, n_j - 1).  K_i is found by
 * binary search over k >= S as the smallest k with d(k) >= S, equality taken up
 * to rounding (relative 1e-9); K_i is infinite when d never reaches S, i.e.
 * when fewer than S other lines are ever used;
 * cdf_i = 1 - (1 - f_i)^K_i and the hit rate is sum_i f_i cdf_i.  Plain
 * O(L) evaluation of d(k).  cdf may be NULL.
 */
static double orc_cache_d(const double *f, int64_t L, int64_t i, double k, int64_t others)
{
    double fi = f[i], rep = 0.0;
    int64_t repeating = 0;
    for (int64_t j = 0; j < L; j++) {
        if (j == i)
            continue;
        double n = k * f[j] / (1.0 - fi);
        if (n > 1.0) {
            rep += n - 1.0;
            repeating++;
        }
    }
    /* once every other used line repeats, sum_{j != i} n_j = k exactly and
     * d(k) = others; computing it directly avoids cancellation at large k */
    if (repeating == others)
        return (double)others;
    return k - rep;
}

int orc_cache_hit_rate(const double *f, int64_t L, int64_t S, double *hit, double *cdf)
{
    if (!f || L < 1 || S < 1 || !hit)
        return ORC_EINVAL;
    int64_t used = 0;
    double f_pos_min = 1.0;
    for (int64_t j = 0; j < L; j++) {
        if (f[j] < 0.0)
            return ORC_EINVAL;
        if (f[j] > 0.0) {
            used++;
            if (f[j] < f_pos_min)
                f_pos_min = f[j];
        }
    }
    double h = 0.0;
    for (int64_t i = 0; i < L; i++) {
        double c;
        int64_t others = used - (f[i] > 0.0 ? 1 : 0);
        if (f[i] <= 0.0) {
            c = 0.0;
        } else if (f[i] >= 1.0) {
            c = 1.0;
        } else if (others < S) {
            c = 1.0; /* d(k) <= others < S for every k: never evicted */
        } else {
            /* d(k) is non-decreasing and reaches `others` once every n_j >= 1.
             * "d(K) = S" is read as equality up to rounding: d >= S (1 - 1e-9).
             * K is capped at 64 / f_i, where 1 - (1 - f_i)^K differs from 1 by
             * less than e^-64. */
            const double target = (double)S * (1.0 - 1e-9);
            const double kmax = ceil(64.0 / f[i]) + (double)S;
            double lo = (double)S, hi = (double)S;
            while (hi < kmax && orc_cache_d(f, L, i, hi, others) < target) {
                hi = hi * 2.0 + 1.0 / f_pos_min;
                if (hi > kmax)
                    hi = kmax;
            }
            if (orc_cache_d(f, L, i, hi, others) < target) {
                c = 1.0; /* d never reaches S before the cap */
            } else {
                while (hi - lo >= 1.0) { /* integer binary search for the smallest k with d(k) >= S */
                    double mid = lo + floor((hi - lo) / 2.0);
                    if (orc_cache_d(f, L, i, mid, others) >= target)
                        hi = mid;
                    else
                        lo = mid + 1.0;
                }
                double K = lo;
                c = 1.0 - pow(1.0 - f[i], K);
            }
        }
        if (cdf)
            cdf[i] = c;
        h += f[i] * c;
    }
    *hit = h;
    return ORC_OK;
}

/* Threshold t of Section IV-B from the Section III-C model: lines are given
 * in transformed-id order, each holding rows_per_line ids; ids below t are the
 * ones expected to hit the cache, read as: t covers the leading lines whose
 * modelled hit probability cdf_j is at least p. */
int orc_cache_threshold(const double *f, int64_t L, int64_t S, double p, int32_t rows_per_line, int64_t *t)
{
    if (!t || rows_per_line < 1 || !(p > 0.0 && p <= 1.0) || L < 1)
        return ORC_EINVAL;
    double *cdf = (double *)malloc(sizeof(double) * (size_t)L);
    if (!cdf)
        return ORC_EINVAL;
    double hit;
    int st = orc_cache_hit_rate(f, L, S, &hit, cdf);
    if (st) {
        free(cdf);
        return st;
    }
    int64_t j = 0;
    while (j < L && cdf[j] >= p)
        j++;
    free(cdf);
    *t = j * (int64_t)rows_per_line;
    return ORC_OK;
}

/* Section III-C: a power-law frequency distribution is a straight line in a
 * log-log plot; fit it by ordinary least squares, log y = a + b log x, over
 * the points with x > 0 and y > 0:
 *   b = (m Sum uv - Sum u Sum v) / (m Sum u^2 - (Sum u)^2),  a = (Sum v - b Sum u) / m
 * with u = log x, v = log y and m usable points. */
int orc_powerlaw_fit(const double *x, const double *y, int64_t n, double *slope, double *intercept)
{
    if (!x || !y || n < 0 || !slope || !intercept)
        return ORC_EINVAL;
    long double su = 0, sv = 0, suu = 0, suv = 0;
    int64_t m = 0;
    for (int64_t k = 0; k < n; k++) {
        if (!(x[k] > 0.0) || !(y[k] > 0.0))
            continue;
        long double u = logl((long double)x[k]), v = logl((long double)y[k]);
        su += u;
        sv += v;
        suu += u * u;
        suv += u * v;
        m++;
    }
    if (m < 2)
        return ORC_EINVAL;
    long double den = (long double)m * suu - su * su;
    if (!(den > 0))
        return ORC_EINVAL;
    long double b = ((long double)m * suv - su * sv) / den;
    *slope = (double)b;
    *intercept = (double)((sv - b * su) / (long double)m);
    return ORC_OK;
}

/* Q1 materialisation (Sections I and IV-A): the attribute col of the
 * dimension row each fact row references, out[i] = rows[fk[i]][col]. */
int orc_materialize(const int32_t *rows, int32_t N, int32_t row_words, int32_t col, const int32_t *fk, int64_t F,
                    int32_t *out)
{
    if (!rows || N < 1 || row_words < 1 || col < 0 || col >= row_words || F < 0 || (F > 0 && (!fk || !out)))
        return ORC_EINVAL;
    for (int64_t i = 0; i < F; i++) {
        int32_t v = fk[i];
        if (v < 0 || v >= N)
            return ORC_EKEY;
        out[i] = rows[(int64_t)v * row_words + col];
    }
    return ORC_OK;
}
