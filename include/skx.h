/*
 * skx.h -- C ABI of the GB300 permutation-index library (libskx.so).
 *
 * The permutation index of Zhang & Ross, "Exploiting Data Skew for Improved
 * Query Performance" (ICDE 2020, arXiv 1910.10063): count how often each
 * foreign key occurs in a fact column, order the dimension rows by that
 * popularity, and relabel both sides with the resulting permutation so that
 * popular rows sit together at the front of the dimension table.  Queries
 * that join through the FK then touch a small, contiguous hot prefix.
 *
 * Conventions (all entry points):
 *   - Data pointers named d_* are DEVICE pointers (cudaMalloc / torch CUDA
 *     tensors) owned by the caller, on the current CUDA device.  h_* are
 *     host pointers (pinned memory gives the fastest copies).
 *   - Columns are dense little-endian int32 arrays; a foreign key is a
 *     0-based row offset into the dimension table (Section II-B).
 *   - Dimension tables are row-major records of `row_bytes` bytes
 *     (a multiple of 4); column c of a row is the int32 at byte offset 4*c.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it; the call returns once
 *     the work is enqueued.
 *   - Argument errors are returned synchronously and enqueue nothing.
 *     Errors found in the data by the kernels (a foreign key outside
 *     [0, N), a group key outside [0, G)) never fault: the offending row is
 *     skipped and a per-device error word is set; skx_stream_status()
 *     reports and clears it.
 *   - Every output buffer is fully overwritten.
 *   - Sizes: F (fact rows) up to 2^32 - 1, N (dimension rows) up to 2^31 - 1.
 */
#ifndef SKX_H
#define SKX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SKX_VERSION_MAJOR 1
#define SKX_VERSION_MINOR 0

typedef enum skx_status {
    SKX_OK = 0,
    SKX_EINVAL = 1,      /* bad argument: null pointer, negative or too large size, bad column */
    SKX_ENOMEM = 2,      /* a device or pinned-host allocation failed */
    SKX_EKEYRANGE = 3,   /* the data held a foreign key outside [0, N) */
    SKX_EGROUPRANGE = 4, /* the data held a group key outside [0, G) */
    SKX_ECUDA = 5,       /* a CUDA runtime call failed (see skx_last_cuda_error) */
    SKX_ETIMEOUT = 6,    /* a bounded device-side wait expired */
    SKX_EBUSY = 7,       /* no free slot / resource (serving admission) */
    SKX_ENOTSUP = 8      /* valid request the library does not support */
} skx_status;

/* Human-readable name of a status code (static string, never NULL). */
const char *skx_strerror(skx_status s);

/* Message of the last CUDA error seen by this library in this thread. */
const char *skx_last_cuda_error(void);

/* Library version as (major << 16) | minor. */
int32_t skx_version(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (all devices, all streams); a diagnostic for counting launches per call. */
uint64_t skx_kernel_launches(void);

/*
 * Synchronises `stream`, then reports and clears the per-device data-error
 * word of the current device: SKX_EKEYRANGE or SKX_EGROUPRANGE if any kernel
 * of this library on this device met such data since the last call (from any
 * stream), SKX_ETIMEOUT if a bounded device-side wait expired, SKX_EINVAL if
 * a frequency sort met counts whose sum exceeds the F it was given,
 * SKX_ECUDA if the stream itself failed, else SKX_OK.  The word is a fixed
 * variable of the library's device image (no allocation).
 */
skx_status skx_stream_status(void *stream);

/* ------------------------------------------------------------------------
 * Index build (Section III and III-A).
 *
 * The index is the popularity order of the dimension ids: a count of each
 * value of the fact column C (the Q3 aggregation), then the ids sorted by
 * decreasing count.  It is held in both representations of Section III:
 *   perm[r]  offset representation, new -> old: the id of rank r;
 *   rank[v]  rank representation,  old -> new: the rank of id v;
 * so rank[perm[r]] == r.  Ties are broken by ascending id and ids that never
 * occur follow all others (ascending), so perm is a bijection on [0, N)
 * and is unique for given data.  counts[v] (uint32) is kept as well.
 * ------------------------------------------------------------------------ */
typedef struct skx_index skx_index; /* opaque; owns device memory until destroyed */

/*
 * Builds the index of the FK column d_fk[F] over dimension ids [0, N).
 * Allocates the index's arrays (3 * 4 * N bytes) and temporary scratch with
 * stream-ordered allocation on `stream`; *out receives the handle
 * immediately, its arrays become valid in stream order.  Keys outside
 * [0, N) are not counted and raise SKX_EKEYRANGE at skx_stream_status.
 * Errors: SKX_EINVAL (null d_fk with F > 0, N < 1, F >= 2^32, null out),
 * SKX_ENOMEM, SKX_ECUDA.
 */
skx_status skx_build_index(const int32_t *d_fk, int64_t F, int32_t N, void *stream,
                           skx_index **out);

/*
 * The two halves of skx_build_index, for callers that want the Q3 count on its
 * own (Section I, query Q3; Section III-A, first step).
 * skx_count: d_counts[v] = #{i : d_fk[i] == v} for v in [0, N) (uint32,
 * fully overwritten; keys outside [0, N) are skipped and raise SKX_EKEYRANGE).
 * skx_build_index_from_counts: sorts the ids by (count desc, id asc) and
 * returns an index that takes a copy of the counts.  F bounds the sum of the
 * counts (the fact rows they were taken from; it sets how many key bits are
 * sorted); counts that break the bound give SKX_EINVAL at skx_stream_status.
 */
skx_status skx_count(const int32_t *d_fk, int64_t F, int32_t N, uint32_t *d_counts, void *stream);
skx_status skx_build_index_from_counts(const uint32_t *d_counts, int32_t N, int64_t F, void *stream,
                                       skx_index **out);

/*
 * The count of skx_count with the algorithm chosen by the caller (both give
 * identical counts; the choice only moves time between kernels):
 *   SKX_COUNT_AUTO         what skx_count and skx_build_index use.  For
 *                          2^16 <= N <= 2^28 and F >= 2^26 (when the
 *                          partitioned count's scratch can be allocated) a
 *                          kernel samples 8192 keys of d_fk and picks on the
 *                          device, without a host synchronisation: the single
 *                          pass when 85 % or more of the sampled keys repeat
 *                          in the sample (heavy skew), the partitioned count
 *                          when fewer than 60 % do, and in between the
 *                          partitioned count from N >= 2^24 ids (above 2^25
 *                          ids only while fewer than 70 % repeat).  Smaller
 *                          inputs take the single pass;
 *   SKX_COUNT_SINGLE_PASS  one pass over d_fk, a per-CTA shared-memory cache
 *                          of hot ids and L2 atomics for the rest;
 *   SKX_COUNT_PARTITIONED  radix partition of the keys by 2^15-id buckets
 *                          (2 bytes per key of scratch written and read back)
 *                          and a shared-memory count per bucket; no random
 *                          global access.  Up to 2^25 ids (1024 buckets) and
 *                          for 65536 <= F < 2^32 / 3 the bucket regions are
 *                          sized from a sample of 65536 keys and d_fk is read
 *                          once; otherwise, or when a bucket outgrows its
 *                          sampled region, an exact pre-count pass sizes them
 *                          (d_fk read twice).  Needs N <= 2^28; allocates
 *                          4 * F bytes of stream-ordered scratch with sampled
 *                          regions, 2 * F bytes otherwise (plus a few MB).
 * Errors: as skx_count; SKX_EINVAL for an unknown method; SKX_ENOTSUP when
 * SKX_COUNT_PARTITIONED is asked for with N > 2^28.
 */
typedef enum {
    SKX_COUNT_AUTO = 0,
    SKX_COUNT_SINGLE_PASS = 1,
    SKX_COUNT_PARTITIONED = 2
} skx_count_method;
skx_status skx_count_ex(const int32_t *d_fk, int64_t F, int32_t N, uint32_t *d_counts, int32_t method,
                        void *stream);

/*
 * Allocation-free variant of the frequency sort, for callers that must not
 * allocate device memory when they build the order -- for example because a
 * framework's caching allocator already holds almost all of HBM, because an
 * allocation (which can synchronise the device or fail under memory
 * pressure) is not acceptable in a latency-critical loop, or because the
 * caller is a plug-in that is handed its buffers and may not call the CUDA
 * allocator.  The paper has no counterpart; this is a property of this
 * library's interface only.
 *
 * Same result as skx_build_index_from_counts: d_perm[r] (new -> old) and
 * d_rank[v] (old -> new), int32[N] in caller-owned device buffers, from
 * d_counts (uint32[N]); F bounds the sum of the counts (counts that break
 * the bound -- one above F, or more ids with a count of 255 or more than
 * F / 255 allows -- are reported as SKX_EINVAL by skx_stream_status, and the
 * order is then incomplete).  The scratch space is a
 * fixed ~16 MiB array inside the library's device image, so N is limited to
 * skx_sort_by_count_noalloc_max_n() = 2^20 ids; a larger N is rejected
 * with SKX_EINVAL before anything is enqueued.
 *
 * When the array is reserved: CUDA loads a library's device code lazily
 * (unless CUDA_MODULE_LOADING=EAGER, which reserves the array when the
 * library is loaded), so a device reserves the ~16 MiB the first time this
 * function runs on it, and keeps it until the process exits.  A caller whose
 * memory will later be tight should make that first call early: a call with
 * N = 0 (the pointers may be NULL) does only this set-up and enqueues
 * nothing.  Make it before any stream capture too.  Every later call looks
 * up the array's device address again (no allocation; a cached address would
 * go stale after cudaDeviceReset).  All calls share the one array: calls
 * whose work overlaps on the GPU (different streams, or different threads)
 * race and must be serialised by the caller.
 */
skx_status skx_sort_by_count_noalloc(const uint32_t *d_counts, int32_t N, int64_t F, int32_t *d_perm,
                                     int32_t *d_rank, void *stream);
int32_t skx_sort_by_count_noalloc_max_n(void);

/* Borrowed device pointers into the index (valid until skx_index_destroy). */
skx_status skx_index_perm(const skx_index *idx, const int32_t **d_perm);     /* new -> old, int32[N] */
skx_status skx_index_rank(const skx_index *idx, const int32_t **d_rank);     /* old -> new, int32[N] */
skx_status skx_index_counts(const skx_index *idx, const uint32_t **d_counts); /* uint32[N] */
int32_t skx_index_size(const skx_index *idx);                                /* N, or -1 */

/*
 * Index maintenance (Section III-A): n_new dimension rows appended to the
 * table get the ids N .. N+n_new-1 and join the index at its end as the new
 * least frequent items (count 0); existing ranks do not change, so remapped
 * fact columns stay valid.  Reallocates the index arrays in stream order on
 * `stream` (borrowed pointers from skx_index_perm/rank/counts become invalid).
 * Fact inserts and deletes are not tracked: results stay exact with a stale
 * index, only the layout's benefit fades until skx_build_index is run again.
 */
skx_status skx_index_append(skx_index *idx, int32_t n_new, void *stream);

/*
 * Staleness of an index and the rebuild decision (Section III-A: the index
 * tolerates changes to the fact column -- results stay exact -- and only
 * its benefit fades; when to rebuild is a decision made from the data).
 * The decision looks where the benefit lives: the likely-hit region of
 * ranks [0, t) (Section IV-B; for example t from skx_split_threshold).
 *   share_stale  the share of the sampled fact keys whose rank under the
 *                current index is below t (accesses the layout keeps hot);
 *   share_fresh  the share held by the sample's own t most frequent ids
 *                (what a rebuilt index would put below t);
 *   loss         share_fresh - share_stale: accesses a rebuild would move
 *                into the hot region;
 *   rebuild      1 when loss > max_loss.
 * skx_index_drift takes a device sample of the current fact column in
 * ORIGINAL ids (d_fk_sample[n]), recodes it through the index and counts it
 * by rank on `stream` (stream-ordered scratch of 4 (n + N) bytes), copies the
 * N counts to the host and synchronises `stream`.  Sample keys outside
 * [0, N) are left out (and reported by skx_stream_status as SKX_EKEYRANGE).
 * skx_drift_from_counts is its host half, from h_counts_by_rank[N].
 * Errors: SKX_EINVAL (null pointer, n < 1, t < 1, t > N, max_loss < 0, an
 * empty sample), SKX_ENOMEM, SKX_ECUDA.
 */
typedef struct skx_drift {
    int64_t sample;      /* sampled keys counted (in [0, N)) */
    int64_t t;           /* the hot region [0, t) the shares refer to */
    double share_stale;
    double share_fresh;
    double loss;
    int32_t rebuild;
    int32_t reserved;
} skx_drift;
skx_status skx_index_drift(const skx_index *idx, const int32_t *d_fk_sample, int64_t n, int64_t t, double max_loss,
                           skx_drift *out, void *stream);
skx_status skx_drift_from_counts(const uint32_t *h_counts_by_rank, int32_t N, int64_t t, double max_loss,
                                 skx_drift *out);

/* Frees the index (stream-ordered on the stream it was built on). NULL is a no-op. */
void skx_index_destroy(skx_index *idx);

/* ------------------------------------------------------------------------
 * Recode of the fact column (Section III-A): d_fk_out[i] = rank[d_fk_in[i]].
 * d_fk_out may equal d_fk_in (in place); other overlaps are not allowed.
 * Keys outside [0, N) are copied through unchanged and raise SKX_EKEYRANGE.
 * ------------------------------------------------------------------------ */
skx_status skx_remap(const skx_index *idx, const int32_t *d_fk_in, int32_t *d_fk_out, int64_t F,
                     void *stream);

/* ------------------------------------------------------------------------
 * Materialisation, query Q1 (Sections I and IV-A): d_out[i] = column col
 * (int32) of row d_fk[i] of d_rows (N rows of row_bytes bytes, row-major,
 * 4-byte aligned, row_bytes a multiple of 4), for i < F, int32.  Works on
 * either layout: (plain rows, original keys) or (reordered rows, recoded
 * keys) give the same d_out.  Keys outside [0, N) give 0 and raise
 * SKX_EKEYRANGE at skx_stream_status.  d_out must not overlap the inputs.
 * Errors: SKX_EINVAL (null pointer with F > 0, N < 1, bad row_bytes, col
 * outside the row, F >= 2^32, misaligned pointers), SKX_ENOMEM, SKX_ECUDA.
 * ------------------------------------------------------------------------ */
skx_status skx_materialize(const void *d_rows, int32_t N, int32_t row_bytes, int32_t col, const int32_t *d_fk,
                           int64_t F, int32_t *d_out, void *stream);

/* ------------------------------------------------------------------------
 * Permuted copy of the dimension table (Section III-B):
 * row r of d_rows_out = row perm[r] of d_rows_in, row_bytes bytes each
 * (a multiple of 4).  Input and output must not overlap.
 * ------------------------------------------------------------------------ */
skx_status skx_reorder(const skx_index *idx, const void *d_rows_in, void *d_rows_out, int32_t N,
                       int32_t row_bytes, void *stream);

/* ------------------------------------------------------------------------
 * FK-join probe + filter + aggregation (Sections I and IV: the Q1 gather
 * through the FK, the Q2 filter on a dimension attribute, and aggregation;
 * Section IV-B threshold processing for the hot prefix).
 *
 *   COUNT        out[0] = #{i : row(fk[i]).filter_col < filter_lt}
 *   SUM          out[0] = sum of measure[i] * row(fk[i]).payload_col over those i
 *   GROUPBY_SUM  out[g] = the same sum restricted to row(fk[i]).group_col == g,
 *                for g in [0, num_groups)
 *
 * Products are formed in int64 and sums wrap modulo 2^64 (bit-exact, order
 * free).  filter_col = -1 disables the filter; payload_col = -1 uses payload
 * 1 (SUM(measure)).  d_measure may be NULL for COUNT.
 *
 * The call is layout agnostic: on (plain rows, original keys) and on
 * (skx_reorder'ed rows, skx_remap'ped keys) it returns identical results.
 *
 * One exception to the data-error reporting: a row of the hot prefix (keys
 * below hot_keys) is looked up once per CTA with the sum of its measures, and
 * not at all when that sum is 0 modulo 2^64 -- so a group key outside
 * [0, G) on such a row can go unreported.  The result is exact either way
 * (the row contributes 0).
 * With a remapped layout, rows [0, hot_keys) -- the most popular -- are
 * aggregated per key in shared memory without touching the dimension table
 * until the end of each CTA (threshold-based processing of Section IV-B).
 * ------------------------------------------------------------------------ */
typedef enum skx_agg { SKX_AGG_COUNT = 0, SKX_AGG_SUM = 1, SKX_AGG_GROUPBY_SUM = 2 } skx_agg;

typedef struct skx_query {
    int32_t agg;         /* skx_agg */
    int32_t filter_col;  /* column tested with "< filter_lt", or -1 for no filter */
    int32_t filter_lt;
    int32_t group_col;   /* GROUPBY_SUM only */
    int32_t num_groups;  /* G, GROUPBY_SUM only, 1 .. 2^24 */
    int32_t payload_col; /* column multiplied with the measure, or -1 for 1 */
} skx_query;

/* ------------------------------------------------------------------------
 * Query preprocessing copies (Section III-B: a query may work on its own
 * copy of just the dimension columns it needs, laid out in the index's order).
 * idx may be NULL for the identity order (the same narrow copy of the plain
 * layout, so that both layouts can be compared on equal terms).
 *
 * skx_reorder_columns: row r of d_out is the int32 columns h_cols[0..ncols)
 *   (a host array, 1 <= ncols <= 16, each < row_bytes/4) of source row
 *   perm[r] (or r); d_out rows are 4*ncols bytes.
 * skx_reorder_query: the query's predicate is evaluated once per dimension
 *   row (as for the Q2 bitmap, Section I) and folded into an 8-byte row
 *   {key, payload}: key = the group (GROUPBY_SUM) or 0 (COUNT, SUM) when the
 *   row passes the filter and the sentinel num_groups (or 1) when it does
 *   not; payload = payload_col (1 for payload_col = -1 or COUNT).  Running
 *   skx_query_prefiltered(q) over that table gives the result of q.  Every
 *   row that passes the filter with a group outside [0, num_groups) raises
 *   SKX_EGROUPRANGE (through skx_stream_status) here, referenced by a fact
 *   row or not: the prefiltered probe could not tell a group >= num_groups
 *   from the sentinel.
 * Input and output must not overlap.
 * ------------------------------------------------------------------------ */
skx_status skx_reorder_columns(const skx_index *idx, const void *d_rows_in, int32_t N, int32_t row_bytes,
                               const int32_t *h_cols, int32_t ncols, void *d_out, void *stream);
skx_status skx_reorder_query(const skx_index *idx, const void *d_rows_in, int32_t N, int32_t row_bytes,
                             const skx_query *q, void *d_out, void *stream);
/* The query to run over a skx_reorder_query table: filter "key < G", group key
 * (column 0), payload (column 1). */
skx_query skx_query_prefiltered(const skx_query *q);


/* Launch and threshold parameters; zero-initialise and set what you need.
 * A field left at 0 takes the library default (chosen from N, F, the query
 * and the device).  Resolved values never contain 0: "off" and "as many as
 * fit" are -1. */
typedef struct skx_tuning {
    int32_t block_threads; /* 128, 256 or 512 (default 512) */
    int32_t ctas_per_sm;   /* resident CTAs per SM of the persistent grid; default 1024 threads
                              per SM; -1 = as many as fit */
    int32_t hot_keys;      /* t: keys [0, t) aggregated per key in shared memory (default: as
                              many as fit with two CTAs per SM); -1 = off (plain processing) */
    int32_t lane_keys;     /* keys [0, t_lane), t_lane <= t, get one copy per warp lane
                              (default 32); -1 = off */
    int32_t warp_aggregate;/* reserved, keep 0 */
    int32_t unroll;        /* 16-byte fact vectors per thread per step: 1 (default), 2 or 4 */
    int32_t gather_policy; /* L2 eviction priority of the dimension gathers: 1 evict_last,
                              2 evict_normal, 3 evict_first, 4 evict_unchanged (default 2) */
    int32_t split_keys;    /* t of the split (Section IV-B, remapped layout): fact rows with key
                              >= t (the likely misses) are deferred to a second pass that
                              resolves them bucket by bucket in rank order; keys in
                              [hot_keys, t) are gathered at once.  Default (0) and -1: off.
                              skx_split_threshold derives t from the index with the cache model.
                              Needs t > hot_keys and fk, measure at the same offset mod 16 bytes
                              (otherwise the probe runs unsplit); uses stream-ordered scratch of
                              about 4 F bytes (deferred rows beyond F/2 are resolved at once). */
    int32_t split_bucket;  /* log2 of the ranks per bucket of the second pass (default 19, range
                              12..26; raised until there are at most 512 buckets) */
    int32_t reserved[7];
} skx_tuning;

skx_status skx_probe_aggregate(const void *d_rows, int32_t N, int32_t row_bytes, const int32_t *d_fk,
                               const int32_t *d_measure, int64_t F, const skx_query *q, int64_t *d_out,
                               const skx_tuning *tuning /* NULL = defaults */, void *stream);

/*
 * The query copy packed in 32 bits per row (Section III-B's copy of the needed
 * columns, made as small as the query allows: a row costs 4 bytes of cache
 * instead of 8, so twice as many rows share a line and the table takes half
 * the L2).  skx_reorder_query_packed writes the 8-byte copy of
 * skx_reorder_query to d_out8 (N x 8 bytes) and, in the same pass, d_out4
 * (N x 4 bytes, 4-byte aligned, overlapping neither d_out8 nor the input):
 *   d_out4[r] = key << (32 - b) | (payload & (2^(32-b) - 1)),
 * key = the row's group (GROUP BY; 0 for SUM and COUNT), or G for a row that
 * fails the filter (G = num_groups for GROUP BY, else 1), payload as a
 * (32 - b)-bit two's complement number (0 for a row that fails the filter:
 * it is never used), and b = skx_query_packed_key_bits(q),
 * the smallest b with 2^b >= G + 2.  A row whose key lies outside [0, G] or
 * whose payload needs more bits is written with the escape code: the key field
 * all ones; its values are read from the 8-byte copy when probed.  Errors: as
 * skx_reorder_query, and SKX_EINVAL for a null or misaligned d_out4 or
 * overlapping buffers.
 *
 * skx_probe_packed joins d_fk / d_measure (keys of the same order as the copy:
 * d_fk' for a permuted copy) against both tables and gives the result of q
 * (the original query) in d_out, as skx_probe_aggregate over the 8-byte copy
 * with skx_query_prefiltered(q) would, exactly.  tuning: only block_threads
 * and ctas_per_sm are used (NULL: 512 threads, as many CTAs as fit).  Errors:
 * SKX_EINVAL (bad agg or num_groups, null or misaligned pointer, N < 1,
 * F >= 2^32); data errors (a key outside [0, N), a group outside [0, G)) as
 * skx_probe_aggregate, through skx_stream_status.
 */
skx_status skx_reorder_query_packed(const skx_index *idx, const void *d_rows_in, int32_t N, int32_t row_bytes,
                                    const skx_query *q, void *d_out8, uint32_t *d_out4, void *stream);
int32_t skx_query_packed_key_bits(const skx_query *q); /* b above, or -1 for a bad query */
skx_status skx_probe_packed(const uint32_t *d_rows4, const void *d_rows8, int32_t N, const int32_t *d_fk,
                            const int32_t *d_measure, int64_t F, const skx_query *q, int64_t *d_out,
                            const skx_tuning *tuning, void *stream);

/* The tuning skx_probe_aggregate would use for these arguments when given
 * tuning = NULL (the autotuner's cached choice for this shape if there is
 * one, else the defaults), written to *out. */
skx_status skx_probe_default_tuning(int32_t N, int32_t row_bytes, int64_t F, const skx_query *q,
                                    int remapped, skx_tuning *out);

/* The tuning skx_probe_aggregate resolves *in to for these arguments (every
 * default filled in; a split threshold outside (hot_keys, N) turned off; the
 * split's bucket size raised until there are at most 512 buckets), written to
 * *out.  Host only: it launches nothing. */
skx_status skx_probe_resolve_tuning(int32_t N, int32_t row_bytes, int64_t F, const skx_query *q,
                                    const skx_tuning *in, skx_tuning *out);

/*
 * Autotuner for the probe (threshold-based processing, Section IV-B, picks t
 * by measurement): runs skx_probe_aggregate with each candidate launch shape
 * and hot-prefix size on the first min(F, 2^26) rows of the given data,
 * synchronously on `stream`, and returns the fastest in *out (and its time
 * scaled to F in *best_ms if not NULL).  remapped = 0 restricts the search to
 * plain processing (no hot prefix).  d_out (num_groups or 1 int64) is used as
 * scratch.  The choice is cached per (device, N, row_bytes, agg, log2 F,
 * remapped); skx_probe_aggregate with tuning = NULL uses the remapped entry
 * of its shape when present.
 */
skx_status skx_probe_autotune(const void *d_rows, int32_t N, int32_t row_bytes, const int32_t *d_fk,
                              const int32_t *d_measure, int64_t F, const skx_query *q, int remapped,
                              int64_t *d_out, void *stream, skx_tuning *out, float *best_ms);
/* The same search, plus the split probe when remapped != 0 and hint is not
 * NULL with hint->split_keys = t_model > 0 (for example from
 * skx_split_threshold): split thresholds t_model / 2, t_model and 2 t_model,
 * each with hot_keys in {off, 2048, 8192} and one or as many CTAs per SM as
 * fit.  Other fields of hint are ignored.  Because the split pays through
 * cold rows the whole column references several times, the split candidates
 * and the best unsplit shape are then timed again on the first min(F, 2^28)
 * rows.  skx_probe_autotune is this call with hint = NULL. */
skx_status skx_probe_autotune_ex(const void *d_rows, int32_t N, int32_t row_bytes, const int32_t *d_fk,
                                 const int32_t *d_measure, int64_t F, const skx_query *q, int remapped,
                                 const skx_tuning *hint, int64_t *d_out, void *stream, skx_tuning *out,
                                 float *best_ms);

/* ------------------------------------------------------------------------
 * The paper's other operators over the remapped layout.
 * ------------------------------------------------------------------------ */

/* Heavy hitters (query Q3a, Sections I and IV-B): with an up-to-date index the
 * k most frequent values are the transformed ids 0..k-1, so d_out[r] (int64,
 * k entries, fully overwritten) = #{i : d_fk[i] == r} for r < k and keys
 * >= k are skipped.  The ids are perm[0..k).  Counters stay in shared memory
 * for k up to about 55K. */
skx_status skx_topk_counts(const int32_t *d_fk, int64_t F, int32_t k, int64_t *d_out, void *stream);

/* Selection bitmap (query Q2 preprocessing, Section I): bit r of d_bits
 * (uint32 words, ceil(N/32) of them) = row r's column filter_col < filter_lt. */
skx_status skx_select_bitmap(const void *d_rows, int32_t N, int32_t row_bytes, int32_t filter_col, int32_t filter_lt,
                             uint32_t *d_bits, void *stream);

/* Selection (query Q2, Sections I and IV-A): writes the offsets i of the fact
 * rows with bit d_fk[i] set, in increasing order, to d_offsets (uint32, room
 * for F) and their number to *d_count (device int64).  Keys outside [0, N)
 * are not selected and raise SKX_EKEYRANGE at skx_stream_status.  Uses
 * stream-ordered scratch of about F/2048 bytes. */
skx_status skx_select(const uint32_t *d_bits, int32_t N, const int32_t *d_fk, int64_t F, uint32_t *d_offsets,
                      int64_t *d_count, void *stream);

/* Cache model (Section III-C), host only: estimated LRU hit rate of a cache of
 * S lines for L lines with access frequencies h_f (host, sum 1). */
skx_status skx_cache_hit_rate(const double *h_f, int64_t L, int64_t S, double *hit);

/* The same model's hit probability of each line, cdf_i = 1 - (1 - f_i)^K_i
 * (Section III-C), written to h_cdf[L] (host) in the order of h_f; 0 for lines
 * with f_i = 0.  Errors: SKX_EINVAL (null pointer, L < 1, S < 1, a negative
 * or NaN frequency). */
skx_status skx_cache_line_cdf(const double *h_f, int64_t L, int64_t S, double *h_cdf);

/* The threshold t of Section IV-B derived from the Section III-C model: ids
 * below t are likely cache hits.  h_f lists the lines in transformed-id order
 * (line j holds ids [j * rows_per_line, (j + 1) * rows_per_line), as in the
 * remapped layout); *t = rows_per_line x the number of leading lines whose
 * modelled hit probability is at least p (0 < p <= 1).  Host only.
 * Errors: as skx_cache_line_cdf; SKX_EINVAL for p outside (0, 1],
 * rows_per_line < 1 or a null t. */
skx_status skx_cache_threshold(const double *h_f, int64_t L, int64_t S, double p, int32_t rows_per_line,
                               int64_t *t);

/* Power-law fit of a value-frequency distribution (Section III-C: sample the
 * data and fit it to a known distribution; a power law is a line in a
 * log-log plot): the least-squares line log y = intercept + slope * log x
 * through the points (h_x[k], h_y[k]) with x > 0 and y > 0 (others are
 * skipped).  Host only.  Errors: SKX_EINVAL (null pointer, fewer than two
 * usable points, all usable x equal). */
skx_status skx_powerlaw_fit(const double *h_x, const double *h_y, int64_t n, double *slope, double *intercept);

/* The threshold t of the split probe (skx_tuning.split_keys; Section IV-B)
 * derived from an index with the Section III-C model, as the paper suggests:
 * the index's counts at 48 log-spaced ranks (gathered on the device; `stream`
 * is synchronised) are fitted to a power law (skx_powerlaw_fit), the fitted
 * frequencies are summed over the 128-byte lines of a remapped table with
 * rows of row_bytes, and *t = skx_cache_threshold(those lines, S =
 * cache_bytes / 128, p, rows per line), capped at N.  cache_bytes = 0 takes
 * two thirds of the device's L2 (the share the probe's dimension lines were
 * measured to keep while the fact columns stream past).  Host work is
 * O(N log N) (about a second at N = 20M).  Errors: SKX_EINVAL (null pointer,
 * N < 2, bad row_bytes, p outside (0, 1], negative cache_bytes, fewer than
 * two nonzero counts), SKX_ENOMEM, SKX_ECUDA. */
skx_status skx_split_threshold(const skx_index *idx, int32_t row_bytes, int64_t cache_bytes, double p, int64_t *t,
                               void *stream);
/* The host half of skx_split_threshold for a fitted exponent (log count =
 * intercept + slope * log(rank + 1)): frequencies proportional to
 * (r + 1)^slope for r < N, summed per 128-byte line of rows of row_bytes,
 * and t from skx_cache_threshold over cache_bytes / 128 lines, capped at N.
 * Host only.  Errors: SKX_EINVAL (null t, N < 1, bad row_bytes, cache_bytes
 * below one line, p outside (0, 1], a slope that is not finite). */
skx_status skx_split_threshold_from_fit(double slope, int32_t N, int32_t row_bytes, int64_t cache_bytes, double p,
                                        int64_t *t);

/* Counts of chosen ranks of an index, the input of a frequency fit:
 * h_counts[k] = counts[perm[h_ranks[k]]] (the count of the id with
 * transformed id h_ranks[k]), for n host-side ranks in [0, N).  Gathers on
 * the device on `stream` and synchronises it.  Errors: SKX_EINVAL (null
 * index or buffer, a rank outside [0, N)), SKX_ENOMEM, SKX_ECUDA. */
skx_status skx_index_counts_at_ranks(const skx_index *idx, const int64_t *h_ranks, int64_t n, uint32_t *h_counts,
                                     void *stream);

/* ------------------------------------------------------------------------
 * Batched probes (many queries, one persistent launch).  Each descriptor is
 * one skx_probe_aggregate call against the same dimension table: remapped
 * keys fk[F] and measures (device), the query, and a device output of
 * num_groups (GROUPBY_SUM, at most 4096 in a batch) or 1 int64.  The fact
 * rows of all queries are cut into tiles that a persistent grid pulls from
 * one atomic counter, so uneven batch sizes balance across the SMs; a small
 * prologue kernel clears every output first.  Results equal the single-call
 * results bit for bit.  The paper processes one query at a time; batching is
 * this library's systems extension of the same operator (Sections IV-A, IV-B).
 * ------------------------------------------------------------------------ */
typedef struct skx_probe_desc {
    const int32_t *fk;      /* device, F keys (remapped layout: frequency ranks) */
    const int32_t *measure; /* device, F measures; may be NULL for COUNT */
    int64_t F;
    skx_query q;
    int64_t *out;           /* device, num_groups or 1 entries, fully overwritten */
} skx_probe_desc;

typedef struct skx_batch_plan skx_batch_plan; /* opaque: descriptors and tile table on the device */

/* Uploads the n descriptors (copied; the host array may be reused after the
 * call) and builds the tile table (tile_rows fact rows per tile, 0 = 65536).
 * tuning as for skx_probe_aggregate (hot_keys 0 = 1024 here).  Synchronises
 * `stream` once.  Errors: SKX_EINVAL, SKX_ENOTSUP (more than 4096 groups),
 * SKX_ENOMEM, SKX_ECUDA. */
skx_status skx_batch_plan_create(const void *d_rows, int32_t N, int32_t row_bytes, const skx_probe_desc *h_descs,
                                 int32_t n, const skx_tuning *tuning, int32_t tile_rows, void *stream,
                                 skx_batch_plan **out);
/* Enqueues the batch on `stream` (2 kernels).  use_graph != 0: the two
 * launches are captured once into a CUDA graph (on first use) and the graph
 * is replayed on `stream`. */
skx_status skx_batch_plan_launch(skx_batch_plan *plan, int use_graph, void *stream);
/* Times candidate tile sizes, launch shapes and hot-prefix sizes on the
 * plan's own data (synchronously, outputs used as scratch) and keeps the
 * fastest; returns it in *out, *tile_rows_out, *best_ms (each may be NULL). */
skx_status skx_batch_plan_autotune(skx_batch_plan *plan, void *stream, skx_tuning *out, int32_t *tile_rows_out,
                                   float *best_ms);
void skx_batch_plan_destroy(skx_batch_plan *plan);
/* One-shot: create, launch, synchronise, destroy. */
skx_status skx_probe_batch(const void *d_rows, int32_t N, int32_t row_bytes, const skx_probe_desc *h_descs,
                           int32_t n, const skx_tuning *tuning, void *stream);

/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching over a resident index.
 * The reordered dimension table (d_rows, skx_reorder output) and the index's
 * rank array (old -> new, skx_index_rank) stay resident on the device and
 * are borrowed for the server's lifetime.  Each request carries a fact batch
 * with ORIGINAL keys in host memory (pinned memory copies fastest); the
 * server copies it into a fixed device arena when an in-flight slot and
 * arena room are free (admission by memory, arrival order), recodes the keys
 * through the resident rank array (Section III-A), and runs the remaining
 * rows of all admitted requests together in rounds of the batched probe, so
 * requests arriving while others run join the next round and their copies
 * overlap the running rounds.  Results are bit-identical to
 * skx_probe_aggregate on the same data.  The paper has no serving layer;
 * this is this library's systems extension.
 * ------------------------------------------------------------------------ */
typedef struct skx_server skx_server;

typedef struct skx_server_config {
    int32_t max_inflight;   /* requests admitted at once (device slots); default 128 */
    int32_t tile_rows;      /* fact rows per batch tile; default 65536 */
    int64_t round_rows;     /* fact rows per device round, over all requests; default 64 Mi */
    int64_t memory_budget;  /* device arena for admitted requests, bytes; default min(free/2, 16 GiB) */
    int32_t timeout_ms;     /* bound on any internal wait for the device; default 10000 */
    int32_t cpu_affinity;   /* 0: run the server thread on the CPUs next to the device (read from
                               sysfs; left alone when they cannot be read); -1: leave it alone */
    skx_tuning tuning;      /* batch kernel tuning (hot_keys 0 = 1024) */
    int32_t reserved[8];
} skx_server_config;

typedef struct skx_request {
    const int32_t *h_fk;      /* host, F original keys in [0, N) */
    const int32_t *h_measure; /* host, F measures (ignored for COUNT) */
    int64_t F;
    skx_query q;              /* GROUPBY_SUM: at most 4096 groups */
    int64_t *h_out;           /* host, num_groups or 1 int64, written at completion */
} skx_request;

/* d_rank may be NULL when requests already carry remapped keys.  cfg may be
 * NULL for defaults.  Starts the server thread. */
skx_status skx_server_create(const void *d_rows, int32_t N, int32_t row_bytes, const int32_t *d_rank,
                             const skx_server_config *cfg, skx_server **out);
/* Queues a request (its host buffers must stay valid until it completes);
 * returns at once with a ticket.  SKX_ENOMEM if it can never fit the arena. */
skx_status skx_server_submit(skx_server *s, const skx_request *req, uint64_t *ticket);
/* Waits up to timeout_ms for the request: SKX_OK (h_out written), the
 * request's error, or SKX_ETIMEOUT. */
skx_status skx_server_wait(skx_server *s, uint64_t ticket, int32_t timeout_ms);
/* Host clock seconds (steady clock) of submit, admission and completion. */
skx_status skx_server_request_times(skx_server *s, uint64_t ticket, double *submit_s, double *admit_s,
                                    double *done_s);
/* Forgets a finished ticket (SKX_EBUSY while it runs). */
skx_status skx_server_release(skx_server *s, uint64_t ticket);
/* Open-loop load generator: submits reqs[i] at arrival_s[i] seconds after
 * the call starts (busy-waiting on the host clock), waits for all (bounded by
 * timeout_ms overall) and writes each request's latency from its scheduled
 * arrival to completion (-1 for a failed one) to latency_s[i]. */
skx_status skx_server_replay(skx_server *s, const skx_request *reqs, const double *arrival_s, int32_t n,
                             int32_t timeout_ms, double *latency_s);
skx_status skx_server_stats(skx_server *s, uint64_t *rounds, uint64_t *rows, uint64_t *max_active);
/* Finishes queued work, stops the thread and frees everything. */
void skx_server_destroy(skx_server *s);

/* ------------------------------------------------------------------------
 * Whole path from host memory (Sections III-A, III-B and IV in sequence):
 * copies h_fk[F], h_measure[F] and the dimension table h_rows[N * row_bytes]
 * to the device, builds the index, remaps the keys, builds the query's
 * permuted copy of the dimension rows (skx_reorder_query_packed: 32 bits
 * per row beside its 8-byte form, Section III-B), runs the query on it
 * (skx_probe_packed) and copies the result (num_groups or 1 int64) to h_out.
 * Device buffers (N * (row_bytes + 12) + 8 F bytes and the index) are
 * stream-ordered allocations on `stream`, released before return.  Synchronous: returns after h_out is
 * written, with any data error of this call already reported (SKX_EKEYRANGE,
 * SKX_EGROUPRANGE) rather than left for skx_stream_status.
 * ------------------------------------------------------------------------ */
skx_status skx_join_aggregate_host(const void *h_rows, int32_t N, int32_t row_bytes, const int32_t *h_fk,
                                   const int32_t *h_measure, int64_t F, const skx_query *q,
                                   int64_t *h_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SKX_H */
