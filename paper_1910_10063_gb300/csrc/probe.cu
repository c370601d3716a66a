// probe.cu -- FK-join probe + filter + aggregation over the (re)ordered
// layout: the Q1 gather of a dimension row through the FK used as an array
// offset, the Q2 predicate on one of its attributes, and a COUNT / SUM /
// GROUP BY SUM aggregation (Sections I and IV-A of the paper).
//
// GB300 design.
//  * Persistent grid (a multiple of the SM count); each thread streams the
//    fk and measure columns with 16-byte loads marked L2 evict-first and keeps
//    4 x UNROLL rows in flight, issuing all of their dimension gathers before
//    consuming any of them.  Gathers carry the L2 eviction priority chosen by
//    skx_tuning.gather_policy: evict-normal by default (evict-last for the hot
//    rows, or a split of the priority by rank, measured no faster while the
//    fact stream is marked evict-first).
//  * Threshold-based processing (Section IV-B): after remapping, a key k < t
//    is one of the t most popular rows.  Those rows are not gathered at all
//    while streaming: the CTA adds the row's measure (or 1 for COUNT) into a
//    per-key shared-memory sum, and at the end looks up each hot row once and
//    folds sum * payload into its group.  This is exact in modular integer
//    arithmetic: sum_i m_i * p == p * sum_i m_i (mod 2^64).
//  * The t_lane hottest keys get one shared-memory copy per warp lane, so
//    the lanes of a warp never collide on the same address -- the paper's
//    per-SIMD-lane copies of the top values (Section IV-B, aggregation).
//  * Group sums live in shared memory (two 32-bit words per group, low and
//    high, with exact carries: 32-bit shared atomics are native, 64-bit ones
//    are not) and are merged into the output with one global atomic per group
//    per CTA: the paper's hybrid of private buffers for hot data and shared
//    atomics (Section IV-C).
//    COUNT and SUM accumulate in registers and reduce once per CTA.
// With t = 0 the same kernel is the plain probe used on the original layout.
#include "probe_core.cuh"

namespace skx {
namespace {

using namespace pcore;

template <int AGG, int PATH, bool GSMEM, int UNROLL>
__global__ void __launch_bounds__(512) k_probe(PP p) {
    extern __shared__ unsigned long long smem[];
    const int ngrp = GSMEM ? p.G : 0;
    GrpRef g;
    g.lo = reinterpret_cast<uint32_t *>(smem);
    g.hi = g.lo + ngrp;
    HotArrays h;
    h.lo = reinterpret_cast<uint32_t *>(smem + ngrp);
    h.hi = reinterpret_cast<int32_t *>(h.lo + p.t_hot);
    h.lane_lo = reinterpret_cast<uint32_t *>(h.hi + p.t_hot);
    h.lane_hi = reinterpret_cast<int32_t *>(h.lane_lo + (p.t_lane << 5));
    const int nsm = ngrp + p.t_hot + (p.t_lane << 5);  // 8-byte words
    for (int i = threadIdx.x; i < nsm; i += blockDim.x) smem[i] = 0;
    __syncthreads();

    const uint64_t pol_s = policy_evict_first();
    const uint64_t pol_g = policy_by_code(p.gather_policy);
    const unsigned lane = lane_id();
    unsigned long long acc = 0;

    const int4 *fk4 = reinterpret_cast<const int4 *>(p.fk + p.head);
    const int4 *m4 = reinterpret_cast<const int4 *>((AGG == SKX_AGG_COUNT ? p.fk : p.measure) + p.head);
    const int64_t nvec = (p.F - p.head) >> 2;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nthr = int64_t(gridDim.x) * blockDim.x;

    if (UNROLL > 0) {
        constexpr int U = UNROLL > 0 ? UNROLL : 1;
        // software pipeline: the 16-byte fk / measure vectors of the next
        // iteration are in flight while this iteration's gathers resolve
        int4 nk[U], nm[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = tid + u * nthr;
            nk[u] = make_int4(0, 0, 0, 0);
            nm[u] = make_int4(0, 0, 0, 0);
            if (i < nvec) {
                nk[u] = ld_stream16(fk4 + i, pol_s);
                if (AGG != SKX_AGG_COUNT) nm[u] = ld_stream16(m4 + i, pol_s);
            }
        }
        for (int64_t base = tid; base < nvec; base += nthr * U) {
            int32_t key[4 * U], mea[4 * U];
            bool valid[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                valid[u] = base + u * nthr < nvec;
                key[4 * u + 0] = nk[u].x; key[4 * u + 1] = nk[u].y; key[4 * u + 2] = nk[u].z; key[4 * u + 3] = nk[u].w;
                mea[4 * u + 0] = nm[u].x; mea[4 * u + 1] = nm[u].y; mea[4 * u + 2] = nm[u].z; mea[4 * u + 3] = nm[u].w;
            }
            int4 row[4 * U];
#pragma unroll
            for (int j = 0; j < 4 * U; ++j) {
                const uint32_t k = (uint32_t)key[j];
                row[j] = make_int4(0, 0, 0, 0);
                if (valid[j / 4] && k >= (uint32_t)p.t_hot && k < (uint32_t)p.N)
                    row[j] = fetch_row<PATH, AGG>(p, key[j], pol_g);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = base + (U + u) * nthr;
                if (i < nvec) {
                    nk[u] = ld_stream16(fk4 + i, pol_s);
                    if (AGG != SKX_AGG_COUNT) nm[u] = ld_stream16(m4 + i, pol_s);
                }
            }
#pragma unroll
            for (int j = 0; j < 4 * U; ++j)
                if (valid[j / 4]) handle_row<AGG, PATH, GSMEM>(p, key[j], mea[j], row[j], acc, g, h, lane);
        }
        // unaligned head (< 4 rows) and ragged tail (< 4 rows)
        if (tid < 8) {
            const int64_t tail0 = p.head + (nvec << 2);
            int64_t idx = -1;
            if (tid < p.head) idx = tid;
            else if (tid >= 4 && tail0 + (tid - 4) < p.F) idx = tail0 + (tid - 4);
            if (idx >= 0) {
                const int32_t k = p.fk[idx];
                const int32_t m = AGG == SKX_AGG_COUNT ? 0 : p.measure[idx];
                int4 row = make_int4(0, 0, 0, 0);
                if ((uint32_t)k >= (uint32_t)p.t_hot && (uint32_t)k < (uint32_t)p.N)
                    row = fetch_row<PATH, AGG>(p, k, pol_g);
                handle_row<AGG, PATH, GSMEM>(p, k, m, row, acc, g, h, lane);
            }
        }
    } else {
        // fk and measure at different offsets mod 16 bytes: 4-byte loads, one row per step
        for (int64_t i = tid; i < p.F; i += nthr) {
            const int32_t k = ld_stream4(p.fk + i, pol_s);
            const int32_t m = AGG == SKX_AGG_COUNT ? 0 : ld_stream4(p.measure + i, pol_s);
            int4 row = make_int4(0, 0, 0, 0);
            if ((uint32_t)k >= (uint32_t)p.t_hot && (uint32_t)k < (uint32_t)p.N) row = fetch_row<PATH, AGG>(p, k, pol_g);
            handle_row<AGG, PATH, GSMEM>(p, k, m, row, acc, g, h, lane);
        }
    }
    __syncthreads();

    // hot prefix: one lookup per hot row per CTA
    for (int k = threadIdx.x; k < p.t_hot; k += blockDim.x) {
        unsigned long long s = hot_value(h.lo[k], h.hi[k]);
        if (k < p.t_lane) {
#pragma unroll 8
            for (int l = 0; l < 32; ++l) s += hot_value(h.lane_lo[(size_t(k) << 5) + l], h.lane_hi[(size_t(k) << 5) + l]);
        }
        if (s == 0) continue;
        const int4 v = fetch_row<PATH, AGG>(p, k, pol_g);
        fold_sum<AGG, GSMEM>(p, v, s, acc, g);
    }
    flush_groups<AGG, GSMEM>(p, acc, g);
}

// The probe over 8-byte rows without a hot prefix -- the query's permuted copy
// of Section III-B, the timed path -- as k_probe<AGG, kRow8, GSMEM, 1> computes
// it with t = 0 and the default gather priority, in a leaner kernel: no
// hot-prefix state, the rows kept as 8-byte pairs, 32-bit loop indices.  At
// most 40 registers (against 54) let three 512-thread CTAs share an SM instead
// of two, so half as many gathers again are in flight.
template <int AGG, bool GSMEM>
__global__ void __launch_bounds__(512, 3) k_probe_r8(PP p) {
    extern __shared__ unsigned long long smem[];
    GrpRef g;
    g.lo = reinterpret_cast<uint32_t *>(smem);
    g.hi = g.lo + (GSMEM ? p.G : 0);
    if (GSMEM)
        for (int i = threadIdx.x; i < p.G; i += blockDim.x) smem[i] = 0;
    __syncthreads();
    const uint64_t pol_s = policy_evict_first();
    unsigned long long acc = 0;
    const int2 *rows = reinterpret_cast<const int2 *>(p.rows);
    const int4 *fk4 = reinterpret_cast<const int4 *>(p.fk + p.head);
    const int4 *m4 = reinterpret_cast<const int4 *>((AGG == SKX_AGG_COUNT ? p.fk : p.measure) + p.head);
    // F < 2^32, so the vector count and indices fit 32 bits
    const uint32_t nvec = (uint32_t)((p.F - p.head) >> 2);
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nthr = gridDim.x * blockDim.x;
    // the row's filter, group and payload values from the pair (columns 0 or 1)
    auto unpack = [&p](const int2 &r) {
        int4 v;
        v.x = p.fcol >= 0 ? sel2(r, p.fcol) : 0;
        v.y = AGG == SKX_AGG_GROUPBY_SUM ? sel2(r, p.gcol) : 0;
        v.z = p.pcol >= 0 ? sel2(r, p.pcol) : 1;
        v.w = 0;
        return v;
    };
    int4 nk = make_int4(0, 0, 0, 0), nm = nk;
    if (tid < nvec) {
        nk = ld_stream16(fk4 + tid, pol_s);
        if (AGG != SKX_AGG_COUNT) nm = ld_stream16(m4 + tid, pol_s);
    }
    for (uint32_t i = tid; i < nvec; i += nthr) {
        const int32_t key[4] = {nk.x, nk.y, nk.z, nk.w};
        const int32_t mea[4] = {nm.x, nm.y, nm.z, nm.w};
        int2 r[4];
        bool use[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            use[j] = (uint32_t)key[j] < (uint32_t)p.N;
            r[j] = use[j] ? __ldg(rows + key[j]) : make_int2(0, 0);
        }
        // the next vectors are in flight while these gathers resolve
        if (nvec - i > nthr) {
            nk = ld_stream16(fk4 + (i + nthr), pol_s);
            if (AGG != SKX_AGG_COUNT) nm = ld_stream16(m4 + (i + nthr), pol_s);
        }
        if (!(use[0] && use[1] && use[2] && use[3])) raise_error(p.err, kErrKeyRange);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (use[j]) fold_row<AGG, GSMEM>(p, unpack(r[j]), mea[j], acc, g);
    }
    // unaligned head (< 4 rows) and ragged tail (< 4 rows)
    if (tid < 8) {
        const int64_t tail0 = p.head + (int64_t(nvec) << 2);
        int64_t idx = -1;
        if (tid < p.head) idx = tid;
        else if (tid >= 4 && tail0 + (tid - 4) < p.F) idx = tail0 + (tid - 4);
        if (idx >= 0) {
            const int32_t k = p.fk[idx];
            const int32_t m = AGG == SKX_AGG_COUNT ? 0 : p.measure[idx];
            if ((uint32_t)k < (uint32_t)p.N) fold_row<AGG, GSMEM>(p, unpack(__ldg(rows + k)), m, acc, g);
            else raise_error(p.err, kErrKeyRange);
        }
    }
    flush_groups<AGG, GSMEM>(p, acc, g);
}

template <int AGG, bool GSMEM>
cudaError_t launch_r8(const PP &p, const skx_tuning &t, size_t smem, cudaStream_t st);

// The probe over the packed query copy: 4-byte rows, key = code >> (32 - kbits)
// (a group, or G for a filtered row), payload = the code's low 32 - kbits bits
// sign-extended; the escape (key field all ones) reads the row's 8-byte copy
// (p.rows).  p carries the prefiltered form of the query (filter "key < G" on
// column 0, group column 0, payload column 1), so each row folds exactly as the
// probe over the 8-byte copy folds it.  Half the bytes per row: twice as many
// rows per cache line and a table half the size in L2.
template <int AGG, bool GSMEM>
__global__ void __launch_bounds__(512, 3) k_probe_p4(PP p, const uint32_t *__restrict__ rows4, int32_t kbits) {
    extern __shared__ unsigned long long smem[];
    GrpRef g;
    g.lo = reinterpret_cast<uint32_t *>(smem);
    g.hi = g.lo + (GSMEM ? p.G : 0);
    if (GSMEM)
        for (int i = threadIdx.x; i < p.G; i += blockDim.x) smem[i] = 0;
    __syncthreads();
    const uint64_t pol_s = policy_evict_first();
    unsigned long long acc = 0;
    const int2 *rows8 = reinterpret_cast<const int2 *>(p.rows);
    const int4 *fk4 = reinterpret_cast<const int4 *>(p.fk + p.head);
    const int4 *m4 = reinterpret_cast<const int4 *>((AGG == SKX_AGG_COUNT ? p.fk : p.measure) + p.head);
    const uint32_t nvec = (uint32_t)((p.F - p.head) >> 2);  // F < 2^32
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nthr = gridDim.x * blockDim.x;
    const uint32_t esc = (1u << kbits) - 1u;
    // {key, key, payload} of row k from its code c
    auto decode = [&](uint32_t c, int32_t k) {
        int4 v;
        if ((c >> (32 - kbits)) == esc) {
            const int2 r = __ldg(rows8 + k);
            v.x = r.x;
            v.z = r.y;
        } else {
            v.x = (int32_t)(c >> (32 - kbits));
            v.z = (int32_t)(c << kbits) >> kbits;
        }
        v.y = v.x;
        v.w = 0;
        return v;
    };
    int4 nk = make_int4(0, 0, 0, 0), nm = nk;
    if (tid < nvec) {
        nk = ld_stream16(fk4 + tid, pol_s);
        if (AGG != SKX_AGG_COUNT) nm = ld_stream16(m4 + tid, pol_s);
    }
    for (uint32_t i = tid; i < nvec; i += nthr) {
        const int32_t key[4] = {nk.x, nk.y, nk.z, nk.w};
        const int32_t mea[4] = {nm.x, nm.y, nm.z, nm.w};
        uint32_t c[4];
        bool use[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            use[j] = (uint32_t)key[j] < (uint32_t)p.N;
            c[j] = use[j] ? __ldg(rows4 + key[j]) : 0u;
        }
        if (nvec - i > nthr) {
            nk = ld_stream16(fk4 + (i + nthr), pol_s);
            if (AGG != SKX_AGG_COUNT) nm = ld_stream16(m4 + (i + nthr), pol_s);
        }
        if (!(use[0] && use[1] && use[2] && use[3])) raise_error(p.err, kErrKeyRange);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (use[j]) fold_row<AGG, GSMEM>(p, decode(c[j], key[j]), mea[j], acc, g);
    }
    if (tid < 8) {  // unaligned head (< 4 rows) and ragged tail (< 4 rows)
        const int64_t tail0 = p.head + (int64_t(nvec) << 2);
        int64_t idx = -1;
        if (tid < p.head) idx = tid;
        else if (tid >= 4 && tail0 + (tid - 4) < p.F) idx = tail0 + (tid - 4);
        if (idx >= 0) {
            const int32_t k = p.fk[idx];
            const int32_t m = AGG == SKX_AGG_COUNT ? 0 : p.measure[idx];
            if ((uint32_t)k < (uint32_t)p.N) fold_row<AGG, GSMEM>(p, decode(__ldg(rows4 + k), k), m, acc, g);
            else raise_error(p.err, kErrKeyRange);
        }
    }
    flush_groups<AGG, GSMEM>(p, acc, g);
}

template <typename K, typename... Args>
cudaError_t launch_lean(K kern, int64_t F, int64_t head, const skx_tuning &t, size_t smem, cudaStream_t st,
                        Args... args) {
    cudaError_t e = set_smem_limit_once(reinterpret_cast<const void *>(kern), -1);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, t.block_threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (t.ctas_per_sm > 0 && t.ctas_per_sm < per_sm) per_sm = t.ctas_per_sm;
    const int64_t need = (((F - head) >> 2) + t.block_threads - 1) / t.block_threads;
    int64_t grid = int64_t(device_sm_count()) * per_sm;
    if (need < grid) grid = need < 1 ? 1 : need;
    kern<<<(unsigned)grid, t.block_threads, smem, st>>>(args...);
    note_launches(1);
    return cudaGetLastError();
}

template <int AGG, bool GSMEM>
cudaError_t launch_r8(const PP &p, const skx_tuning &t, size_t smem, cudaStream_t st) {
    return launch_lean(k_probe_r8<AGG, GSMEM>, p.F, p.head, t, smem, st, p);
}

template <int AGG, int PATH, bool GSMEM, int UNROLL>
cudaError_t launch_one(const PP &p, const skx_tuning &t, size_t smem, cudaStream_t st) {
    auto kern = k_probe<AGG, PATH, GSMEM, UNROLL>;
    // dynamic + static shared memory must fit the per-block limit
    cudaError_t e = set_smem_limit_once(reinterpret_cast<const void *>(kern), -1);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, t.block_threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (t.ctas_per_sm > 0 && t.ctas_per_sm < per_sm) per_sm = t.ctas_per_sm;
    const int sms = device_sm_count();
    const int64_t work = UNROLL > 0 ? ((p.F - p.head) >> 2) : p.F;
    const int64_t per_thread = UNROLL > 0 ? UNROLL : 1;
    int64_t need = (work + int64_t(t.block_threads) * per_thread - 1) / (int64_t(t.block_threads) * per_thread);
    int64_t grid = int64_t(sms) * per_sm;
    if (need < grid) grid = need < 1 ? 1 : need;
    kern<<<(unsigned)grid, t.block_threads, smem, st>>>(p);
    note_launches(1);
    return cudaGetLastError();
}

template <int AGG, int PATH, bool GSMEM>
cudaError_t launch_unroll(const PP &p, const skx_tuning &t, size_t smem, cudaStream_t st, bool vec) {
    if (!vec) return launch_one<AGG, PATH, GSMEM, 0>(p, t, smem, st);
    // the lean kernel gathers with the default L2 priority (gather_policy 2)
    if (PATH == kRow8 && p.t_hot == 0 && t.unroll == 1 && p.gather_policy == 2)
        return launch_r8<AGG, GSMEM>(p, t, smem, st);
    switch (t.unroll) {
        case 1: return launch_one<AGG, PATH, GSMEM, 1>(p, t, smem, st);
        case 4: return launch_one<AGG, PATH, GSMEM, 4>(p, t, smem, st);
        default: return launch_one<AGG, PATH, GSMEM, 2>(p, t, smem, st);
    }
}

template <int AGG>
cudaError_t launch_agg(const PP &p, int path, bool gsmem, const skx_tuning &t, size_t smem, cudaStream_t st,
                       bool vec) {
    if (AGG != SKX_AGG_GROUPBY_SUM) gsmem = false;  // COUNT and SUM accumulate in registers
    if (path == kRow16) {
        if (gsmem) return launch_unroll<AGG, kRow16, true>(p, t, smem, st, vec);
        return launch_unroll<AGG, kRow16, false>(p, t, smem, st, vec);
    }
    if (path == kRow8) {
        if (gsmem) return launch_unroll<AGG, kRow8, true>(p, t, smem, st, vec);
        return launch_unroll<AGG, kRow8, false>(p, t, smem, st, vec);
    }
    if (gsmem) return launch_unroll<AGG, kRowGeneric, true>(p, t, smem, st, vec);
    return launch_unroll<AGG, kRowGeneric, false>(p, t, smem, st, vec);
}

int32_t clamp32(int64_t v, int64_t lo, int64_t hi) { return (int32_t)(v < lo ? lo : (v > hi ? hi : v)); }

}  // namespace

skx_status validate_query(const skx_query *q, int32_t row_bytes) {
    if (!q || row_bytes <= 0 || row_bytes % 4 != 0) return SKX_EINVAL;
    const int32_t words = row_bytes / 4;
    if (q->agg < SKX_AGG_COUNT || q->agg > SKX_AGG_GROUPBY_SUM) return SKX_EINVAL;
    if (q->filter_col < -1 || q->filter_col >= words) return SKX_EINVAL;
    if (q->payload_col < -1 || q->payload_col >= words) return SKX_EINVAL;
    if (q->agg == SKX_AGG_GROUPBY_SUM) {
        if (q->group_col < 0 || q->group_col >= words) return SKX_EINVAL;
        if (q->num_groups < 1 || q->num_groups > (1 << 24)) return SKX_EINVAL;
    }
    return SKX_OK;
}

void resolve_hot(const ProbeArgs &a, skx_tuning &t, int64_t other_smem);

// Fills the defaults of `t` in place.  Idempotent: a resolved tuning resolves
// to itself ("off" and "as many as fit" are -1, never 0).
void resolve_probe_tuning(const ProbeArgs &a, skx_tuning &t) {
    if (t.block_threads != 128 && t.block_threads != 256 && t.block_threads != 512) t.block_threads = 512;
    // one 16-byte vector per thread per step and 1024 threads per SM by default: the
    // gathers are latency bound, so resident warps matter more than per-thread depth
    if (t.unroll != 1 && t.unroll != 2 && t.unroll != 4) t.unroll = 1;
    if (t.ctas_per_sm == 0) t.ctas_per_sm = 1024 / t.block_threads;
    if (t.ctas_per_sm < 0) t.ctas_per_sm = -1;
    if (t.gather_policy < 1 || t.gather_policy > 4) t.gather_policy = 2;
    if (t.split_bucket < 12 || t.split_bucket > 26) t.split_bucket = 19;
    if (t.split_keys <= 0 || t.split_keys >= a.N) t.split_keys = -1;
    {
        // the split's staging must fit beside the group sums in one CTA
        const bool grp = a.q.agg == SKX_AGG_GROUPBY_SUM;
        const int64_t gbytes = (grp && a.q.num_groups <= kMaxSmemGroups) ? int64_t(a.q.num_groups) * 8 : 0;
        if (t.split_keys > 0 && gbytes + kSplitSmemBytes + 1024 > device_max_smem_optin()) t.split_keys = -1;
    }
    resolve_hot(a, t, t.split_keys > 0 ? kSplitSmemBytes : 0);
    // the split needs keys [hot_keys, split_keys) to exist
    const int32_t hot = t.hot_keys > 0 ? t.hot_keys : 0;
    if (t.split_keys <= hot || t.split_keys >= a.N) t.split_keys = -1;
    if (t.split_keys > 0) split_buckets(a.N, t.split_keys, &t.split_bucket);
}

// The hot prefix's shared-memory share: whatever the groups and, for the split
// probe, its staging area (other_smem bytes) leave.
void resolve_hot(const ProbeArgs &a, skx_tuning &t, int64_t other_smem) {
    if (t.hot_keys < 0) {
        t.hot_keys = -1;
        t.lane_keys = -1;
        return;
    }
    const bool grp = a.q.agg == SKX_AGG_GROUPBY_SUM;
    const int64_t gbytes = (grp && a.q.num_groups <= kMaxSmemGroups) ? int64_t(a.q.num_groups) * 8 : 0;
    const int64_t optin = device_max_smem_optin();
    if (t.lane_keys == 0) t.lane_keys = 32;
    if (t.lane_keys < 0) t.lane_keys = 0;
    if (t.hot_keys == 0) {  // sized so that two CTAs fit per SM
        const int64_t budget = optin / 2 - 2048 - other_smem;
        t.hot_keys = (int32_t)(((budget - gbytes - int64_t(t.lane_keys) * 256) / 8) & ~int64_t(1023));
    }
    const int64_t room = (optin - 1024 - gbytes - other_smem) / 8;  // 8 bytes per hot key, 256 per lane key
    if (room < 1 || t.hot_keys < 1) {  // no shared memory left for a hot prefix
        t.hot_keys = -1;
        t.lane_keys = -1;
        return;
    }
    t.hot_keys = clamp32(t.hot_keys, 1, a.N);
    t.lane_keys = clamp32(t.lane_keys, 0, t.hot_keys);
    if (int64_t(t.hot_keys) + int64_t(t.lane_keys) * 32 > room) {
        t.lane_keys = clamp32(t.lane_keys, 0, room / 64);
        t.hot_keys = clamp32(t.hot_keys, 1, room - int64_t(t.lane_keys) * 32);
        t.lane_keys = clamp32(t.lane_keys, 0, t.hot_keys);
    }
    if (t.lane_keys == 0) t.lane_keys = -1;
}

cudaError_t launch_probe(const ProbeArgs &a, const skx_tuning &t, cudaStream_t st) {
    PP p{};
    p.fk = a.fk;
    p.measure = a.measure;
    p.F = a.F;
    p.rows = static_cast<const char *>(a.rows);
    p.N = a.N;
    p.row_bytes = a.row_bytes;
    p.fcol = a.q.filter_col;
    p.flt = a.q.filter_lt;
    p.gcol = a.q.group_col;
    p.G = a.q.agg == SKX_AGG_GROUPBY_SUM ? a.q.num_groups : 1;
    p.pcol = a.q.payload_col;
    p.t_hot = t.hot_keys > 0 ? t.hot_keys : 0;
    p.t_lane = t.lane_keys > 0 ? t.lane_keys : 0;
    p.gather_policy = t.gather_policy;
    p.out = reinterpret_cast<unsigned long long *>(a.out);
    p.err = a.err;
    const int nout = a.q.agg == SKX_AGG_GROUPBY_SUM ? a.q.num_groups : 1;
    cudaError_t e = a.accumulate ? cudaSuccess : cudaMemsetAsync(a.out, 0, size_t(nout) * 8, st);
    if (e != cudaSuccess || a.F <= 0) return e;

    // vector path needs fk and measure at the same offset mod 16 bytes
    const uintptr_t af = reinterpret_cast<uintptr_t>(a.fk) & 15u;
    const uintptr_t am = a.q.agg == SKX_AGG_COUNT ? af : (reinterpret_cast<uintptr_t>(a.measure) & 15u);
    const int64_t mis = (int64_t)(af >> 2);
    p.head = mis ? (a.F < 4 - mis ? a.F : 4 - mis) : 0;
    int path = kRowGeneric;
    if (a.row_bytes % 16 == 0 && aligned16(a.rows) && p.fcol < 4 && p.gcol < 4 && p.pcol < 4)
        path = kRow16;
    else if (a.row_bytes == 8 && (reinterpret_cast<uintptr_t>(a.rows) & 7u) == 0 && p.fcol < 2 && p.gcol < 2 &&
             p.pcol < 2)
        path = kRow8;
    const bool gsmem = a.q.agg == SKX_AGG_GROUPBY_SUM && a.q.num_groups <= kMaxSmemGroups;
    const size_t smem = size_t((gsmem ? a.q.num_groups : 0) + p.t_hot + p.t_lane * 32) * 8;

    const bool vec = af == am;
    if (vec && t.split_keys > 0) {
        bool ran = false;
        e = launch_probe_split(p, a.q.agg, path, gsmem, t, st, &ran);
        if (e != cudaSuccess || ran) return e;
    }
    switch (a.q.agg) {
        case SKX_AGG_COUNT: return launch_agg<SKX_AGG_COUNT>(p, path, gsmem, t, smem, st, vec);
        case SKX_AGG_SUM: return launch_agg<SKX_AGG_SUM>(p, path, gsmem, t, smem, st, vec);
        default: return launch_agg<SKX_AGG_GROUPBY_SUM>(p, path, gsmem, t, smem, st, vec);
    }
}

cudaError_t launch_probe_packed(const ProbeArgs &a, const uint32_t *rows4, const skx_tuning &t_in, cudaStream_t st) {
    const skx_query qp = skx_query_prefiltered(&a.q);
    PP p{};
    p.fk = a.fk;
    p.measure = a.measure;
    p.F = a.F;
    p.rows = static_cast<const char *>(a.rows);
    p.N = a.N;
    p.row_bytes = 8;
    p.fcol = qp.filter_col;
    p.flt = qp.filter_lt;
    p.gcol = qp.group_col;
    p.G = qp.num_groups;
    p.pcol = qp.payload_col;
    p.gather_policy = 2;
    p.out = reinterpret_cast<unsigned long long *>(a.out);
    p.err = a.err;
    const int nout = a.q.agg == SKX_AGG_GROUPBY_SUM ? a.q.num_groups : 1;
    cudaError_t e = a.accumulate ? cudaSuccess : cudaMemsetAsync(a.out, 0, size_t(nout) * 8, st);
    if (e != cudaSuccess || a.F <= 0) return e;
    skx_tuning t = t_in;
    if (t.block_threads != 128 && t.block_threads != 256 && t.block_threads != 512) t.block_threads = 512;
    if (t.ctas_per_sm == 0) t.ctas_per_sm = -1;
    const int32_t kbits = packed_key_bits(a.q);
    const bool gsmem = a.q.agg == SKX_AGG_GROUPBY_SUM && a.q.num_groups <= kMaxSmemGroups;
    const size_t smem = gsmem ? size_t(a.q.num_groups) * 8 : 0;
    const uintptr_t af = reinterpret_cast<uintptr_t>(a.fk) & 15u;
    const uintptr_t am = a.q.agg == SKX_AGG_COUNT ? af : (reinterpret_cast<uintptr_t>(a.measure) & 15u);
    if (af == am) {
        const int64_t mis = (int64_t)(af >> 2);
        p.head = mis ? (a.F < 4 - mis ? a.F : 4 - mis) : 0;
    } else {
        // fk and measure at different offsets mod 16 bytes: the kernel's 16-byte loads cannot
        // serve both, so the rows are probed through the 8-byte copy instead
        skx_tuning t8{};
        t8.block_threads = t.block_threads;
        t8.ctas_per_sm = t.ctas_per_sm;
        t8.hot_keys = -1;
        t8.lane_keys = -1;
        ProbeArgs a8 = a;
        a8.row_bytes = 8;
        a8.q = qp;
        a8.accumulate = true;
        resolve_probe_tuning(a8, t8);
        return launch_probe(a8, t8, st);
    }
    switch (a.q.agg) {
        case SKX_AGG_COUNT:
            return launch_lean(k_probe_p4<SKX_AGG_COUNT, false>, p.F, p.head, t, smem, st, p, rows4, kbits);
        case SKX_AGG_SUM:
            return launch_lean(k_probe_p4<SKX_AGG_SUM, false>, p.F, p.head, t, smem, st, p, rows4, kbits);
        default:
            if (gsmem)
                return launch_lean(k_probe_p4<SKX_AGG_GROUPBY_SUM, true>, p.F, p.head, t, smem, st, p, rows4, kbits);
            return launch_lean(k_probe_p4<SKX_AGG_GROUPBY_SUM, false>, p.F, p.head, t, smem, st, p, rows4, kbits);
    }
}

}  // namespace skx
