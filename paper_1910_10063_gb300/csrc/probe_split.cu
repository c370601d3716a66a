// probe_split.cu -- the FK-join probe with threshold-based splitting of the
// fact stream (Section IV-B: ids below a threshold t are likely cache hits
// and are resolved at once; the likely misses are written to a buffer and
// resolved by a second pass over that buffer).
//
// On this GPU the cost of a miss is not its latency (resident warps hide
// it) but the DRAM line it fetches: a cold dimension row that several fact
// rows reference is evicted between its references by the streaming fact
// columns and fetched again each time.  So the second pass here does more
// than the paper's: the buffer is bucketed by rank range, and the pass walks
// the buckets in rank order across the whole GPU, so that the dimension
// lines of the bucket in progress stay in L2 and every cold line is fetched
// close to once per probe.
//
// Pass 1 (k_probe_split), a persistent grid streaming fk and measure with
// 16-byte loads, one vector (4 rows) per thread per sub-step:
//   * k < t_hot          per-key shared-memory sums (threshold processing),
//                        folded once per CTA at the end (as in probe.cu);
//   * t_hot <= k < t     gathered and folded at once (likely L2 hits);
//   * t <= k < N         deferred: staged in shared memory with its rank
//                        within its bucket (bucket = (k - t) >> bshift).
// Each class's shared atomics for the 4 rows are issued together.  After a
// sub-step that leaves at least kFlushAt rows staged, the CTA lays them out
// bucket by bucket in its own region of the global buffer (no global
// atomics: every CTA owns cap / grid entries) and records the flush in a
// run table: per flush its start in the buffer, and per bucket the run's
// offset and length packed in one word (bucket-major, so the second pass
// reads the runs of one bucket contiguously).  A CTA whose region is full
// resolves its staged rows itself.
// Pass 2 (k_probe_deferred): each warp takes units (bucket, CTA, 8
// consecutive flushes of that CTA) from an atomic counter in bucket-major
// order, concatenates the 8 runs, and resolves them 128 entries per round
// with the next round's entries already loading.
// Sums are exact modulo 2^64 in any order, so the result equals probe.cu's.
#include <algorithm>

#include "probe_core.cuh"

namespace skx {
namespace {

using namespace pcore;

constexpr int kSplitThreads = 512;
constexpr int kStage = 4096;                          // staged rows per CTA
constexpr int kFlushAt = kStage - 4 * kSplitThreads;  // one more sub-step always fits
constexpr int kMaxBuckets = 512;
constexpr int kRunsPerUnit = 8;
constexpr int kUnitBatch = 4;  // entries per lane per round of pass 2 (fold4 takes four)

static_assert(kFlushAt > 0 && kStage < 65536, "staging sizes (offsets and lengths packed in 16 bits)");
static_assert(int64_t(kStage) * 10 + int64_t(kMaxBuckets) * 8 <= kSplitSmemBytes, "staging smem budget");

struct SP {
    int2 *miss;         // deferred (key, measure) rows: CTA c owns [c * region, (c + 1) * region)
    uint32_t region;    // entries per CTA
    uint32_t max_flush; // numbered flushes per CTA at most
    uint32_t *fbase;    // [grid][max_flush] first buffer entry of each flush
    uint32_t *runs;     // [B][grid][max_flush] run offset (low 16 bits) and length (high 16 bits)
    uint32_t *nflush;   // [grid] numbered flushes of each CTA
    uint32_t *ctr;      // [0] largest nflush, [1] pass-2 units taken
    int32_t t_split;
    int32_t bshift;
    int32_t B;
    int32_t grid;       // CTAs of pass 1
};

__device__ __forceinline__ void st_evict_first8(int2 *p, int2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.s32 [%0], {%1,%2}, %3;" ::"l"(p), "r"(v.x), "r"(v.y), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ int2 ld_stream8(const int2 *p, uint64_t pol) {
    int2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.s32 {%0,%1}, [%2], %3;"
                 : "=r"(v.x), "=r"(v.y)
                 : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, unsigned lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (unsigned)o) v += y;
    }
    return v;
}

struct Stage {
    int2 *rows;      // kStage entries
    uint16_t *rank;  // kStage ranks within their bucket
    uint32_t *cnt;   // B
    uint32_t *off;   // B
    uint32_t *fill;  // staged rows
    uint32_t *cur;   // [0] entries of the CTA's region used, [1] numbered flushes
};

// Moves the staged rows into the CTA's region of the global buffer (or
// resolves them here when the region is full) and clears the stage.  Called
// by every thread of the CTA after a barrier, with the same stage contents.
template <int AGG, int PATH, bool GSMEM>
__device__ void flush_stage(const PP &p, const SP &d, const Stage &s, uint64_t pol_g, uint64_t pol_w,
                            unsigned long long &acc, GrpRef g) {
    const uint32_t n = *s.fill;
    const uint32_t used = s.cur[0], k = s.cur[1];
    const bool ok = used + n <= d.region && k < d.max_flush;
    if (threadIdx.x < 32) {
        const unsigned lane = lane_id();
        uint32_t carry = 0;
        for (int b0 = 0; b0 < d.B; b0 += 32) {
            const int b = b0 + (int)lane;
            const uint32_t c = b < d.B ? s.cnt[b] : 0u;
            const uint32_t incl = warp_incl_scan(c, lane);
            if (b < d.B) s.off[b] = carry + incl - c;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    if (ok) {
        const size_t fi = size_t(blockIdx.x) * d.max_flush + k;
        const uint32_t base = blockIdx.x * d.region + used;
        if (threadIdx.x == 0) d.fbase[fi] = base;
        const size_t stride = size_t(d.grid) * d.max_flush;
        for (int b = threadIdx.x; b < d.B; b += blockDim.x) d.runs[size_t(b) * stride + fi] = s.off[b] | (s.cnt[b] << 16);
        for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
            const int2 v = s.rows[e];
            const int b = (v.x - d.t_split) >> d.bshift;
            st_evict_first8(d.miss + (size_t(base) + s.off[b] + s.rank[e]), v, pol_w);
        }
    } else {
        // no room left in this CTA's region: resolve the staged rows here
        for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
            const int2 v = s.rows[e];
            const int4 row = fetch_row<PATH, AGG>(p, v.x, pol_g);
            fold_row<AGG, GSMEM>(p, row, v.y, acc, g);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < d.B; b += blockDim.x) s.cnt[b] = 0;
    if (threadIdx.x == 0) {
        *s.fill = 0;
        if (ok) {
            s.cur[0] = used + n;
            s.cur[1] = k + 1;
        }
    }
    __syncthreads();
}

template <int AGG, int PATH, bool GSMEM>
__global__ void __launch_bounds__(kSplitThreads, 2) k_probe_split(PP p, SP d) {
    extern __shared__ unsigned long long smem[];
    __shared__ uint32_t s_fill, s_cur[2];
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
    Stage s;
    s.rows = reinterpret_cast<int2 *>(smem + nsm);
    s.rank = reinterpret_cast<uint16_t *>(s.rows + kStage);
    s.cnt = reinterpret_cast<uint32_t *>(s.rank + kStage);
    s.off = s.cnt + d.B;
    s.fill = &s_fill;
    s.cur = s_cur;
    for (int i = threadIdx.x; i < nsm; i += blockDim.x) smem[i] = 0;
    for (int b = threadIdx.x; b < d.B; b += blockDim.x) s.cnt[b] = 0;
    if (threadIdx.x == 0) {
        s_fill = 0;
        s_cur[0] = 0;
        s_cur[1] = 0;
    }
    __syncthreads();

    const uint64_t pol_s = policy_evict_first();
    const uint64_t pol_g = policy_by_code(p.gather_policy);
    const unsigned lane = lane_id();
    unsigned long long acc = 0;
    const uint32_t t_hot = (uint32_t)p.t_hot, t_split = (uint32_t)d.t_split, nkeys = (uint32_t)p.N;

    const int4 *fk4 = reinterpret_cast<const int4 *>(p.fk + p.head);
    const int4 *m4 = reinterpret_cast<const int4 *>((AGG == SKX_AGG_COUNT ? p.fk : p.measure) + p.head);
    const int64_t nvec = (p.F - p.head) >> 2;
    const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
    const int64_t cta0 = int64_t(blockIdx.x) * blockDim.x;

    int4 nk = make_int4(0, 0, 0, 0), nm = make_int4(0, 0, 0, 0);
    if (cta0 + threadIdx.x < nvec) {
        nk = ld_stream16(fk4 + cta0 + threadIdx.x, pol_s);
        if (AGG != SKX_AGG_COUNT) nm = ld_stream16(m4 + cta0 + threadIdx.x, pol_s);
    }
    // every thread of the CTA runs the same number of sub-steps (base is CTA-uniform)
    for (int64_t base = cta0; base < nvec; base += nthr) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < nvec;
        const int32_t key[4] = {nk.x, nk.y, nk.z, nk.w};
        const int32_t mea[4] = {nm.x, nm.y, nm.z, nm.w};
        bool hot[4], direct[4], defer[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t k = (uint32_t)key[j];
            hot[j] = valid && k < t_hot;
            direct[j] = valid && k >= t_hot && k < t_split;
            defer[j] = valid && k >= t_split && k < nkeys;
            if (valid && k >= nkeys) raise_error(p.err, kErrKeyRange);
        }
        int4 row[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            row[j] = make_int4(0, 0, 0, 0);
            if (direct[j]) row[j] = fetch_row<PATH, AGG>(p, key[j], pol_g);
        }
        if (i + nthr < nvec) {
            nk = ld_stream16(fk4 + i + nthr, pol_s);
            if (AGG != SKX_AGG_COUNT) nm = ld_stream16(m4 + i + nthr, pol_s);
        }
        if (t_hot) hot_add4<AGG>(p, h, key, mea, hot, lane);
        // stage slots for the warp's deferred rows: one shared atomic per warp
        const uint32_t ndef = (uint32_t)defer[0] + defer[1] + defer[2] + defer[3];
        const uint32_t incl = warp_incl_scan(ndef, lane);
        const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t wbase = 0;
        if (lane == 31 && wtot) wbase = atomicAdd(&s_fill, wtot);
        uint32_t slot = __shfl_sync(0xffffffffu, wbase, 31) + incl - ndef;
        uint32_t r[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            r[j] = defer[j] ? atomicAdd(s.cnt + (((uint32_t)key[j] - t_split) >> d.bshift), 1u) : 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (defer[j]) {
                s.rows[slot] = make_int2(key[j], mea[j]);
                s.rank[slot] = (uint16_t)r[j];
                ++slot;
            }
        fold4<AGG, GSMEM>(p, row, mea, direct, acc, g);
        // The stage's fill after this sub-step is the largest value any warp's
        // reservation returned, so the barrier's OR over those tells every thread
        // the same answer (reading s_fill itself here would race with warps that
        // already reserve for the next sub-step).
        const bool full = lane == 31 && wtot && wbase + wtot >= (uint32_t)kFlushAt;
        if (__syncthreads_or(full)) flush_stage<AGG, PATH, GSMEM>(p, d, s, pol_g, pol_s, acc, g);
    }
    __syncthreads();
    if (s_fill > 0) flush_stage<AGG, PATH, GSMEM>(p, d, s, pol_g, pol_s, acc, g);
    if (threadIdx.x == 0) {
        d.nflush[blockIdx.x] = s_cur[1];
        atomicMax(d.ctr + 0, s_cur[1]);
    }

    // unaligned head (< 4 rows) and ragged tail (< 4 rows): resolved here
    const int64_t tid = cta0 + threadIdx.x;
    if (tid < 8) {
        const int64_t tail0 = p.head + (nvec << 2);
        int64_t idx = -1;
        if (tid < p.head) idx = tid;
        else if (tid >= 4 && tail0 + (tid - 4) < p.F) idx = tail0 + (tid - 4);
        if (idx >= 0) {
            const int32_t k = p.fk[idx];
            const int32_t m = AGG == SKX_AGG_COUNT ? 0 : p.measure[idx];
            int4 rw = make_int4(0, 0, 0, 0);
            if ((uint32_t)k >= t_hot && (uint32_t)k < nkeys) rw = fetch_row<PATH, AGG>(p, k, pol_g);
            handle_row<AGG, PATH, GSMEM>(p, k, m, rw, acc, g, h, lane);
        }
    }
    __syncthreads();

    // hot prefix: one lookup per hot row per CTA
    for (int k = threadIdx.x; k < p.t_hot; k += blockDim.x) {
        unsigned long long sum = hot_value(h.lo[k], h.hi[k]);
        if (k < p.t_lane) {
#pragma unroll 8
            for (int l = 0; l < 32; ++l)
                sum += hot_value(h.lane_lo[(size_t(k) << 5) + l], h.lane_hi[(size_t(k) << 5) + l]);
        }
        if (sum == 0) continue;
        const int4 v = fetch_row<PATH, AGG>(p, k, pol_g);
        fold_sum<AGG, GSMEM>(p, v, sum, acc, g);
    }
    flush_groups<AGG, GSMEM>(p, acc, g);
}

// Pass 2: the deferred rows, bucket by bucket.  Each lane holds kUnitBatch
// entries of the current round while the next round's entries load, so a warp
// keeps two rounds of memory accesses in flight.
template <int AGG, int PATH, bool GSMEM>
__global__ void __launch_bounds__(kSplitThreads, 2) k_probe_deferred(PP p, SP d) {
    extern __shared__ unsigned long long smem[];
    const int ngrp = GSMEM ? p.G : 0;
    GrpRef g;
    g.lo = reinterpret_cast<uint32_t *>(smem);
    g.hi = g.lo + ngrp;
    for (int i = threadIdx.x; i < ngrp; i += blockDim.x) smem[i] = 0;
    __syncthreads();
    const uint64_t pol_s = policy_evict_first();
    const uint64_t pol_g = policy_by_code(p.gather_policy);
    const unsigned lane = lane_id();
    unsigned long long acc = 0;
    const uint32_t mf = *(volatile uint32_t *)(d.ctr + 0);
    const uint32_t most = mf < d.max_flush ? mf : d.max_flush;
    const uint32_t ku = (most + kRunsPerUnit - 1) / kRunsPerUnit;  // units per CTA per bucket
    const uint64_t upb = uint64_t(ku) * uint64_t(d.grid);          // units per bucket
    const uint64_t total = upb * uint64_t(d.B);
    const size_t stride = size_t(d.grid) * d.max_flush;
    for (;;) {
        uint32_t u = 0;
        if (lane == 0) u = atomicAdd(d.ctr + 1, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (uint64_t(u) >= total) break;
        const uint32_t b = (uint32_t)(u / upb);
        const uint32_t rest = (uint32_t)(u % upb);
        const uint32_t c = rest / ku, k0 = (rest % ku) * kRunsPerUnit;
        const uint32_t nf = d.nflush[c];
        uint32_t cn = 0, st = 0;
        if (lane < (unsigned)kRunsPerUnit && k0 + lane < nf && k0 + lane < d.max_flush) {
            const size_t fi = size_t(c) * d.max_flush + k0 + lane;
            const uint32_t w = d.runs[size_t(b) * stride + fi];
            cn = w >> 16;
            st = d.fbase[fi] + (w & 0xffffu);
        }
        const uint32_t incl = warp_incl_scan(cn, lane);
        const uint32_t excl = incl - cn;
        const uint32_t T = __shfl_sync(0xffffffffu, incl, kRunsPerUnit - 1);
        // entry j of the unit's concatenated runs -> its buffer position
        auto load_round = [&](uint32_t j0, int2 *e) {
#pragma unroll
            for (int q = 0; q < kUnitBatch; ++q) {
                const uint32_t j = j0 + q * 32 + lane;
                uint32_t t = 0;  // the number of runs whose inclusive end is <= j
                if (__shfl_sync(0xffffffffu, incl, 3) <= j) t = 4;
                if (__shfl_sync(0xffffffffu, incl, t + 1) <= j) t += 2;
                if (__shfl_sync(0xffffffffu, incl, t) <= j) t += 1;
                const uint32_t rs = __shfl_sync(0xffffffffu, st, t);
                const uint32_t rx = __shfl_sync(0xffffffffu, excl, t);
                e[q] = make_int2(0, 0);
                if (j < T) e[q] = ld_stream8(d.miss + (size_t(rs) + (j - rx)), pol_s);
            }
        };
        int2 nxt[kUnitBatch];
        load_round(0, nxt);
        for (uint32_t j0 = 0; j0 < T; j0 += 32 * kUnitBatch) {
            int2 e[kUnitBatch];
            int4 row[kUnitBatch];
            int32_t mea[kUnitBatch];
            bool use[kUnitBatch];
#pragma unroll
            for (int q = 0; q < kUnitBatch; ++q) {
                e[q] = nxt[q];
                use[q] = j0 + q * 32 + lane < T;
                mea[q] = e[q].y;
                row[q] = make_int4(0, 0, 0, 0);
                if (use[q]) row[q] = fetch_row<PATH, AGG>(p, e[q].x, pol_g);
            }
            if (j0 + 32 * kUnitBatch < T) load_round(j0 + 32 * kUnitBatch, nxt);
            fold4<AGG, GSMEM>(p, row, mea, use, acc, g);
        }
    }
    flush_groups<AGG, GSMEM>(p, acc, g);
}

template <typename K>
cudaError_t persistent_grid(K kern, size_t smem, int ctas_per_sm, int64_t work_threads, int *grid) {
    cudaError_t e = set_smem_limit_once(reinterpret_cast<const void *>(kern), -1);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSplitThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    int64_t g = int64_t(device_sm_count()) * per_sm;
    const int64_t need = (work_threads + kSplitThreads - 1) / kSplitThreads;
    if (need < g) g = need < 1 ? 1 : need;
    *grid = (int)g;
    return cudaSuccess;
}

// Sizes, allocates (stream-ordered), launches both passes and frees.  *ran is
// false when the scratch could not be allocated (nothing was enqueued then).
template <int AGG, int PATH, bool GSMEM>
cudaError_t run_split(const PP &p, const skx_tuning &t, int32_t bshift, int32_t B, cudaStream_t st, bool *ran) {
    *ran = false;
    auto k1 = k_probe_split<AGG, PATH, GSMEM>;
    auto k2 = k_probe_deferred<AGG, PATH, GSMEM>;
    const size_t grp = size_t(GSMEM ? p.G : 0) * 8;
    const size_t smem1 = grp + size_t(p.t_hot + p.t_lane * 32) * 8 + size_t(kStage) * 10 + size_t(B) * 8;
    const int resident1 = t.ctas_per_sm > 0 ? std::max(1, t.ctas_per_sm * t.block_threads / kSplitThreads) : -1;
    const int64_t nvec = (p.F - p.head) >> 2;
    int g1 = 0, g2 = 0;
    cudaError_t e = persistent_grid(k1, smem1, resident1, nvec, &g1);
    if (e != cudaSuccess) return e;
    e = persistent_grid(k2, grp, -1, int64_t(1) << 40, &g2);
    if (e != cudaSuccess) return e;

    SP d{};
    d.t_split = t.split_keys;
    d.bshift = bshift;
    d.B = B;
    d.grid = g1;
    // Deferred rows beyond about half the column are resolved in pass 1 (if
    // more than half the rows miss, splitting them off no longer pays): each
    // CTA owns (F / 2) / grid entries plus one stage.  A numbered flush holds
    // at least kFlushAt rows except a CTA's last.
    const uint64_t region = uint64_t(p.F) / 2 / uint64_t(g1) + kStage;
    d.region = (uint32_t)region;
    d.max_flush = (uint32_t)(region / kFlushAt + 1);
    const size_t nfl = size_t(g1) * d.max_flush;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t off_nf = 256, off_fb = off_nf + up(size_t(g1) * 4), off_runs = off_fb + up(nfl * 4);
    const size_t off_miss = off_runs + up(nfl * size_t(B) * 4);
    const size_t bytes = off_miss + size_t(region) * g1 * 8;
    char *w = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void **>(&w), bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return cudaSuccess;
    }
    d.ctr = reinterpret_cast<uint32_t *>(w);
    d.nflush = reinterpret_cast<uint32_t *>(w + off_nf);
    d.fbase = reinterpret_cast<uint32_t *>(w + off_fb);
    d.runs = reinterpret_cast<uint32_t *>(w + off_runs);
    d.miss = reinterpret_cast<int2 *>(w + off_miss);
    *ran = true;
    e = cudaMemsetAsync(d.ctr, 0, 16, st);
    if (e == cudaSuccess) {
        k1<<<(unsigned)g1, kSplitThreads, smem1, st>>>(p, d);
        k2<<<(unsigned)g2, kSplitThreads, grp, st>>>(p, d);
        note_launches(2);
        e = cudaGetLastError();
    }
    cudaFreeAsync(w, st);
    return e;
}

template <int AGG, int PATH>
cudaError_t run_split_g(const PP &p, bool gsmem, const skx_tuning &t, int32_t bshift, int32_t B, cudaStream_t st,
                        bool *ran) {
    if (AGG == SKX_AGG_GROUPBY_SUM && gsmem) return run_split<AGG, PATH, true>(p, t, bshift, B, st, ran);
    return run_split<AGG, PATH, false>(p, t, bshift, B, st, ran);
}

template <int AGG>
cudaError_t run_split_p(const PP &p, int path, bool gsmem, const skx_tuning &t, int32_t bshift, int32_t B,
                        cudaStream_t st, bool *ran) {
    if (path == kRow16) return run_split_g<AGG, kRow16>(p, gsmem, t, bshift, B, st, ran);
    if (path == kRow8) return run_split_g<AGG, kRow8>(p, gsmem, t, bshift, B, st, ran);
    return run_split_g<AGG, kRowGeneric>(p, gsmem, t, bshift, B, st, ran);
}

}  // namespace

int32_t split_buckets(int32_t N, int32_t t_split, int32_t *bshift) {
    int32_t sh = *bshift;
    int64_t b = ((int64_t(N) - t_split) + (int64_t(1) << sh) - 1) >> sh;
    while (b > kMaxBuckets) {
        ++sh;
        b = ((int64_t(N) - t_split) + (int64_t(1) << sh) - 1) >> sh;
    }
    *bshift = sh;
    return (int32_t)b;
}

cudaError_t launch_probe_split(const PP &p, int agg, int path, bool gsmem, const skx_tuning &t, cudaStream_t st,
                               bool *ran) {
    *ran = false;
    if (t.split_keys <= 0 || t.split_keys >= p.N || t.split_keys < p.t_hot) return cudaSuccess;
    int32_t bshift = t.split_bucket;
    const int32_t B = split_buckets(p.N, t.split_keys, &bshift);
    switch (agg) {
        case SKX_AGG_COUNT: return run_split_p<SKX_AGG_COUNT>(p, path, gsmem, t, bshift, B, st, ran);
        case SKX_AGG_SUM: return run_split_p<SKX_AGG_SUM>(p, path, gsmem, t, bshift, B, st, ran);
        default: return run_split_p<SKX_AGG_GROUPBY_SUM>(p, path, gsmem, t, bshift, B, st, ran);
    }
}

}  // namespace skx
