// histogram_part.cu -- the FK count by radix partitioning (the Q3 aggregation
// that starts the index build, Section III-A), for large N and F.
//
// The single-pass count (histogram.cu) sends every key that is not cached in
// its CTA to a random 4-byte counter in L2.  When the counter array is tens
// of MB, the cold half of a Zipf column is hundreds of millions of random L2
// atomics, and the L2 request rate, not HBM, bounds the kernel.  This version
// touches no random global address:
//   A  every CTA owns a contiguous slice of the column and counts its keys
//      per bucket of 2^15 consecutive ids in shared memory -> a bucket-major
//      matrix mat[b][cta] (plus one trailing zero);
//   -  an exclusive scan of the matrix gives each CTA its write position in
//      every bucket (and, at the end, the number of valid keys);
//   C  each CTA (1024 threads, one per SM) re-reads its slice in tiles of
//      16384 keys (16 per thread), groups a tile by bucket in shared memory,
//      and writes the keys' 15-bit offsets in their bucket (2 bytes each) to
//      its region of that bucket, so the part array holds every bucket's keys
//      contiguously; the longer a tile, the longer each bucket's run and the
//      fewer partly written sectors;
//   D  the buckets are cut into even chunks of at most 2^20 keys; a
//      persistent grid takes chunks from an atomic counter and counts a chunk
//      in 2^15 shared-memory counters, then writes them with plain stores (a
//      bucket in one chunk) or adds them with atomics (a bucket split over
//      several chunks).
// Same-address shared atomics serialise, and a bucket can hold most of a
// tile when the column is very skewed.  So in phases A and C each warp
// samples 32 keys of its tile, and when one bucket fills at least 12 of them
// the warp counts or ranks that bucket's keys in registers with one atomic
// per warp.  Phase D has no such path: its shared-memory adds return no
// value, and measured over Zipf s = 0 .. 2 and an all-equal column the
// plain adds were never slower than the register path.
// HBM traffic: the column twice (A, C), 2 bytes per key written (C) and read
// (D), the counters written once.  Whether this count or the single pass
// runs is decided on the device from a sample of the keys (k_count_choose).
//
// Sampled layout (up to 1024 buckets, the usual case): phase A and its scan
// are replaced by a plan from 65536 keys at an even stride (k_part_sample,
// k_part_plan).  Each bucket gets a region of the part array sized from its
// sample count with six standard deviations of slack, and C claims each
// tile's run in a bucket with one global atomic on the bucket's cursor.  Runs
// of different CTAs then interleave within a region, which D does not mind.
// If a bucket outgrows its region (a column whose even-stride sample
// misleads), C writes that run to a spare tile past the regions and raises a
// flag on which the exact layout (A, scan, C, D) recounts everything; its
// kernels are enqueued behind and return at once otherwise.  The column is
// then read once by C instead of twice.
#include <algorithm>

#include "skx_internal.cuh"

namespace skx {
namespace {

constexpr int kBktLog = 15;
constexpr uint32_t kBkt = 1u << kBktLog;   // ids per bucket
constexpr int kMaxBuckets = 8192;          // so N <= 2^28
constexpr int kPBlock = 1024;              // threads of phases A and C
constexpr int kTileVec = 4096;             // 16-byte vectors per phase-C tile
constexpr int kTileKeys = kTileVec * 4;    // 16384 keys
constexpr int kVecPT = kTileVec / kPBlock; // vectors per thread per tile
constexpr int kDBlock = 1024;              // threads of phase D
constexpr int kDUnroll = 4;                // 16-byte vectors per thread per phase-D step
constexpr uint64_t kChunk = uint64_t(1) << 20;
constexpr int kPlanSample = 65536;                // keys sampled to size the regions of the sampled layout
constexpr int kPlanCtas = kPlanSample / kPBlock;  // one sampled key per thread
constexpr int kSampledMaxB = kPBlock;             // sampled layout: C's thread b owns bucket b

struct Slices {
    const int32_t *fk;
    int64_t F, head, nvec, per_cta;  // head: keys before the first 16-byte boundary
    int32_t N, B;
    uint32_t trash;  // sampled layout: first of kTileKeys spare slots past the P slots of part
};

// bucket of a key; invalid slots and keys outside [0, N) go to the spare bucket B
__device__ __forceinline__ uint32_t bucket_of(int32_t k, bool ok, const Slices &s, bool &bad) {
    const bool in = (uint32_t)k < (uint32_t)s.N;
    bad |= ok && !in;
    return (ok && in) ? ((uint32_t)k >> kBktLog) : (uint32_t)s.B;
}

// index of the CTA-0 key handled outside the vector loop by thread t (< 8), or -1:
// threads 0..3 take the unaligned head, threads 4..7 the ragged tail.
__device__ __forceinline__ int64_t extra_index(const Slices &s, int t) {
    if (t < s.head) return t;
    const int64_t tail0 = s.head + (s.nvec << 2);
    if (t >= 4 && t < 8 && tail0 + (t - 4) < s.F) return tail0 + (t - 4);
    return -1;
}

// The most frequent of the warp's 32 values v (ties: the lowest lane's) in
// the low 27 bits, its multiplicity (1..32) in the high 5 bits minus one.
constexpr int kDominant = 12;  // a sampled value this frequent takes the register path
__device__ __forceinline__ uint32_t warp_mode(uint32_t v, uint32_t &mult) {
    const unsigned m = __match_any_sync(~0u, v);
    const uint32_t best = __reduce_max_sync(~0u, ((uint32_t)__popc(m) << 5) | (31u - lane_id()));
    mult = best >> 5;
    return __shfl_sync(~0u, v, 31 - (int)(best & 31u));
}

// bucket of a key (B when it lies outside [0, N))
__device__ __forceinline__ uint32_t bucket(int32_t k, const Slices &s) {
    return (uint32_t)k < (uint32_t)s.N ? ((uint32_t)k >> kBktLog) : (uint32_t)s.B;
}

// Exclusive scan of in[0, n) into out[0, n) by a block of NT threads; each
// thread owns a run of consecutive elements and calls each(i, excl) for its
// own after the scan.  Returns the total.  s_w holds 33 words.  Ends with a
// barrier.
template <int NT, typename Each>
__device__ uint32_t block_scan(const uint32_t *in, uint32_t *out, int n, uint32_t *s_w, Each each) {
    const int per = (n + NT - 1) / NT;
    const int i0 = threadIdx.x * per;
    uint32_t loc = 0;
    for (int j = 0; j < per; ++j)
        if (i0 + j < n) loc += in[i0 + j];
    uint32_t x = loc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(~0u, x, d);
        if ((int)lane_id() >= d) x += y;
    }
    const int w = threadIdx.x >> 5;
    if (lane_id() == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        const uint32_t t = lane_id() < NT / 32 ? s_w[lane_id()] : 0u;
        uint32_t inc = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(~0u, inc, d);
            if ((int)lane_id() >= d) inc += y;
        }
        if (lane_id() < NT / 32) s_w[lane_id()] = inc - t;
        if (lane_id() == 31) s_w[32] = inc;
    }
    __syncthreads();
    uint32_t run = s_w[w] + x - loc;
    for (int j = 0; j < per; ++j) {
        if (i0 + j < n) {
            const uint32_t v = in[i0 + j];
            out[i0 + j] = run;
            each(i0 + j, run);
            run += v;
        }
    }
    const uint32_t total = s_w[32];
    __syncthreads();
    return total;
}

// ---------------------------------------------------------------- phase A
__global__ void __launch_bounds__(kPBlock)
    k_part_count(Slices s, uint32_t *__restrict__ mat, uint32_t *__restrict__ queue, unsigned *err,
                 const uint32_t *run) {
    if (run && !*run) return;  // the single pass was chosen on the device
    extern __shared__ uint32_t s_h[];  // [B + 1]; [B] takes padding slots and keys outside [0, N)
    for (int b = threadIdx.x; b <= s.B; b += kPBlock) s_h[b] = 0;
    __syncthreads();
    const uint64_t pol = policy_evict_first();
    const int4 *vec = reinterpret_cast<const int4 *>(s.fk + s.head);
    const int64_t v0 = int64_t(blockIdx.x) * s.per_cta;
    const int64_t v1 = min(v0 + s.per_cta, s.nvec);
    for (int64_t t = v0; t < v1; t += kTileVec) {  // uniform over the block
        int4 k[kVecPT];
#pragma unroll
        for (int j = 0; j < kVecPT; ++j) {
            const int64_t v = t + j * kPBlock + threadIdx.x;
            k[j] = v < v1 ? ld_stream16(vec + v, pol) : make_int4(-1, -1, -1, -1);
        }
        // when 32 sampled keys of the warp share a bucket often, the keys of
        // that bucket are counted in a register (uniform branch per warp)
        uint32_t mult;
        const uint32_t hot = warp_mode(bucket(k[0].x, s), mult);
        if (mult >= kDominant) {
            uint32_t hc = 0;
#pragma unroll
            for (int j = 0; j < kVecPT; ++j) {
                const int32_t kk[4] = {k[j].x, k[j].y, k[j].z, k[j].w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t b = bucket(kk[q], s);
                    if (b == hot) ++hc;
                    else atomicAdd(s_h + b, 1u);
                }
            }
            hc = __reduce_add_sync(~0u, hc);
            if (lane_id() == 0) atomicAdd(s_h + hot, hc);
        } else {
#pragma unroll
            for (int j = 0; j < kVecPT; ++j) {
                atomicAdd(s_h + bucket(k[j].x, s), 1u);
                atomicAdd(s_h + bucket(k[j].y, s), 1u);
                atomicAdd(s_h + bucket(k[j].z, s), 1u);
                atomicAdd(s_h + bucket(k[j].w, s), 1u);
            }
        }
    }
    bool bad = false;  // the vector path's invalid keys show in the spare bucket's count
    if (blockIdx.x == 0) {
        const int64_t e = threadIdx.x < 8 ? extra_index(s, threadIdx.x) : -1;
        if (e >= 0) {
            const uint32_t b = bucket_of(s.fk[e], true, s, bad);
            if (b < (uint32_t)s.B) atomicAdd(s_h + b, 1u);
        }
        if (threadIdx.x == 0) {
            mat[size_t(s.B) * gridDim.x] = 0;  // after the scan: the number of valid keys
            *queue = 0;                        // chunk counter of phase D
        }
    }
    __syncthreads();
    // padding slots of the last tile: 4 per vector slot past v1
    const int64_t tiles = v1 > v0 ? (v1 - v0 + kTileVec - 1) / kTileVec : 0;
    const uint32_t pad = (uint32_t)(4 * (tiles * kTileVec - (v1 > v0 ? v1 - v0 : 0)));
    if (threadIdx.x == 0 && s_h[s.B] != pad) bad = true;
    if (bad) raise_error(err, kErrKeyRange);
    for (int b = threadIdx.x; b < s.B; b += kPBlock) mat[size_t(b) * gridDim.x + blockIdx.x] = s_h[b];
}

// ---------------------------------------------------------------- phase C
// Shared memory of phase C, in 32-bit words: two arrays of tile counts per
// bucket (B + 1 each, alternating between tiles), the tile's first slot per
// bucket, the per-bucket write cursor, the tile's global-minus-local offset
// per bucket, and the tile.
__host__ __device__ constexpr size_t scatter_smem_words(int B) {
    return 2 * size_t(B + 1) + 3 * size_t(B) + kTileKeys;
}

// Each tile is grouped by bucket in shared memory, then written in slot
// order: consecutive threads write consecutive positions of one bucket's run.
// SAMPLED: positions come from the bucket cursors (one global atomic per
// bucket and tile, its latency hidden behind the placement), bounded by the
// regions of k_part_plan; keys outside [0, N) are detected here, as phase A
// does in the exact layout.
template <bool SAMPLED>
__global__ void __launch_bounds__(kPBlock, 1)
    k_part_scatter(Slices s, const uint32_t *__restrict__ off, uint16_t *__restrict__ part, const uint32_t *run,
                   const uint32_t *__restrict__ bstart, uint32_t *cursor, uint32_t *exact, unsigned *err) {
    if (run && !*run) return;
    extern __shared__ uint32_t sm[];
    const int B = s.B;
    uint32_t *s_cnt0 = sm;                // [B + 1] keys of even tiles per bucket ([B]: invalid)
    uint32_t *s_cnt1 = s_cnt0 + B + 1;    // [B + 1] odd tiles
    uint32_t *s_start = s_cnt1 + B + 1;   // [B] first slot of each bucket in s_tile
    uint32_t *s_g = s_start + B;          // [B] next global position of this CTA per bucket
                                          //     (SAMPLED: the end of the bucket's region)
    uint32_t *s_delta = s_g + B;          // [B] global position minus tile slot, this tile
    uint32_t *s_tile = s_delta + B;       // [kTileKeys] the tile grouped by bucket
    __shared__ uint32_t s_w[33];
    for (int b = threadIdx.x; b <= B; b += kPBlock) {
        s_cnt0[b] = 0;
        s_cnt1[b] = 0;
        if (b < B) s_g[b] = SAMPLED ? bstart[b + 1] : off[size_t(b) * gridDim.x + blockIdx.x];
    }
    __syncthreads();
    bool overflow = false;
    uint32_t spare = 0;  // SAMPLED: keys of the spare bucket (padding slots and invalid keys)
    const uint64_t pol = policy_evict_first();
    const int4 *vec = reinterpret_cast<const int4 *>(s.fk + s.head);
    const int64_t v0 = int64_t(blockIdx.x) * s.per_cta;
    const int64_t v1 = min(v0 + s.per_cta, s.nvec);
    int par = 0;
    // keys of the next tile are loaded while the current one is written out
    int4 k[kVecPT];
#pragma unroll
    for (int j = 0; j < kVecPT; ++j) {
        const int64_t v = v0 + j * kPBlock + threadIdx.x;
        k[j] = v < v1 ? ld_stream16(vec + v, pol) : make_int4(-1, -1, -1, -1);
    }
    for (int64_t t = v0; t < v1; t += kTileVec, par ^= 1) {
        uint32_t *cnt = par ? s_cnt1 : s_cnt0;
        uint32_t *cnt_next = par ? s_cnt0 : s_cnt1;
        uint32_t bk[kVecPT * 4];  // bucket (B: none) | offset << 16
#pragma unroll
        for (int j = 0; j < kVecPT; ++j) {
            const int32_t kk[4] = {k[j].x, k[j].y, k[j].z, k[j].w};
#pragma unroll
            for (int q = 0; q < 4; ++q) bk[4 * j + q] = bucket(kk[q], s) | (((uint32_t)kk[q] & (kBkt - 1)) << 16);
        }
        // rank of each key within its bucket in this tile; when the warp's
        // sampled keys share a bucket often, that bucket is ranked with one
        // atomic per warp (uniform branch per warp)
        uint32_t r[kVecPT * 2];  // two 16-bit ranks per word (a rank is < kTileKeys)
        uint32_t mult;
        const uint32_t hot = warp_mode(bk[0] & 0xFFFFu, mult);
        if (mult >= kDominant) {
            uint32_t nh = 0, hmask = 0;
#pragma unroll
            for (int q = 0; q < kVecPT * 4; ++q) {
                const uint32_t b = bk[q] & 0xFFFFu;
                uint32_t rq;
                if (b == hot) {
                    rq = nh++;
                    hmask |= 1u << q;
                } else {
                    rq = atomicAdd(cnt + b, 1u);
                }
                if (q & 1) r[q >> 1] |= rq << 16;
                else r[q >> 1] = rq;
            }
            uint32_t incl = nh;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(~0u, incl, d);
                if ((int)lane_id() >= d) incl += y;
            }
            const uint32_t wtot = __shfl_sync(~0u, incl, 31);
            uint32_t hbase = 0;
            if (lane_id() == 0) hbase = atomicAdd(cnt + hot, wtot);
            hbase = __shfl_sync(~0u, hbase, 0) + incl - nh;
#pragma unroll
            for (int q = 0; q < kVecPT * 4; ++q)
                if (hmask & (1u << q)) r[q >> 1] += hbase << ((q & 1) * 16);
        } else {
#pragma unroll
            for (int q = 0; q < kVecPT * 4; q += 2)
                r[q >> 1] = atomicAdd(cnt + (bk[q] & 0xFFFFu), 1u) | (atomicAdd(cnt + (bk[q + 1] & 0xFFFFu), 1u) << 16);
        }
        __syncthreads();
        // tile layout; each bucket's global offset for this tile; advance the
        // cursors; clear the other count array for the next tile
        uint32_t my_g = 0, my_n = 0, my_excl = 0;  // SAMPLED: bucket threadIdx.x of this tile
        const uint32_t n = block_scan<kPBlock>(cnt, s_start, B, s_w, [&](int b, uint32_t excl) {
            if (SAMPLED) {
                my_n = cnt[b];
                my_excl = excl;
                if (my_n) my_g = atomicAdd(cursor + b, my_n);
            } else {
                const uint32_t g = s_g[b];
                s_delta[b] = g - excl;
                s_g[b] = g + cnt[b];
            }
            cnt_next[b] = 0;
        });
        if (threadIdx.x == 0) {
            if (SAMPLED) spare += cnt[B];
            cnt_next[B] = 0;
        }
#pragma unroll
        for (int q = 0; q < kVecPT * 4; ++q) {
            const uint32_t b = bk[q] & 0xFFFFu;
            if (b < (uint32_t)B) s_tile[s_start[b] + ((r[q >> 1] >> ((q & 1) * 16)) & 0xFFFFu)] = bk[q];
        }
        if (SAMPLED && my_n) {  // thread b owns bucket b (B <= kPBlock)
            // a run that does not fit its region goes to the spare tile past the P slots
            const bool fits = my_g <= s_g[threadIdx.x] && my_n <= s_g[threadIdx.x] - my_g;
            s_delta[threadIdx.x] = (fits ? my_g : s.trash) - my_excl;
            overflow |= !fits;
        }
#pragma unroll
        for (int j = 0; j < kVecPT; ++j) {
            const int64_t v = t + kTileVec + j * kPBlock + threadIdx.x;
            k[j] = v < v1 ? ld_stream16(vec + v, pol) : make_int4(-1, -1, -1, -1);
        }
        __syncthreads();
#pragma unroll 4
        for (uint32_t i = threadIdx.x; i < n; i += kPBlock) {
            const uint32_t x = s_tile[i];
            part[s_delta[x & 0xFFFFu] + i] = (uint16_t)(x >> 16);
        }
        // the next tile's first barrier also orders this write-out before its placement
    }
    __syncthreads();
    bool bad = false;
    if (blockIdx.x == 0 && threadIdx.x < 8) {
        const int64_t e = extra_index(s, threadIdx.x);
        if (e >= 0) {
            const int32_t k = s.fk[e];
            const uint32_t b = bucket(k, s);
            if (b < (uint32_t)B) {
                if (SAMPLED) {
                    const uint32_t pos = atomicAdd(cursor + b, 1u);
                    if (pos < s_g[b]) part[pos] = (uint16_t)((uint32_t)k & (kBkt - 1));
                    else overflow = true;
                } else {
                    part[atomicAdd(s_g + b, 1u)] = (uint16_t)((uint32_t)k & (kBkt - 1));
                }
            } else if (SAMPLED) {
                bad = true;
            }
        }
    }
    if (SAMPLED) {
        if (overflow) *exact = 1u;
        if (threadIdx.x == 0) {  // padding slots of the last tile: 4 per vector slot past v1
            const int64_t tiles = v1 > v0 ? (v1 - v0 + kTileVec - 1) / kTileVec : 0;
            const uint32_t pad = (uint32_t)(4 * (tiles * kTileVec - (v1 > v0 ? v1 - v0 : 0)));
            if (spare != pad) bad = true;
        }
        if (bad) raise_error(err, kErrKeyRange);
    }
}

// ---------------------------------------------------------------- phase D
// Bucket b's keys are part[starts[b * ss], ends[b * es]): the scanned matrix
// (ss = es = G, ends = starts + G) or the sampled layout's region starts and
// cursors (ss = es = 1).  Runs iff *run (when given) and not *skip.
__global__ void __launch_bounds__(kDBlock, 1)
    k_part_hist(const uint16_t *__restrict__ part, const uint32_t *__restrict__ starts, int32_t ss,
                const uint32_t *__restrict__ ends, int32_t es, int32_t B, int32_t N, uint32_t *queue,
                uint32_t *__restrict__ cnt, const uint32_t *run, const uint32_t *skip) {
    if ((run && !*run) || (skip && *skip)) return;
    extern __shared__ uint32_t sm[];
    uint32_t *s_c = sm;          // [kBkt] counters of the current chunk
    uint32_t *s_cs = sm + kBkt;  // [B + 1] first chunk of each bucket
    __shared__ uint32_t s_w[33];
    __shared__ uint32_t s_t;
    __shared__ int32_t s_b;
    for (int b = threadIdx.x; b < B; b += kDBlock) {
        const uint64_t n = ends[size_t(b) * es] - starts[size_t(b) * ss];
        s_cs[b] = (uint32_t)((n + kChunk - 1) / kChunk);
    }
    __syncthreads();
    const uint32_t total = block_scan<kDBlock>(s_cs, s_cs, B, s_w, [](int, uint32_t) {});
    if (threadIdx.x == 0) s_cs[B] = total;
    __syncthreads();
    const uint64_t pol = policy_evict_first();
    while (true) {
        if (threadIdx.x == 0) {
            const uint32_t t = atomicAdd(queue, 1u);
            s_t = t;
            if (t < total) {  // last bucket whose first chunk is <= t
                int lo = 0, hi = B - 1;
                while (lo < hi) {
                    const int mid = lo + ((hi - lo + 1) >> 1);
                    if (s_cs[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                s_b = lo;
            }
        }
        for (uint32_t i = threadIdx.x; i < kBkt; i += kDBlock) s_c[i] = 0;
        __syncthreads();
        const uint32_t t = s_t;
        if (t >= total) break;
        const int32_t b = s_b;
        const uint32_t j = t - s_cs[b], nc = s_cs[b + 1] - s_cs[b];
        const uint64_t b0 = starts[size_t(b) * ss];
        const uint64_t n = ends[size_t(b) * es] - b0;
        const uint64_t lo = b0 + n * j / nc, hi = b0 + n * (j + 1) / nc;
        uint64_t a0 = (lo + 7) & ~uint64_t(7);
        if (a0 > hi) a0 = hi;
        const uint64_t a1 = a0 + ((hi - a0) & ~uint64_t(7));
        for (uint64_t i = lo + threadIdx.x; i < a0; i += kDBlock) atomicAdd(s_c + part[i], 1u);
        for (uint64_t i = a1 + threadIdx.x; i < hi; i += kDBlock) atomicAdd(s_c + part[i], 1u);
        const int4 *p4 = reinterpret_cast<const int4 *>(part + a0);
        const uint64_t n4 = (a1 - a0) >> 3;
        for (uint64_t vb = threadIdx.x; vb < n4; vb += uint64_t(kDBlock) * kDUnroll) {
            int4 x[kDUnroll];
            bool ok[kDUnroll];
#pragma unroll
            for (int u = 0; u < kDUnroll; ++u) {
                const uint64_t v = vb + uint64_t(u) * kDBlock;
                ok[u] = v < n4;
                x[u] = ok[u] ? ld_stream16(p4 + v, pol) : make_int4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < kDUnroll; ++u) {
                if (!ok[u]) continue;
                const uint32_t w[4] = {(uint32_t)x[u].x, (uint32_t)x[u].y, (uint32_t)x[u].z, (uint32_t)x[u].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    atomicAdd(s_c + (w[e] & 0xFFFFu), 1u);
                    atomicAdd(s_c + (w[e] >> 16), 1u);
                }
            }
        }
        __syncthreads();
        const uint32_t base = (uint32_t)b << kBktLog;
        const uint32_t lim = min(kBkt, (uint32_t)N - base);
        if (nc == 1) {
            for (uint32_t i = threadIdx.x; i < lim; i += kDBlock) cnt[base + i] = s_c[i];
        } else {
            for (uint32_t i = threadIdx.x; i < lim; i += kDBlock) {
                const uint32_t c = s_c[i];
                if (c) atomicAdd(cnt + base + i, c);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- choice
// Which count to run, from kSample keys taken at an even stride: the share of
// sampled keys whose id occurs at least twice in the sample approximates the
// share of the column that the single pass's per-CTA cache of hot ids
// absorbs (ids drawn about once per F / kSample keys or more often).
constexpr int kSample = 8192;
constexpr int kSampleLog = 14;
constexpr int kSampleSlots = 1 << kSampleLog;  // open-addressing table, load <= 1/2
// The choice, from the share d of sampled keys whose id repeats in the sample
// (about the share of the column the single pass's per-CTA cache absorbs):
// d >= kHotPerMille -> the single pass; d < kFlatPerMille -> the partitioned
// count; in between the partitioned count only from kMidSkewMinN ids (below
// them the single pass's counters stay in L2 and it is faster), and with the
// exact layout (more than 1024 buckets) only while d < kMidExactPerMille.
// Measured at F = 500M over N = 1M..60M and Zipf s = 0.8..1.7, this picks the
// faster count at every point (for example N = 20M: d = 781 (s = 1.2)
// partitioned 1.57 ms against 1.80; d = 869 (s = 1.3) single 1.39 against 1.69;
// N = 8M, d = 640 (s = 1.1): single 1.22 against 1.45).
constexpr uint32_t kHotPerMille = 850;
constexpr uint32_t kFlatPerMille = 600;
constexpr uint32_t kMidExactPerMille = 700;
constexpr int32_t kMidSkewMinN = 1 << 24;
constexpr int kChooseBlock = 1024;

__global__ void __launch_bounds__(kChooseBlock)
    k_count_choose(const int32_t *__restrict__ fk, int64_t F, int32_t N, bool sampled, uint32_t *flag) {
    extern __shared__ uint32_t sm[];
    int32_t *s_key = reinterpret_cast<int32_t *>(sm);  // [kSampleSlots], -1 = empty
    uint32_t *s_n = sm + kSampleSlots;                 // [kSampleSlots]
    __shared__ uint32_t s_valid, s_dup;
    for (int i = threadIdx.x; i < kSampleSlots; i += kChooseBlock) {
        s_key[i] = -1;
        s_n[i] = 0;
    }
    if (threadIdx.x == 0) {
        s_valid = 0;
        s_dup = 0;
    }
    __syncthreads();
    const int64_t stride = F / kSample;
    constexpr int kPer = kSample / kChooseBlock;
    int32_t kk[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) kk[j] = fk[int64_t(threadIdx.x + j * kChooseBlock) * stride];
    uint32_t valid = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int32_t k = kk[j];
        if ((uint32_t)k >= (uint32_t)N) continue;
        ++valid;
        uint32_t slot = ((uint32_t)k * 0x9E3779B1u) >> (32 - kSampleLog);
        for (int p = 0; p < kSampleSlots; ++p) {  // the table never fills: this ends
            const int32_t prev = atomicCAS(s_key + slot, -1, k);
            if (prev == -1 || prev == k) {
                atomicAdd(s_n + slot, 1u);
                break;
            }
            slot = (slot + 1) & (kSampleSlots - 1);
        }
    }
    valid = __reduce_add_sync(~0u, valid);
    if (lane_id() == 0) atomicAdd(&s_valid, valid);
    __syncthreads();
    uint32_t dup = 0;
    for (int i = threadIdx.x; i < kSampleSlots; i += kChooseBlock) {
        const uint32_t n = s_n[i];
        if (n >= 2) dup += n;
    }
    dup = __reduce_add_sync(~0u, dup);
    if (lane_id() == 0) atomicAdd(&s_dup, dup);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t d = uint64_t(s_dup) * 1000, v = s_valid;
        const bool heavy = v > 0 && d >= v * kHotPerMille;
        const bool flat = v == 0 || d < v * kFlatPerMille;
        const bool mid = N >= kMidSkewMinN && (sampled || d < v * kMidExactPerMille);
        *flag = heavy ? 0u : ((flat || mid) ? 1u : 0u);
    }
}

// ---------------------------------------------------------------- plan
// Regions of the sampled layout.  kPlanSample keys at an even stride are
// counted per bucket (k_part_sample, spread over kPlanCtas SMs so that their
// loads overlap); with c of the S valid sampled keys in bucket b (c is about
// Binomial(S, p_b)), the region holds ceil(F (c + 6 sqrt(c) + 8) / S) keys.
// flags[0] = run the sampled layout, flags[1] = run the exact one: the exact
// one runs instead when the regions exceed the P slots of the part array or
// no sampled key is valid.  Both kernels run only when the partitioned count
// was chosen (*choose, when given); otherwise both flags are 0.

// kPlanCtas CTAs each count kPBlock sampled keys (key q at q * (F / kPlanSample))
// per bucket into smat[cta][b]; b = B for keys outside [0, N).
__global__ void __launch_bounds__(kPBlock)
    k_part_sample(const int32_t *__restrict__ fk, int64_t F, int32_t N, int32_t B, const uint32_t *choose,
                  uint32_t *__restrict__ smat) {
    __shared__ uint32_t s_c[kSampledMaxB + 1];
    if (choose && !*choose) return;
    for (int b = threadIdx.x; b <= B; b += kPBlock) s_c[b] = 0;
    __syncthreads();
    const int64_t stride = F / kPlanSample;  // >= 1: F >= kPlanSample
    const int32_t k = __ldg(fk + (int64_t(blockIdx.x) * kPBlock + threadIdx.x) * stride);
    atomicAdd(s_c + ((uint32_t)k < (uint32_t)N ? ((uint32_t)k >> kBktLog) : (uint32_t)B), 1u);
    __syncthreads();
    for (int b = threadIdx.x; b <= B; b += kPBlock) smat[size_t(blockIdx.x) * (B + 1) + b] = s_c[b];
}

__global__ void __launch_bounds__(kPBlock)
    k_part_plan(const uint32_t *__restrict__ smat, int64_t F, int32_t B, uint64_t P, const uint32_t *choose,
                uint32_t *__restrict__ bstart, uint32_t *__restrict__ cursor, uint32_t *flags, uint32_t *queue) {
    __shared__ uint32_t s_invalid;
    __shared__ unsigned long long s_w[33];
    if (choose && !*choose) {
        if (threadIdx.x == 0) {
            flags[0] = 0;
            flags[1] = 0;
        }
        return;
    }
    uint32_t c_own = 0;  // sampled keys of bucket threadIdx.x
    if ((int)threadIdx.x < B) {
#pragma unroll 16
        for (int c = 0; c < kPlanCtas; ++c) c_own += smat[size_t(c) * (B + 1) + threadIdx.x];
    }
    if (threadIdx.x < 32) {  // sampled keys outside [0, N): column B
        uint32_t v = 0;
        for (int c = lane_id(); c < kPlanCtas; c += 32) v += smat[size_t(c) * (B + 1) + B];
        v = __reduce_add_sync(~0u, v);
        if (lane_id() == 0) s_invalid = v;
    }
    __syncthreads();
    const uint32_t S = kPlanSample - s_invalid;
    unsigned long long cap = 0;
    if ((int)threadIdx.x < B && S > 0) {
        const double c = c_own;
        const double want = ceil(double(F) * (c + 6.0 * sqrt(c) + 8.0) / double(S));
        cap = want > double(P) ? (unsigned long long)P + 1 : (unsigned long long)want;
    }
    // exclusive 64-bit scan of cap, one bucket per thread
    unsigned long long x = cap;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(~0u, x, d);
        if ((int)lane_id() >= d) x += y;
    }
    const int w = threadIdx.x >> 5;
    if (lane_id() == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        const unsigned long long t = s_w[lane_id()];
        unsigned long long inc = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(~0u, inc, d);
            if ((int)lane_id() >= d) inc += y;
        }
        s_w[lane_id()] = inc - t;
        if (lane_id() == 31) s_w[32] = inc;
    }
    __syncthreads();
    const unsigned long long excl = s_w[w] + x - cap, total = s_w[32];
    const bool ok = S > 0 && total <= P;
    if (ok && (int)threadIdx.x < B) {
        bstart[threadIdx.x] = (uint32_t)excl;
        cursor[threadIdx.x] = (uint32_t)excl;
    }
    if (threadIdx.x == 0) {
        if (ok) bstart[B] = (uint32_t)total;
        flags[0] = ok ? 1u : 0u;
        flags[1] = ok ? 0u : 1u;
        *queue = 0;
    }
}

struct PartLayout {
    int32_t B, G;
    uint32_t L;    // matrix entries + the trailing total
    bool sampled;  // the sampled layout is tried first
    uint64_t P;    // slots of the part array (the sampled layout has kTileKeys spare ones past them)
    size_t off_mat, off_bsum, off_queue, off_flag, off_bstart, off_cursor, off_flags, off_smat, off_part, total;
};

// CTAs of phases A and C: one 1024-thread CTA per SM (phase C holds 64
// registers per thread, the whole register file)
int part_grid(int32_t B) {
    (void)B;
    return device_sm_count();
}

// The sampled layout needs C's one-bucket-per-thread ownership (B <= 1024),
// a full sample (F >= kPlanSample) and 32-bit cursors that cannot wrap: a
// cursor ends at most F past its start, starts are below P = 2F, and the
// spare tile sits at P.
bool sampled_layout(int32_t B, int64_t F) {
    return B <= kSampledMaxB && F >= kPlanSample && 3 * F < (int64_t(1) << 32);
}

PartLayout part_layout(int32_t N, int64_t F) {
    PartLayout p{};
    p.B = (int32_t)((int64_t(N) + kBkt - 1) >> kBktLog);
    p.G = part_grid(p.B);
    p.L = (uint32_t)(size_t(p.B) * p.G + 1);
    p.sampled = sampled_layout(p.B, F);
    p.P = p.sampled ? 2 * uint64_t(F) : uint64_t(F);
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t o = 0;
    p.off_mat = o;
    o = up(o + 4 * size_t(p.L));
    p.off_bsum = o;
    o = up(o + 4 * size_t(exclusive_scan_block_sums(p.L)));
    p.off_queue = o;
    o = up(o + 4);
    p.off_flag = o;
    o = up(o + 4);
    p.off_bstart = o;
    o = up(o + 4 * size_t(kSampledMaxB + 1));
    p.off_cursor = o;
    o = up(o + 4 * size_t(kSampledMaxB));
    p.off_flags = o;
    o = up(o + 8);
    p.off_smat = o;
    o = up(o + 4 * size_t(kPlanCtas) * (kSampledMaxB + 1));
    p.off_part = o;
    o = up(o + 2 * (size_t(p.P) + (p.sampled ? kTileKeys : 0)));
    p.total = o;
    return p;
}

}  // namespace

bool histogram_partitioned_fits(int32_t N, int64_t F) {
    return N >= 1 && ((int64_t(N) + kBkt - 1) >> kBktLog) <= kMaxBuckets && F >= 1 && F < (int64_t(1) << 32);
}

size_t histogram_partitioned_scratch(int32_t N, int64_t F) {
    if (!histogram_partitioned_fits(N, F)) return 0;
    return part_layout(N, F).total;
}

cudaError_t launch_histogram_partitioned(const int32_t *d_fk, int64_t F, int32_t N, uint32_t *d_cnt, unsigned *d_err,
                                         void *d_scratch, size_t scratch_bytes, cudaStream_t st,
                                         const uint32_t *run_if_set) {
    if (F <= 0) return cudaSuccess;
    if (!histogram_partitioned_fits(N, F)) return cudaErrorInvalidValue;
    const PartLayout p = part_layout(N, F);
    const int G = p.G;
    if (!d_scratch || scratch_bytes < p.total || !aligned16(d_scratch)) return cudaErrorInvalidValue;
    char *w = static_cast<char *>(d_scratch);
    uint32_t *mat = reinterpret_cast<uint32_t *>(w + p.off_mat);
    uint32_t *bsum = reinterpret_cast<uint32_t *>(w + p.off_bsum);
    uint32_t *queue = reinterpret_cast<uint32_t *>(w + p.off_queue);
    uint16_t *part = reinterpret_cast<uint16_t *>(w + p.off_part);

    Slices s{};
    s.fk = d_fk;
    s.F = F;
    const int64_t mis = (int64_t)((reinterpret_cast<uintptr_t>(d_fk) & 15u) >> 2);
    s.head = mis ? std::min<int64_t>(F, 4 - mis) : 0;
    s.nvec = (F - s.head) >> 2;
    const int64_t tiles = (s.nvec + kTileVec - 1) / kTileVec;
    s.per_cta = ((tiles + G - 1) / G) * kTileVec;
    s.N = N;
    s.B = p.B;
    s.trash = (uint32_t)p.P;

    const size_t smem_a = size_t(p.B + 1) * 4;
    const size_t smem_c = scatter_smem_words(p.B) * 4;
    const size_t smem_d = (size_t(kBkt) + p.B + 1) * 4;
    cudaError_t e = set_smem_limit_once(reinterpret_cast<const void *>(k_part_count), (kMaxBuckets + 1) * 4);
    if (e == cudaSuccess)
        e = set_smem_limit_once(reinterpret_cast<const void *>(k_part_scatter<false>),
                                (int)(scatter_smem_words(kMaxBuckets) * 4));
    if (e == cudaSuccess)
        e = set_smem_limit_once(reinterpret_cast<const void *>(k_part_scatter<true>),
                                (int)(scatter_smem_words(kSampledMaxB) * 4));
    if (e == cudaSuccess)
        e = set_smem_limit_once(reinterpret_cast<const void *>(k_part_hist), (int)((kBkt + kMaxBuckets + 1) * 4));
    if (e != cudaSuccess) return e;
    const uint32_t *run_exact = run_if_set;
    if (p.sampled) {
        uint32_t *bstart = reinterpret_cast<uint32_t *>(w + p.off_bstart);
        uint32_t *cursor = reinterpret_cast<uint32_t *>(w + p.off_cursor);
        uint32_t *flags = reinterpret_cast<uint32_t *>(w + p.off_flags);
        uint32_t *smat = reinterpret_cast<uint32_t *>(w + p.off_smat);
        k_part_sample<<<kPlanCtas, kPBlock, 0, st>>>(d_fk, F, N, p.B, run_if_set, smat);
        k_part_plan<<<1, kPBlock, 0, st>>>(smat, F, p.B, p.P, run_if_set, bstart, cursor, flags, queue);
        k_part_scatter<true><<<G, kPBlock, smem_c, st>>>(s, nullptr, part, flags, bstart, cursor, flags + 1, d_err);
        k_part_hist<<<device_sm_count(), kDBlock, smem_d, st>>>(part, bstart, 1, cursor, 1, p.B, N, queue, d_cnt,
                                                                flags, flags + 1);
        note_launches(4);
        run_exact = flags + 1;  // set by the plan, or by C when a region overflowed
    }
    k_part_count<<<G, kPBlock, smem_a, st>>>(s, mat, queue, d_err, run_exact);
    e = exclusive_scan_u32(mat, p.L, bsum, st, run_exact);
    if (e != cudaSuccess) return e;
    k_part_scatter<false><<<G, kPBlock, smem_c, st>>>(s, mat, part, run_exact, nullptr, nullptr, nullptr, d_err);
    k_part_hist<<<device_sm_count(), kDBlock, smem_d, st>>>(part, mat, G, mat + G, G, p.B, N, queue, d_cnt,
                                                            run_exact, nullptr);
    note_launches(3);  // the scan counts its own
    return cudaGetLastError();
}

cudaError_t launch_count_choice(const int32_t *d_fk, int64_t F, int32_t N, void *d_scratch, size_t scratch_bytes,
                                const uint32_t **flag, cudaStream_t st) {
    if (!histogram_partitioned_fits(N, F) || F < kSample) return cudaErrorInvalidValue;
    const PartLayout p = part_layout(N, F);
    if (!d_scratch || scratch_bytes < p.total) return cudaErrorInvalidValue;
    uint32_t *f = reinterpret_cast<uint32_t *>(static_cast<char *>(d_scratch) + p.off_flag);
    const cudaError_t e = set_smem_limit_once(reinterpret_cast<const void *>(k_count_choose), kSampleSlots * 8);
    if (e != cudaSuccess) return e;
    k_count_choose<<<1, kChooseBlock, kSampleSlots * 8, st>>>(d_fk, F, N, p.sampled, f);
    note_launches(1);
    *flag = f;
    return cudaGetLastError();
}

}  // namespace skx
