// sort.cu -- order the dimension ids by decreasing frequency (Section III,
// the offset representation; Section III-A: the sort runs over the small
// dimension domain), and derive the rank representation (rank[perm[r]] = r)
// in the same pass.
//
// GB300 design: a stable least-significant-digit radix sort whose key is the
// count and whose payload is the id.  The ids enter in ascending order, so
// stability alone breaks ties by ascending id -- the id never has to be part
// of the key.  A count is at most F, so only ceil(log2(F+1)) key bits are
// sorted (8 bits per pass); descending order comes from sorting ~count.
// Each pass is upsweep (per-tile digit counts) -> exclusive scan of the
// digit-major count matrix -> downsweep (stable scatter).  Stability inside
// a tile comes from processing each warp's 128 keys in 32-key rounds in
// order, ranking equal digits with __match_any_sync.  The final pass writes
// perm[pos] = id and rank[id] = pos directly.
//
// Skewed counts are mostly small: under Zipf most ids occur fewer than 255
// times.  So when the average count F/N is small, one stable pass on the
// clamped digit 255 - min(count, 255) already puts every id with count < 255
// at its final place (written straight to perm and rank), and collects the
// "heavy" ids (count >= 255, at most F/255 of them) in ascending id order at
// the front.  Only that heavy prefix, whose length H is known on the device
// alone, goes through the full multi-pass sort; those kernels read H from
// device memory and their grids are sized for the bound F/255.
#include <algorithm>

#include "skx_internal.cuh"

namespace skx {
namespace {

constexpr int kBits = 8;
constexpr int kBins = 1 << kBits;
constexpr int kSortBlock = 1024;           // 32 warps
constexpr int kWarps = kSortBlock / 32;
constexpr int kRounds = 4;                 // 32-key rounds per warp
constexpr int kTile = kSortBlock * kRounds;  // 4096 keys per tile
constexpr int kScanItems = 4;
constexpr int kScanTile = kSortBlock * kScanItems;  // 4096


// Key sources of a pass.
enum KeySrc {
    kSrcClamped = 0,  // key = 255 - min(cnt[i], 255), id = i     (the heavy/light split pass)
    kSrcCounts = 1,   // key = ~cnt[i], id = i                     (first pass of the plain sort)
    kSrcPairs = 2,    // key = keys_in[i], id = vals_in[i]         (later passes)
    kSrcGather = 3,   // id = vals_in[i], key = ~cnt[id]           (first pass over the heavy ids)
};
// Outputs of a pass.
enum Out {
    kOutPairs = 0,  // keys_out[pos], vals_out[pos]
    kOutFinal = 1,  // perm[pos] = id, rank[id] = pos
    kOutSplit = 2,  // digit 0 (heavy): vals_out[pos] = id; other digits: final
};

template <int SRC>
__device__ __forceinline__ void load_key(const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ keys_in,
                                         const uint32_t *__restrict__ vals_in, uint32_t i, uint32_t &key,
                                         uint32_t &val) {
    if (SRC == kSrcClamped) {
        const uint32_t c = cnt[i];
        key = 255u - (c < 255u ? c : 255u);
        val = i;
    } else if (SRC == kSrcCounts) {
        key = ~cnt[i];
        val = i;
    } else if (SRC == kSrcPairs) {
        key = keys_in[i];
        val = vals_in[i];
    } else {
        val = vals_in[i];
        key = ~cnt[val];
    }
}

// n_dev != null: the element count is read from the device (heavy passes).
template <int SRC>
__global__ void __launch_bounds__(kSortBlock)
    k_radix_upsweep(const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ keys_in,
                    const uint32_t *__restrict__ vals_in, uint32_t n_host, const uint32_t *__restrict__ n_dev,
                    int shift, uint32_t *__restrict__ tile_hist, uint32_t num_tiles, uint32_t cmax,
                    unsigned *err) {
    __shared__ uint32_t s_hist[kBins];  // the tile's digit counts (no order needed here)
    const uint32_t n = n_dev ? *n_dev : n_host;
    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    // a length read from the device that exceeds the grid (more heavy ids than the
    // bound F / 255 allows) would leave ids unsorted: report it
    if (n_dev && blockIdx.x == 0 && threadIdx.x == 0 && n > gridDim.x * kTile) raise_error(err, kErrCountBound);
    const uint32_t tile = blockIdx.x;
    const uint32_t base = tile * kTile + warp * (32 * kRounds);
    const bool live = tile * kTile < n;  // tiles past the end (heavy passes) publish zero counts
    // the keys are loaded first, so that their latency overlaps the histogram's clearing
    uint32_t dig[kRounds];
    bool over = false;
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const uint32_t i = base + r * 32 + lane;
        dig[r] = kBins;  // sentinel for lanes past the end
        if (live && i < n) {
            uint32_t key, val;
            load_key<SRC>(cnt, keys_in, vals_in, i, key, val);
            dig[r] = (key >> shift) & (kBins - 1);
            // the first pass reads every count: one above the bound F would be
            // truncated to the sorted key bits
            if ((SRC == kSrcClamped || SRC == kSrcCounts) && cnt[i] > cmax) over = true;
        }
    }
    for (int i = threadIdx.x; i < kBins; i += kSortBlock) s_hist[i] = 0;
    __syncthreads();
    if (live) {
        if (over) raise_error(err, kErrCountBound);
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            const uint32_t d = dig[r];
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (d < (uint32_t)kBins && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(s_hist + d, __popc(peers));
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += kSortBlock) tile_hist[(size_t)d * num_tiles + tile] = s_hist[d];
}

// ------------------------------------------------------------------ scan
// Exclusive scan of data[L] in place: reduce -> scan of block sums -> apply.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp, uint32_t &total) {
    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (unsigned)(blockDim.x >> 5) ? s_warp[lane] : 0;
        uint32_t z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= (unsigned)o) z += y;
        }
        if (lane < (unsigned)(blockDim.x >> 5)) s_warp[lane] = z - w;
        if (lane == 31) s_warp[32] = z;
    }
    __syncthreads();
    const uint32_t res = s_warp[warp] + x - v;
    total = s_warp[32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(kSortBlock) k_scan_reduce(const uint32_t *__restrict__ data, uint32_t L,
                                                           uint32_t *__restrict__ block_sums, const uint32_t *go) {
    if (go && !*go) return;
    __shared__ uint32_t s_warp[33];
    const uint32_t base = blockIdx.x * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const uint32_t i = base + j * kSortBlock + threadIdx.x;
        if (i < L) s += data[i];
    }
    uint32_t total;
    block_exclusive_scan(s, s_warp, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_single(uint32_t *__restrict__ data, uint32_t L, const uint32_t *go) {
    if (go && !*go) return;
    __shared__ uint32_t s_warp[33];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < L; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < L ? data[i] : 0;
        uint32_t total;
        const uint32_t e = block_exclusive_scan(v, s_warp, total);
        if (i < L) data[i] = carry + e;
        carry += total;
    }
}

__global__ void __launch_bounds__(kSortBlock) k_scan_apply(uint32_t *__restrict__ data, uint32_t L,
                                                          const uint32_t *__restrict__ block_sums, const uint32_t *go) {
    if (go && !*go) return;
    __shared__ uint32_t s_warp[33];
    // thread t owns kScanItems consecutive elements
    const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = (base + j < L) ? data[base + j] : 0;
        s += v[j];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, s_warp, total) + block_sums[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < L) data[base + j] = run;
        run += v[j];
    }
}

cudaError_t exclusive_scan(uint32_t *d_data, uint32_t L, uint32_t *d_block_sums, cudaStream_t st,
                           const uint32_t *go = nullptr) {
    const uint32_t nb = (L + kScanTile - 1) / kScanTile;
    k_scan_reduce<<<nb, kSortBlock, 0, st>>>(d_data, L, d_block_sums, go);
    k_scan_single<<<1, 1024, 0, st>>>(d_block_sums, nb, go);
    k_scan_apply<<<nb, kSortBlock, 0, st>>>(d_data, L, d_block_sums, go);
    note_launches(3);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ downsweep
template <int SRC, int OUT>
__global__ void __launch_bounds__(kSortBlock)
    k_radix_downsweep(const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ keys_in,
                      const uint32_t *__restrict__ vals_in, uint32_t n_host, const uint32_t *__restrict__ n_dev,
                      uint32_t n_all, int shift, const uint32_t *__restrict__ tile_off, uint32_t num_tiles,
                      uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, uint32_t *__restrict__ perm,
                      int32_t *__restrict__ rank_out) {
    __shared__ uint32_t s_cnt[kWarps][kBins];
    __shared__ uint32_t s_base[kBins];
    const uint32_t n = n_dev ? *n_dev : n_host;
    const uint32_t tile = blockIdx.x;
    if (tile * kTile >= n) return;
    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t base = tile * kTile + warp * (32 * kRounds);
    uint32_t key[kRounds], val[kRounds], loc[kRounds];
    // all of the warp's loads first, so their latencies overlap (with each other and with the
    // tile offsets' loads below); then the ranking rounds
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const uint32_t i = base + r * 32 + lane;
        key[r] = 0;
        val[r] = 0;
        if (i < n) load_key<SRC>(cnt, keys_in, vals_in, i, key[r], val[r]);
    }
    for (int i = threadIdx.x; i < kWarps * kBins; i += kSortBlock) (&s_cnt[0][0])[i] = 0;
    for (int d = threadIdx.x; d < kBins; d += kSortBlock) s_base[d] = tile_off[(size_t)d * num_tiles + tile];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const uint32_t i = base + r * 32 + lane;
        const bool valid = i < n;
        const uint32_t d = valid ? ((key[r] >> shift) & (kBins - 1)) : kBins;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (valid && lane == (unsigned)leader) {
            before = s_cnt[warp][d];
            s_cnt[warp][d] = before + __popc(peers);
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        loc[r] = before + __popc(peers & lanemask_lt());
    }
    __syncthreads();
    // exclusive prefix over warps for every digit
    for (int d = threadIdx.x; d < kBins; d += kSortBlock) {
        uint32_t run = s_base[d];
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = s_cnt[w][d];
            s_cnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const uint32_t i = base + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (key[r] >> shift) & (kBins - 1);
            const uint32_t pos = s_cnt[warp][d] + loc[r];
            // pos < n and val < n_all hold when the scan is consistent; the checks keep a
            // defect from ever turning into an out-of-bounds store
            if (pos >= n || val[r] >= n_all) continue;
            if (OUT == kOutFinal || (OUT == kOutSplit && d != 0)) {
                perm[pos] = val[r];
                rank_out[val[r]] = (int32_t)pos;
            } else if (OUT == kOutSplit) {
                vals_out[pos] = val[r];
            } else {
                keys_out[pos] = key[r];
                vals_out[pos] = val[r];
            }
        }
    }
}

// F == 0: every count must be 0 and the order is the identity
__global__ void k_identity_perm(const uint32_t *__restrict__ cnt, int32_t *__restrict__ perm,
                                int32_t *__restrict__ rank, int32_t N, unsigned *err) {
    bool over = false;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
        perm[i] = (int32_t)i;
        rank[i] = (int32_t)i;
        over |= cnt[i] != 0;
    }
    if (over) raise_error(err, kErrCountBound);
}

int key_bits(int64_t F) {
    int b = 0;
    while (b < 63 && (int64_t(1) << b) <= F) ++b;  // smallest b with F < 2^b
    return b;
}

struct SortLayout {
    uint32_t num_tiles, L, nblk;
    size_t off_ka, off_va, off_kb, off_vb, off_hist, off_bsum, off_nh, total;
};

SortLayout sort_layout(int32_t N) {
    SortLayout s{};
    s.num_tiles = (uint32_t)((N + kTile - 1) / kTile);
    s.L = s.num_tiles * kBins;
    s.nblk = (s.L + kScanTile - 1) / kScanTile;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t o = 0;
    s.off_ka = o; o = up(o + 4ull * N);
    s.off_va = o; o = up(o + 4ull * N);
    s.off_kb = o; o = up(o + 4ull * N);
    s.off_vb = o; o = up(o + 4ull * N);
    s.off_hist = o; o = up(o + 4ull * s.L);
    s.off_bsum = o; o = up(o + 4ull * (s.nblk + 1));
    s.off_nh = o; o = up(o + 4ull);
    s.total = o;
    return s;
}

}  // namespace

cudaError_t exclusive_scan_u32(uint32_t *d_data, uint32_t L, uint32_t *d_block_sums, cudaStream_t st,
                               const uint32_t *run_if_set) {
    return exclusive_scan(d_data, L, d_block_sums, st, run_if_set);
}

uint32_t exclusive_scan_block_sums(uint32_t L) { return (L + kScanTile - 1) / kScanTile + 1; }

size_t sort_scratch_bytes(int32_t N, int64_t F) {
    (void)F;
    return N > 0 ? sort_layout(N).total : 0;
}
static_assert(sort_scratch_bound(1) == 2560 && sort_scratch_bound(1 << 20) == 17039872, "scratch bound formula");

namespace {

struct Bufs {
    uint32_t *ka, *va, *kb, *vb, *hist, *bsum, *nh;
    uint32_t cmax;  // bound on every count (F)
    unsigned *err;  // data-error word, or null
};

template <int SRC, int OUT>
cudaError_t radix_pass(const uint32_t *cnt, const uint32_t *kin, const uint32_t *vin, uint32_t n_host,
                       const uint32_t *n_dev, uint32_t n_all, uint32_t tiles, int shift, const Bufs &b,
                       uint32_t *kout, uint32_t *vout, uint32_t *perm, int32_t *rank, cudaStream_t st) {
    const uint32_t L = tiles * kBins;
    k_radix_upsweep<SRC><<<tiles, kSortBlock, 0, st>>>(cnt, kin, vin, n_host, n_dev, shift, b.hist, tiles, b.cmax,
                                                       b.err);
    cudaError_t e = exclusive_scan(b.hist, L, b.bsum, st);
    if (e != cudaSuccess) return e;
    k_radix_downsweep<SRC, OUT><<<tiles, kSortBlock, 0, st>>>(cnt, kin, vin, n_host, n_dev, n_all, shift, b.hist,
                                                              tiles, kout, vout, perm, rank);
    note_launches(2);  // upsweep + downsweep
    return cudaGetLastError();
}

// LSD passes over key bits [0, bits): first pass from SRC_FIRST, last writes perm/rank.
template <int SRC_FIRST>
cudaError_t lsd_sort(const uint32_t *cnt, const uint32_t *ids, uint32_t n_host, const uint32_t *n_dev,
                     uint32_t n_all, uint32_t tiles, int bits, const Bufs &b, uint32_t *perm, int32_t *rank,
                     cudaStream_t st) {
    const int passes = (bits + kBits - 1) / kBits;
    const uint32_t *kin = nullptr, *vin = ids;
    uint32_t *kout = b.ka, *vout = b.va;
    for (int p = 0; p < passes; ++p) {
        const int shift = p * kBits;
        const bool first = p == 0, last = p == passes - 1;
        cudaError_t e;
        if (first && last)
            e = radix_pass<SRC_FIRST, kOutFinal>(cnt, kin, vin, n_host, n_dev, n_all, tiles, shift, b, nullptr,
                                                 nullptr, perm, rank, st);
        else if (first)
            e = radix_pass<SRC_FIRST, kOutPairs>(cnt, kin, vin, n_host, n_dev, n_all, tiles, shift, b, kout, vout,
                                                 nullptr, nullptr, st);
        else if (last)
            e = radix_pass<kSrcPairs, kOutFinal>(cnt, kin, vin, n_host, n_dev, n_all, tiles, shift, b, nullptr,
                                                 nullptr, perm, rank, st);
        else
            e = radix_pass<kSrcPairs, kOutPairs>(cnt, kin, vin, n_host, n_dev, n_all, tiles, shift, b, kout, vout,
                                                 nullptr, nullptr, st);
        if (e != cudaSuccess) return e;
        kin = kout;
        vin = vout;
        if (kout == b.ka) {
            kout = b.kb;
            vout = b.vb;
        } else {
            kout = b.ka;
            vout = b.va;
        }
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_sort_by_count(const uint32_t *d_cnt, int32_t N, int64_t F, int32_t *d_perm, int32_t *d_rank,
                                 void *d_scratch, size_t scratch_bytes, unsigned *d_err, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const int bits = key_bits(F);
    if (bits == 0) {  // F == 0: every count is 0, the order is the identity
        const int sms = device_sm_count();
        k_identity_perm<<<sms * 4, 256, 0, st>>>(d_cnt, d_perm, d_rank, N, d_err);
        note_launches(1);
        return cudaGetLastError();
    }
    const SortLayout s = sort_layout(N);
    if (s.total != sort_scratch_bound(size_t(N))) return cudaErrorInvalidValue;  // layout and bound agree
    if (scratch_bytes < s.total || d_scratch == nullptr) return cudaErrorInvalidValue;
    char *w = static_cast<char *>(d_scratch);
    Bufs b;
    b.ka = reinterpret_cast<uint32_t *>(w + s.off_ka);
    b.va = reinterpret_cast<uint32_t *>(w + s.off_va);
    b.kb = reinterpret_cast<uint32_t *>(w + s.off_kb);
    b.vb = reinterpret_cast<uint32_t *>(w + s.off_vb);
    b.hist = reinterpret_cast<uint32_t *>(w + s.off_hist);
    b.bsum = reinterpret_cast<uint32_t *>(w + s.off_bsum);
    b.nh = reinterpret_cast<uint32_t *>(w + s.off_nh);
    b.cmax = (uint32_t)F;
    b.err = d_err;
    const uint32_t n = (uint32_t)N;
    uint32_t *perm = reinterpret_cast<uint32_t *>(d_perm);

    // heavy/light split when counts are mostly small and more than one pass is needed
    const bool split = bits > kBits && F <= int64_t(64) * N;
    if (!split) return lsd_sort<kSrcCounts>(d_cnt, nullptr, n, nullptr, n, s.num_tiles, bits, b, perm, d_rank, st);

    // pass A: light ids final, heavy ids (digit 0) collected at the front of vb
    cudaError_t e = radix_pass<kSrcClamped, kOutSplit>(d_cnt, nullptr, nullptr, n, nullptr, n, s.num_tiles, 0, b,
                                                       nullptr, b.vb, perm, d_rank, st);
    if (e != cudaSuccess) return e;
    // H = number of heavy ids = scanned offset of (digit 1, tile 0)
    e = cudaMemcpyAsync(b.nh, b.hist + s.num_tiles, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    // heavy ids: at most F / 255 of them
    const int64_t hmax = std::min<int64_t>(N, F / 255 + 1);
    const uint32_t htiles = (uint32_t)((hmax + kTile - 1) / kTile);
    // the heavy ids move from vb into ka/va and back, so pass them in a buffer the
    // ping-pong does not write first: copy to vb is the input, lsd writes ka/va first
    return lsd_sort<kSrcGather>(d_cnt, b.vb, 0, b.nh, n, htiles, bits, b, perm, d_rank, st);
}

}  // namespace skx
