// sort.cu -- order the dimension ids by decreasing frequency (Section III:
// the offset representation lists the values "in decreasing frequency
// order"; Section III-A: the sort runs over the small dimension domain), and
// derive the rank representation (rank[perm[r]] = r) in the same pass.
//
// GB300 design: a stable least-significant-digit radix sort whose key is the
// count and whose payload is the id.  The ids enter in ascending order, so
// stability alone breaks ties by ascending id -- the id never has to be part
// of the key.  A count is at most F, so only ceil(log2(F+1)) key bits are
// sorted (8 bits per pass); descending order comes from sorting ~count.
// Each pass is upsweep (per-tile digit counts) -> exclusive scan of the
// digit-major count matrix -> downsweep (stable scatter).  Stability inside
// a tile comes from processing each warp's 512 keys in 32-key rounds in
// order, ranking equal digits with __match_any_sync.  The final pass writes
// perm[pos] = id and rank[id] = pos directly.
#include "skx_internal.cuh"

namespace skx {
namespace {

constexpr int kBits = 8;
constexpr int kBins = 1 << kBits;
constexpr int kSortBlock = 256;            // 8 warps
constexpr int kWarps = kSortBlock / 32;
constexpr int kRounds = 16;                // 32-key rounds per warp
constexpr int kTile = kSortBlock * kRounds;  // 4096 keys per tile
constexpr int kScanItems = 16;
constexpr int kScanTile = kSortBlock * kScanItems;  // 4096

__device__ __forceinline__ uint32_t first_key(const uint32_t *cnt, uint32_t i) { return ~cnt[i]; }

// ------------------------------------------------------------------ upsweep
template <bool FIRST>
__global__ void __launch_bounds__(kSortBlock)
    k_radix_upsweep(const uint32_t *__restrict__ keys, uint32_t n, int shift, uint32_t *__restrict__ tile_hist,
                    uint32_t num_tiles) {
    __shared__ uint32_t s_cnt[kWarps][kBins];
    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    for (int i = threadIdx.x; i < kWarps * kBins; i += kSortBlock) (&s_cnt[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = blockIdx.x;
    const uint32_t base = tile * kTile + warp * (32 * kRounds);
#pragma unroll 4
    for (int r = 0; r < kRounds; ++r) {
        const uint32_t i = base + r * 32 + lane;
        const bool valid = i < n;
        uint32_t d = kBins;  // sentinel for lanes past the end
        if (valid) d = ((FIRST ? first_key(keys, i) : keys[i]) >> shift) & (kBins - 1);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && lane == (unsigned)(__ffs(peers) - 1)) s_cnt[warp][d] += __popc(peers);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += kSortBlock) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += s_cnt[w][d];
        tile_hist[(size_t)d * num_tiles + tile] = s;
    }
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
                                                           uint32_t *__restrict__ block_sums) {
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

__global__ void __launch_bounds__(1024) k_scan_single(uint32_t *__restrict__ data, uint32_t L) {
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
                                                          const uint32_t *__restrict__ block_sums) {
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

cudaError_t exclusive_scan(uint32_t *d_data, uint32_t L, uint32_t *d_block_sums, cudaStream_t st) {
    const uint32_t nb = (L + kScanTile - 1) / kScanTile;
    k_scan_reduce<<<nb, kSortBlock, 0, st>>>(d_data, L, d_block_sums);
    k_scan_single<<<1, 1024, 0, st>>>(d_block_sums, nb);
    k_scan_apply<<<nb, kSortBlock, 0, st>>>(d_data, L, d_block_sums);
    note_launches(3);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ downsweep
template <bool FIRST, bool LAST>
__global__ void __launch_bounds__(kSortBlock)
    k_radix_downsweep(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, uint32_t n,
                      int shift, const uint32_t *__restrict__ tile_off, uint32_t num_tiles,
                      uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, int32_t *__restrict__ rank_out) {
    __shared__ uint32_t s_cnt[kWarps][kBins];
    __shared__ uint32_t s_base[kBins];
    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    for (int i = threadIdx.x; i < kWarps * kBins; i += kSortBlock) (&s_cnt[0][0])[i] = 0;
    const uint32_t tile = blockIdx.x;
    for (int d = threadIdx.x; d < kBins; d += kSortBlock) s_base[d] = tile_off[(size_t)d * num_tiles + tile];
    __syncthreads();

    const uint32_t base = tile * kTile + warp * (32 * kRounds);
    uint32_t key[kRounds], val[kRounds], loc[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const uint32_t i = base + r * 32 + lane;
        const bool valid = i < n;
        key[r] = 0;
        val[r] = i;
        uint32_t d = kBins;
        if (valid) {
            key[r] = FIRST ? first_key(keys_in, i) : keys_in[i];
            if (!FIRST) val[r] = vals_in[i];
            d = (key[r] >> shift) & (kBins - 1);
        }
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
            // pos < n and val < n hold when the scan is consistent; the checks keep a
            // defect from ever turning into an out-of-bounds store
            if (pos >= n || val[r] >= n) continue;
            if (LAST) {
                vals_out[pos] = val[r];
                rank_out[val[r]] = (int32_t)pos;
            } else {
                keys_out[pos] = key[r];
                vals_out[pos] = val[r];
            }
        }
    }
}

__global__ void k_identity_perm(int32_t *__restrict__ perm, int32_t *__restrict__ rank, int32_t N) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
        perm[i] = (int32_t)i;
        rank[i] = (int32_t)i;
    }
}

int key_bits(int64_t F) {
    int b = 0;
    while (b < 63 && (int64_t(1) << b) <= F) ++b;  // smallest b with F < 2^b
    return b;
}

struct SortLayout {
    uint32_t num_tiles, L, nblk;
    size_t off_ka, off_va, off_kb, off_vb, off_hist, off_bsum, total;
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
    s.total = o;
    return s;
}

}  // namespace

size_t sort_scratch_bytes(int32_t N, int64_t F) {
    (void)F;
    return N > 0 ? sort_layout(N).total : 0;
}

cudaError_t launch_sort_by_count(const uint32_t *d_cnt, int32_t N, int64_t F, int32_t *d_perm, int32_t *d_rank,
                                 void *d_scratch, size_t scratch_bytes, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const int bits = key_bits(F);
    const int passes = (bits + kBits - 1) / kBits;
    if (passes == 0) {
        const int sms = device_sm_count();
        k_identity_perm<<<sms * 4, 256, 0, st>>>(d_perm, d_rank, N);
        note_launches(1);
        return cudaGetLastError();
    }
    const SortLayout s = sort_layout(N);
    if (scratch_bytes < s.total || d_scratch == nullptr) return cudaErrorInvalidValue;
    char *w = static_cast<char *>(d_scratch);
    uint32_t *ka = reinterpret_cast<uint32_t *>(w + s.off_ka), *va = reinterpret_cast<uint32_t *>(w + s.off_va);
    uint32_t *kb = reinterpret_cast<uint32_t *>(w + s.off_kb), *vb = reinterpret_cast<uint32_t *>(w + s.off_vb);
    uint32_t *hist = reinterpret_cast<uint32_t *>(w + s.off_hist);
    uint32_t *bsum = reinterpret_cast<uint32_t *>(w + s.off_bsum);
    const uint32_t n = (uint32_t)N;

    const uint32_t *kin = d_cnt, *vin = nullptr;
    uint32_t *kout = ka, *vout = va;
    for (int p = 0; p < passes; ++p) {
        const int shift = p * kBits;
        const bool first = p == 0, last = p == passes - 1;
        if (first)
            k_radix_upsweep<true><<<s.num_tiles, kSortBlock, 0, st>>>(kin, n, shift, hist, s.num_tiles);
        else
            k_radix_upsweep<false><<<s.num_tiles, kSortBlock, 0, st>>>(kin, n, shift, hist, s.num_tiles);
        cudaError_t e = exclusive_scan(hist, s.L, bsum, st);
        if (e != cudaSuccess) return e;
        uint32_t *perm_u = reinterpret_cast<uint32_t *>(d_perm);
        if (first && last)
            k_radix_downsweep<true, true><<<s.num_tiles, kSortBlock, 0, st>>>(kin, vin, n, shift, hist, s.num_tiles,
                                                                              nullptr, perm_u, d_rank);
        else if (first)
            k_radix_downsweep<true, false><<<s.num_tiles, kSortBlock, 0, st>>>(kin, vin, n, shift, hist, s.num_tiles,
                                                                               kout, vout, nullptr);
        else if (last)
            k_radix_downsweep<false, true><<<s.num_tiles, kSortBlock, 0, st>>>(kin, vin, n, shift, hist, s.num_tiles,
                                                                               nullptr, perm_u, d_rank);
        else
            k_radix_downsweep<false, false><<<s.num_tiles, kSortBlock, 0, st>>>(kin, vin, n, shift, hist,
                                                                                s.num_tiles, kout, vout, nullptr);
        note_launches(2);  // upsweep + downsweep
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        // ping-pong
        kin = kout;
        vin = vout;
        if (kout == ka) {
            kout = kb;
            vout = vb;
        } else {
            kout = ka;
            vout = va;
        }
    }
    return cudaSuccess;
}

}  // namespace skx
