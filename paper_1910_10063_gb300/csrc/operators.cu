// operators.cu -- the other skew-aware operators of the paper over the
// remapped layout:
//
//   heavy-hitter counts (Q3a; Sections I and IV-B): with an up-to-date index
//     the k most frequent values are exactly the transformed ids 0..k-1, so
//     only those are counted and the counters never leave shared memory --
//     the paper's L1-resident output becomes an SM-resident one.  The 32
//     hottest ranks get one counter copy per warp lane (Section IV-B).
//   selection bitmap (Q2 preprocessing; Section I): one bit per dimension
//     row, "col < c", built with a warp ballot per 32 rows.
//   selection (Q2; Sections I and IV-A): the offsets of qualifying fact rows,
//     in increasing order.  GPU analogue of the compressed store
//     (vpcompressd): a warp ballot per 32 fact rows and its population count
//     give each qualifying row its slot; per-tile counts and a scan give each
//     tile its base, so the output order is the fact order.
#include "skx_internal.cuh"

namespace skx {
namespace {

constexpr int kOpBlock = 512;
constexpr int kTopLane = 32;

template <bool SMEM>
__global__ void __launch_bounds__(kOpBlock)
    k_topk(const int32_t *__restrict__ fk, int64_t F, int64_t head, int32_t k, unsigned long long *__restrict__ out) {
    extern __shared__ uint32_t s_top[];  // k counters, then kTopLane x 32 lane copies
    uint32_t *s_lane = s_top + (SMEM ? k : 0);
    const int ns = (SMEM ? k : 0) + kTopLane * 32;
    for (int i = threadIdx.x; i < ns; i += blockDim.x) s_top[i] = 0;
    __syncthreads();
    const uint64_t pol = policy_evict_first();
    const unsigned lane = lane_id();
    auto add = [&](int32_t r) {
        if ((uint32_t)r < (uint32_t)kTopLane && r < k)
            atomicAdd(s_lane + (r << 5) + lane, 1u);
        else if ((uint32_t)r < (uint32_t)k) {
            if (SMEM) atomicAdd(s_top + r, 1u);
            else atomicAdd(out + r, 1ull);
        }
    };
    const int4 *v4 = reinterpret_cast<const int4 *>(fk + head);
    const int64_t nvec = (F - head) >> 2;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, nthr = int64_t(gridDim.x) * blockDim.x;
    int4 nk = make_int4(-1, -1, -1, -1);
    if (tid < nvec) nk = ld_stream16(v4 + tid, pol);
    for (int64_t v = tid; v < nvec; v += nthr) {
        const int4 kk = nk;
        if (v + nthr < nvec) nk = ld_stream16(v4 + v + nthr, pol);
        add(kk.x);
        add(kk.y);
        add(kk.z);
        add(kk.w);
    }
    if (tid < 8) {  // unaligned head and ragged tail
        const int64_t tail0 = head + (nvec << 2);
        int64_t idx = -1;
        if (tid < head) idx = tid;
        else if (tid >= 4 && tail0 + (tid - 4) < F) idx = tail0 + (tid - 4);
        if (idx >= 0) add(fk[idx]);
    }
    __syncthreads();
    const int nflush = SMEM ? k : (k < kTopLane ? k : kTopLane);
    for (int r = threadIdx.x; r < nflush; r += blockDim.x) {
        unsigned long long c = (SMEM && r >= kTopLane) ? s_top[r] : 0;
        if (r < kTopLane) {
            if (SMEM) c += s_top[r];
            for (int l = 0; l < 32; ++l) c += s_lane[(r << 5) + l];
        }
        if (c) atomicAdd(out + r, c);
    }
}

__global__ void __launch_bounds__(kOpBlock)
    k_bitmap(const int32_t *__restrict__ rows, int32_t N, int32_t words, int32_t col, int32_t lt,
             uint32_t *__restrict__ bits) {
    const int64_t nw = (int64_t(N) + 31) >> 5;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const unsigned lane = lane_id();
    for (int64_t w = warp; w < nw; w += nwarps) {
        const int64_t r = (w << 5) + lane;
        const bool pass = r < N && __ldg(rows + r * words + col) < lt;
        const unsigned b = __ballot_sync(0xffffffffu, pass);
        if (lane == 0) bits[w] = b;
    }
}

constexpr int kSelRounds = 16;                         // 32-row rounds per warp
constexpr int kSelTile = kOpBlock * kSelRounds;        // 8192 fact rows per tile

__device__ __forceinline__ bool selected(const int32_t *fk, int64_t i, int64_t F, const uint32_t *bits, int32_t N,
                                         unsigned *err) {
    if (i >= F) return false;
    const int32_t v = fk[i];
    if ((uint32_t)v >= (uint32_t)N) {
        raise_error(err, kErrKeyRange);
        return false;
    }
    return (__ldg(bits + (v >> 5)) >> (v & 31)) & 1u;
}

__global__ void __launch_bounds__(kOpBlock)
    k_select_count(const int32_t *__restrict__ fk, int64_t F, const uint32_t *__restrict__ bits, int32_t N,
                   uint32_t *__restrict__ tile_cnt, unsigned *err) {
    __shared__ uint32_t s_w[kOpBlock / 32];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kSelTile + int64_t(warp) * (32 * kSelRounds);
    uint32_t c = 0;
#pragma unroll 4
    for (int r = 0; r < kSelRounds; ++r) c += __popc(__ballot_sync(0xffffffffu, selected(fk, base + r * 32 + lane, F, bits, N, err)));
    if (lane == 0) s_w[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kOpBlock / 32; ++w) t += s_w[w];
        tile_cnt[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kOpBlock)
    k_select_write(const int32_t *__restrict__ fk, int64_t F, const uint32_t *__restrict__ bits, int32_t N,
                   const uint32_t *__restrict__ tile_off, uint32_t *__restrict__ offsets) {
    __shared__ uint32_t s_w[kOpBlock / 32];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kSelTile + int64_t(warp) * (32 * kSelRounds);
    uint32_t c = 0;
    for (int r = 0; r < kSelRounds; ++r) c += __popc(__ballot_sync(0xffffffffu, selected(fk, base + r * 32 + lane, F, bits, N, nullptr)));
    if (lane == 0) s_w[warp] = c;
    __syncthreads();
    uint32_t before = 0;  // rows selected by the earlier warps of this tile
    for (unsigned w = 0; w < warp; ++w) before += s_w[w];
    uint32_t pos = tile_off[blockIdx.x] + before;
    for (int r = 0; r < kSelRounds; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool p = selected(fk, i, F, bits, N, nullptr);
        const unsigned b = __ballot_sync(0xffffffffu, p);
        if (p) offsets[pos + __popc(b & lanemask_lt())] = (uint32_t)i;
        pos += __popc(b);
    }
}

__global__ void k_select_total(const uint32_t *__restrict__ tile_off, const uint32_t *__restrict__ tile_cnt,
                               uint32_t num_tiles, long long *count) {
    *count = (long long)tile_off[num_tiles - 1] + (long long)tile_cnt[num_tiles - 1];
}

int grid_cap(int64_t items, int per_sm) {
    const int64_t want = (items + kOpBlock - 1) / kOpBlock;
    const int64_t cap = int64_t(device_sm_count()) * per_sm;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace
}  // namespace skx

using namespace skx;

extern "C" {

skx_status skx_topk_counts(const int32_t *d_fk, int64_t F, int32_t k, int64_t *d_out, void *stream) {
    if (F < 0 || F >= (int64_t(1) << 32) || k < 1 || !d_out || (F > 0 && !d_fk) || (reinterpret_cast<uintptr_t>(d_fk) & 3u))
        return SKX_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SKX_CUDA_TRY(cudaMemsetAsync(d_out, 0, size_t(k) * 8, st));
    if (F == 0) return SKX_OK;
    const int optin = device_max_smem_optin();
    const size_t smem_full = (size_t(k) + kTopLane * 32) * 4;
    const bool use_smem = smem_full + 2048 <= (size_t)optin;
    const size_t smem = use_smem ? smem_full : size_t(kTopLane * 32) * 4;
    const int64_t mis = (int64_t)((reinterpret_cast<uintptr_t>(d_fk) & 15u) >> 2);
    const int64_t head = mis ? (F < 4 - mis ? F : 4 - mis) : 0;
    unsigned long long *out = reinterpret_cast<unsigned long long *>(d_out);
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = set_smem_limit_once(reinterpret_cast<const void *>(kern), -1);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kOpBlock, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        kern<<<grid_cap(((F - head) >> 2) + 1, per_sm), kOpBlock, smem, st>>>(d_fk, F, head, k, out);
        note_launches(1);
        return cudaGetLastError();
    };
    SKX_CUDA_TRY(use_smem ? go(k_topk<true>) : go(k_topk<false>));
    return SKX_OK;
}

skx_status skx_select_bitmap(const void *d_rows, int32_t N, int32_t row_bytes, int32_t filter_col, int32_t filter_lt,
                             uint32_t *d_bits, void *stream) {
    if (!d_rows || N < 1 || row_bytes <= 0 || row_bytes % 4 || filter_col < 0 || filter_col >= row_bytes / 4 || !d_bits ||
        (reinterpret_cast<uintptr_t>(d_rows) & 3u))
        return SKX_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_bitmap<<<grid_cap(int64_t(N), 4), kOpBlock, 0, st>>>(static_cast<const int32_t *>(d_rows), N, row_bytes / 4,
                                                           filter_col, filter_lt, d_bits);
    note_launches(1);
    SKX_CUDA_TRY(cudaGetLastError());
    return SKX_OK;
}

skx_status skx_select(const uint32_t *d_bits, int32_t N, const int32_t *d_fk, int64_t F, uint32_t *d_offsets,
                      int64_t *d_count, void *stream) {
    if (!d_bits || N < 1 || F < 0 || F >= (int64_t(1) << 32) || !d_count || (F > 0 && (!d_fk || !d_offsets)) ||
        (reinterpret_cast<uintptr_t>(d_fk) & 3u))
        return SKX_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (F == 0) {
        SKX_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(int64_t), st));
        return SKX_OK;
    }
    unsigned *err = device_error_word();
    if (!err) return SKX_ENOMEM;
    const uint32_t tiles = (uint32_t)((F + kSelTile - 1) / kSelTile);
    const uint32_t nbs = exclusive_scan_block_sums(tiles);
    uint32_t *scratch = nullptr;
    SKX_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&scratch), sizeof(uint32_t) * (2 * size_t(tiles) + nbs), st));
    uint32_t *cnt = scratch, *off = scratch + tiles, *bs = scratch + 2 * size_t(tiles);
    k_select_count<<<tiles, kOpBlock, 0, st>>>(d_fk, F, d_bits, N, cnt, err);
    cudaError_t e = cudaMemcpyAsync(off, cnt, sizeof(uint32_t) * tiles, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = exclusive_scan_u32(off, tiles, bs, st);
    if (e == cudaSuccess) {
        k_select_write<<<tiles, kOpBlock, 0, st>>>(d_fk, F, d_bits, N, off, d_offsets);
        k_select_total<<<1, 1, 0, st>>>(off, cnt, tiles, reinterpret_cast<long long *>(d_count));
        note_launches(3);
        e = cudaGetLastError();
    }
    cudaFreeAsync(scratch, st);
    SKX_CUDA_TRY(e);
    return SKX_OK;
}

}  // extern "C"
