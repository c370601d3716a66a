// histogram.cu -- frequency count of the FK column (the Q3 aggregation that
// starts the index build, Section III-A): cnt[v] = #{i : fk[i] == v}.
//
// GB300 design: the FK column is streamed once with 16-byte loads marked
// L2 evict-first, so the counter array (4 B per dimension id) stays in L2.
// Hot keys are the problem under skew (at Zipf s = 1.5 a third of all rows
// carry the same key): lanes of a warp holding the same key are merged with
// __match_any_sync and one lane issues a single atomic of the group size,
// the GPU counterpart of the paper's conflict handling in SIMD aggregation
// (Section IV-A/IV-B).  Keys outside [0, N) are skipped and flagged.
#include "skx_internal.cuh"

namespace skx {
namespace {

constexpr int kHistBlock = 512;
constexpr int kHistUnroll = 2;  // 16-byte vectors per lane per iteration

__device__ __forceinline__ void count_key(int32_t key, bool valid, int32_t N, uint32_t *__restrict__ cnt,
                                          unsigned *err) {
    const bool ok = valid && (uint32_t)key < (uint32_t)N;
    if (valid && !ok) raise_error(err, kErrKeyRange);
    const unsigned peers = __match_any_sync(0xffffffffu, ok ? key : -1);
    if (ok && (lane_id() == (unsigned)(__ffs(peers) - 1))) atomicAdd(cnt + key, (uint32_t)__popc(peers));
}

__global__ void __launch_bounds__(kHistBlock)
    k_histogram(const int32_t *__restrict__ fk, int64_t F, int64_t head, int32_t N, uint32_t *__restrict__ cnt,
                unsigned *err) {
    const uint64_t pol = policy_evict_first();
    const int4 *vec = reinterpret_cast<const int4 *>(fk + head);
    const int64_t nvec = (F - head) >> 2;
    const int64_t lane = lane_id();
    const int64_t warp = (int64_t(blockIdx.x) * kHistBlock + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * kHistBlock) >> 5;
    constexpr int64_t chunk = 32 * kHistUnroll;

    for (int64_t base = warp * chunk; base < nvec; base += nwarps * chunk) {
        int4 k[kHistUnroll];
        bool v[kHistUnroll];
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) {
            const int64_t i = base + u * 32 + lane;
            v[u] = i < nvec;
            k[u] = v[u] ? ld_stream16(vec + i, pol) : make_int4(-1, -1, -1, -1);
        }
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) {
            count_key(k[u].x, v[u], N, cnt, err);
            count_key(k[u].y, v[u], N, cnt, err);
            count_key(k[u].z, v[u], N, cnt, err);
            count_key(k[u].w, v[u], N, cnt, err);
        }
    }
    // unaligned head and the ragged tail (fewer than 4 + 3 keys) by warp 0
    if (warp == 0) {
        const int64_t tail0 = head + (nvec << 2);
        const int64_t extra = head + (F - tail0);
        for (int64_t j0 = 0; j0 < extra; j0 += 32) {
            const int64_t j = j0 + lane;
            const bool valid = j < extra;
            const int64_t idx = j < head ? j : tail0 + (j - head);
            count_key(valid ? fk[idx] : -1, valid, N, cnt, err);
        }
    }
}

}  // namespace

cudaError_t launch_histogram(const int32_t *d_fk, int64_t F, int32_t N, uint32_t *d_cnt, unsigned *d_err,
                             cudaStream_t st) {
    if (F <= 0) return cudaSuccess;
    const int64_t mis = (int64_t)((reinterpret_cast<uintptr_t>(d_fk) & 15u) >> 2);
    const int64_t head = mis ? (F < 4 - mis ? F : 4 - mis) : 0;
    const int64_t nvec = (F - head) >> 2;
    const int sms = device_sm_count();
    int64_t want = (nvec + 32 * kHistUnroll * (kHistBlock / 32) - 1) / (32 * kHistUnroll * (kHistBlock / 32));
    int64_t cap = (int64_t)sms * (2048 / kHistBlock);
    int grid = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    k_histogram<<<grid, kHistBlock, 0, st>>>(d_fk, F, head, N, d_cnt, d_err);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace skx
