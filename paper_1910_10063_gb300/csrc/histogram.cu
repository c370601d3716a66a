// histogram.cu -- frequency count of the FK column (the Q3 aggregation that
// starts the index build, Section III-A): cnt[v] = #{i : fk[i] == v}.
//
// GB300 design.  The FK column is streamed once with 16-byte loads marked L2
// evict-first, so the counter array (4 B per dimension id) stays in L2.
// Random atomics into L2 are cheap; what is not cheap is skew: atomics on one
// address serialise in its L2 slice, and at Zipf s = 1 the hottest key alone
// takes ~6% of all rows.  So each CTA keeps a small shared-memory cache of
// keys (open addressing, first come first served): a key that owns a slot is
// counted with a shared-memory atomic, any other key goes straight to the
// global counter.  Popular keys show up in the first few hundred rows a CTA
// sees, so they claim slots at once and never reach L2 again; the slots are
// flushed with one global atomic each at the end.  This is the paper's
// hybrid of private buffers for hot items and shared atomics for the rest
// (Section IV-C), with the hot set discovered on the fly because the build
// runs before any frequency order exists.  Keys outside [0, N) are skipped
// and flagged.
#include "skx_internal.cuh"

namespace skx {
namespace {

constexpr int kHistBlock = 512;
constexpr int kHistUnroll = 2;     // 16-byte vectors per lane per iteration
constexpr int kSlotsLog = 12;
constexpr int kSlots = 1 << kSlotsLog;  // 4096 cached keys per CTA (32 KB)
constexpr int kProbes = 2;
constexpr int32_t kEmpty = -1;

__device__ __forceinline__ void count_key(int32_t key, bool valid, int32_t N, uint32_t *__restrict__ cnt,
                                          int32_t *s_key, uint32_t *s_cnt, unsigned *err) {
    if (!valid) return;
    if ((uint32_t)key >= (uint32_t)N) {
        raise_error(err, kErrKeyRange);
        return;
    }
    uint32_t slot = ((uint32_t)key * 0x9E3779B1u) >> (32 - kSlotsLog);
#pragma unroll
    for (int p = 0; p < kProbes; ++p) {
        int32_t owner = s_key[slot];
        if (owner == kEmpty) {
            const int32_t prev = atomicCAS(s_key + slot, kEmpty, key);
            owner = prev == kEmpty ? key : prev;  // claimed now, or taken meanwhile
        }
        if (owner == key) {
            atomicAdd(s_cnt + slot, 1u);
            return;
        }
        slot = (slot + 1) & (kSlots - 1);
    }
    atomicAdd(cnt + key, 1u);
}

__global__ void __launch_bounds__(kHistBlock)
    k_histogram(const int32_t *__restrict__ fk, int64_t F, int64_t head, int32_t N, uint32_t *__restrict__ cnt,
                unsigned *err, const uint32_t *skip_if_set) {
    if (skip_if_set && *skip_if_set) return;  // the partitioned count was chosen on the device
    __shared__ int32_t s_key[kSlots];
    __shared__ uint32_t s_cnt[kSlots];
    for (int i = threadIdx.x; i < kSlots; i += kHistBlock) {
        s_key[i] = kEmpty;
        s_cnt[i] = 0;
    }
    __syncthreads();

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
            count_key(k[u].x, v[u], N, cnt, s_key, s_cnt, err);
            count_key(k[u].y, v[u], N, cnt, s_key, s_cnt, err);
            count_key(k[u].z, v[u], N, cnt, s_key, s_cnt, err);
            count_key(k[u].w, v[u], N, cnt, s_key, s_cnt, err);
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
            count_key(valid ? fk[idx] : -1, valid, N, cnt, s_key, s_cnt, err);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSlots; i += kHistBlock) {
        const int32_t key = s_key[i];
        const uint32_t c = s_cnt[i];
        if (key != kEmpty && c) atomicAdd(cnt + key, c);
    }
}

}  // namespace

cudaError_t launch_histogram(const int32_t *d_fk, int64_t F, int32_t N, uint32_t *d_cnt, unsigned *d_err,
                             cudaStream_t st, const uint32_t *skip_if_set) {
    if (F <= 0) return cudaSuccess;
    const int64_t mis = (int64_t)((reinterpret_cast<uintptr_t>(d_fk) & 15u) >> 2);
    const int64_t head = mis ? (F < 4 - mis ? F : 4 - mis) : 0;
    const int64_t nvec = (F - head) >> 2;
    const int sms = device_sm_count();
    int64_t want = (nvec + 32 * kHistUnroll * (kHistBlock / 32) - 1) / (32 * kHistUnroll * (kHistBlock / 32));
    int64_t cap = (int64_t)sms * (2048 / kHistBlock);
    int grid = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    k_histogram<<<grid, kHistBlock, 0, st>>>(d_fk, F, head, N, d_cnt, d_err, skip_if_set);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_count(const int32_t *d_fk, int64_t F, int32_t N, uint32_t *d_cnt, unsigned *d_err, int method,
                         cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d_cnt, 0, size_t(N) * 4, st);
    if (e != cudaSuccess || F <= 0) return e;
    bool part = method == SKX_COUNT_PARTITIONED;
    if (method == SKX_COUNT_AUTO)
        part = N >= (1 << 16) && F >= (int64_t(1) << 26) && histogram_partitioned_fits(N, F);
    if (!part) return launch_histogram(d_fk, F, N, d_cnt, d_err, st);
    const size_t sb = histogram_partitioned_scratch(N, F);
    void *scratch = nullptr;
    e = cudaMallocAsync(&scratch, sb, st);
    if (e != cudaSuccess) {
        if (method != SKX_COUNT_AUTO) return e;
        (void)cudaGetLastError();
        return launch_histogram(d_fk, F, N, d_cnt, d_err, st);
    }
    if (method == SKX_COUNT_AUTO) {
        // a sample of the column decides on the device which count runs; the
        // other one's kernels return at once
        const uint32_t *flag = nullptr;
        e = launch_count_choice(d_fk, F, N, scratch, sb, &flag, st);
        if (e == cudaSuccess) e = launch_histogram(d_fk, F, N, d_cnt, d_err, st, flag);
        if (e == cudaSuccess) e = launch_histogram_partitioned(d_fk, F, N, d_cnt, d_err, scratch, sb, st, flag);
    } else {
        e = launch_histogram_partitioned(d_fk, F, N, d_cnt, d_err, scratch, sb, st);
    }
    const cudaError_t f = cudaFreeAsync(scratch, st);
    return e != cudaSuccess ? e : f;
}

}  // namespace skx
