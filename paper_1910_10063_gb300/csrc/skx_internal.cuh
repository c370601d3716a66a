// skx_internal.cuh -- shared definitions of the CUDA translation units of libskx.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/skx.h"

namespace skx {

// bits of the per-device data-error word
constexpr unsigned kErrKeyRange = 1u;
constexpr unsigned kErrGroupRange = 2u;
constexpr unsigned kErrTimeout = 4u;
constexpr unsigned kErrCountBound = 8u;  // a sort met a count above the bound F it was given

constexpr int kWarp = 32;

// -------------------------------------------------------------- host helpers
skx_status cuda_status(cudaError_t e);          // records the message, maps to SKX_ECUDA
unsigned *device_error_word();                  // the current device's word (a __device__ variable)
int device_sm_count();                          // SMs of the current device
int device_max_smem_optin();                    // max dynamic smem per block (opt-in)
void note_launches(int n);                      // adds to the process-wide kernel-launch counter
// Raises a kernel's dynamic shared-memory limit on the current device, once per (device,
// kernel): the attribute belongs to each device's context.  dynamic_bytes < 0 asks for the
// device's opt-in limit minus the kernel's static shared memory.
cudaError_t set_smem_limit_once(const void *kernel, int dynamic_bytes);

#define SKX_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t e__ = (expr);                           \
        if (e__ != cudaSuccess) return ::skx::cuda_status(e__); \
    } while (0)

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// -------------------------------------------------------------- device helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// L2 eviction-priority policies (createpolicy) for loads that stream through
// once (evict_first) and for gathers whose lines should outlive the stream
// (evict_last).
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_normal() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_unchanged() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_unchanged.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// 1 evict_last, 2 evict_normal, 3 evict_first, 4 evict_unchanged
__device__ __forceinline__ uint64_t policy_by_code(int code) {
    switch (code) {
        case 1: return policy_evict_last();
        case 3: return policy_evict_first();
        case 4: return policy_evict_unchanged();
        default: return policy_evict_normal();
    }
}

// 16-byte streaming load: read-only path, no L1 allocation, L2 evict-first.
__device__ __forceinline__ int4 ld_stream16(const int4 *p, uint64_t pol) {
    int4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
// Same through the coherent path, for data the kernel itself overwrites (in-place remap).
__device__ __forceinline__ int4 ld_stream16_rw(const int4 *p, uint64_t pol) {
    int4 v;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int ld_stream4(const int *p, uint64_t pol) {
    int v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;"
                 : "=r"(v)
                 : "l"(p), "l"(pol));
    return v;
}
// 16-byte streaming store (evict-first in L2).
__device__ __forceinline__ void st_stream16(int4 *p, int4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.s32 [%0], {%1,%2,%3,%4}, %5;"
                 :
                 : "l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
}
// gathers through the read-only path with an explicit L2 policy
__device__ __forceinline__ int4 ld_gather16(const int4 *p, uint64_t pol) {
    int4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int ld_gather4(const int *p, uint64_t pol) {
    int v;
    asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
// A 4-byte read of a randomly placed row of 64 bytes or more, with the L2
// prefetch-size hint .L2::64B: without it such a miss was seen to bring in a
// whole 128-byte line, half of it another row.  (For narrow rows or small
// arrays the longer line carries useful neighbours, and the hint was slower.)
__device__ __forceinline__ int ld_row4_p64(const int *p) {
    int v;
    asm volatile("ld.global.nc.L2::64B.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
// The same for an aligned 16-byte chunk of a row.
__device__ __forceinline__ int4 ld_row16_p64(const int4 *p) {
    int4 v;
    asm volatile("ld.global.nc.L2::64B.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void raise_error(unsigned *err, unsigned bit) {
    if (err) atomicOr(err, bit);
}

// -------------------------------------------------------------- internal entry points
// (launchers shared between the C-ABI implementation and the batch/serving paths)

// Histogram of keys[F] into cnt[N] (cnt must be zeroed by the caller).  With
// skip_if_set, the kernel returns at once when that device word is nonzero.
cudaError_t launch_histogram(const int32_t *d_fk, int64_t F, int32_t N, uint32_t *d_cnt, unsigned *d_err,
                             cudaStream_t st, const uint32_t *skip_if_set = nullptr);

// The partitioned count (histogram_part.cu): same contract as launch_histogram
// (cnt zeroed by the caller), with caller-provided scratch of at least
// histogram_partitioned_scratch(N, F) bytes (16-byte aligned).
// With run_if_set, its kernels return at once when that device word is zero.
bool histogram_partitioned_fits(int32_t N, int64_t F);
size_t histogram_partitioned_scratch(int32_t N, int64_t F);
cudaError_t launch_histogram_partitioned(const int32_t *d_fk, int64_t F, int32_t N, uint32_t *d_cnt, unsigned *d_err,
                                         void *d_scratch, size_t scratch_bytes, cudaStream_t st,
                                         const uint32_t *run_if_set = nullptr);
// Samples the column and sets a device word (inside the partitioned count's
// scratch; *flag points to it) to 1 when the partitioned count should run, 0
// when the single pass should: the single pass wins when most keys belong to
// ids that its per-CTA cache holds.
cudaError_t launch_count_choice(const int32_t *d_fk, int64_t F, int32_t N, void *d_scratch, size_t scratch_bytes,
                                const uint32_t **flag, cudaStream_t st);

// The count the entry points use (method: skx_count_method).  Zeroes cnt,
// allocates the partitioned count's scratch on st and frees it there; in
// SKX_COUNT_AUTO a failed allocation falls back to the single pass.
cudaError_t launch_count(const int32_t *d_fk, int64_t F, int32_t N, uint32_t *d_cnt, unsigned *d_err, int method,
                         cudaStream_t st);

// Scratch bytes the frequency sort needs for n ids: four 4-byte arrays of n
// (keys and ids, ping-pong), the per-tile digit counts (256 per 4096-id tile),
// the scan's block sums and one word for the heavy-id count, each rounded up
// to 256 bytes.  sort.cu lays its scratch out in exactly this order.
constexpr size_t sort_up256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t sort_scratch_bound(size_t n) {
    return sort_up256(sort_up256(sort_up256(sort_up256(sort_up256(sort_up256(sort_up256(4 * n) + 4 * n) + 4 * n) +
                                                      4 * n) +
                                            4 * (((n + 4095) / 4096) * 256)) +
                                 4 * ((((n + 4095) / 4096) * 256 + 4095) / 4096 + 1)) +
                      4);
}
size_t sort_scratch_bytes(int32_t N, int64_t F);
// Sorts ids by (cnt desc, id asc): writes perm (new->old) and rank (old->new).
// F must bound the sum of the counts.  A count above F, or more ids with a
// count >= 255 than F / 255 allows, raises kErrCountBound on d_err (when not
// null): the order would otherwise be silently incomplete.
cudaError_t launch_sort_by_count(const uint32_t *d_cnt, int32_t N, int64_t F, int32_t *d_perm, int32_t *d_rank,
                                 void *d_scratch, size_t scratch_bytes, unsigned *d_err, cudaStream_t st);

// Exclusive prefix sum of d_data[L] in place (3 kernels); d_block_sums needs
// exclusive_scan_block_sums(L) entries.  With run_if_set, the kernels return
// at once when that device word is zero.
cudaError_t exclusive_scan_u32(uint32_t *d_data, uint32_t L, uint32_t *d_block_sums, cudaStream_t st,
                               const uint32_t *run_if_set = nullptr);
uint32_t exclusive_scan_block_sums(uint32_t L);

cudaError_t launch_remap(const int32_t *d_rank, int32_t N, const int32_t *d_in, int32_t *d_out, int64_t F,
                         unsigned *d_err, cudaStream_t st);
cudaError_t launch_reorder(const int32_t *d_perm, int32_t N, const void *d_in, void *d_out, int32_t row_bytes,
                           cudaStream_t st);
cudaError_t launch_materialize(const void *d_rows, int32_t N, int32_t row_bytes, int32_t col, const int32_t *d_fk,
                               int64_t F, int32_t *d_out, unsigned *d_err, cudaStream_t st);
cudaError_t launch_reorder_columns(const int32_t *d_perm, int32_t N, const void *d_in, int32_t row_bytes,
                                   const int32_t *cols, int32_t ncols, void *d_out, cudaStream_t st);
cudaError_t launch_reorder_query(const int32_t *d_perm, int32_t N, const void *d_in, int32_t row_bytes,
                                 const skx_query &q, void *d_out, unsigned *d_err, cudaStream_t st,
                                 uint32_t *d_out4 = nullptr);
// Key bits of the packed query copy: the smallest b with 2^b >= G + 2 (keys 0..G, G the
// sentinel of a filtered row, and 2^b - 1 the escape), G = num_groups for GROUP BY, else 1.
int32_t packed_key_bits(const skx_query &q);

struct ProbeArgs {
    const void *rows;
    int32_t N, row_bytes;
    const int32_t *fk, *measure;
    int64_t F;
    skx_query q;
    int64_t *out;
    unsigned *err;
    bool accumulate;  // add into out instead of overwriting it (probing a column in chunks)
};
// Resolves defaults in `t` (in place) for these arguments.
void resolve_probe_tuning(const ProbeArgs &a, skx_tuning &t);
// Buckets of the split probe's second pass for keys [t_split, N): raises
// *bshift until there are at most 512 of them, returns their number.
int32_t split_buckets(int32_t N, int32_t t_split, int32_t *bshift);
cudaError_t launch_probe(const ProbeArgs &a, const skx_tuning &t, cudaStream_t st);
// The probe over the packed query copy (a.rows: the 8-byte copy the escapes are read from,
// a.q: the original query); block_threads and ctas_per_sm of t are used.
cudaError_t launch_probe_packed(const ProbeArgs &a, const uint32_t *rows4, const skx_tuning &t, cudaStream_t st);
skx_status validate_query(const skx_query *q, int32_t row_bytes);
// One unit of a batched probe launch (batch.cu): a query over a contiguous
// range of remapped fact rows, accumulating into `out`.
struct BatchDesc {
    const int32_t *fk;
    const int32_t *measure;
    unsigned long long *out;
    int64_t F;
    int32_t agg, fcol, flt, gcol, G, pcol;
    int32_t vec;  // fk and measure 16-byte aligned: 16-byte loads
    int32_t nout;
};

// Row access path for a table (0 generic, 1 16-byte, 2 8-byte rows).
int batch_row_path(const void *rows, int32_t row_bytes, bool cols_beyond16, bool cols_beyond8);
// Enqueues the batched probe over n device descriptors and their tile table.
// clear_outputs: zero every output first (else outputs accumulate).
cudaError_t launch_batch_items(const BatchDesc *d_desc, const uint32_t *d_tile_start, int32_t n,
                               uint32_t total_tiles, int32_t tile_rows, const void *rows, int32_t N,
                               int32_t row_bytes, int path, int32_t max_groups, const skx_tuning &t,
                               bool clear_outputs, uint32_t *d_counter, cudaStream_t st);

// Autotuner cache lookup (autotune.cu).
bool cached_probe_tuning(int32_t N, int32_t row_bytes, const skx_query &q, int64_t F, int remapped, skx_tuning *out);

}  // namespace skx
