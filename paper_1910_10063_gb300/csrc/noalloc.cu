// noalloc.cu -- a variant of the frequency sort that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they need the
// index: a process whose framework has already reserved nearly all of HBM in
// its own caching allocator, a latency-critical loop in which an allocation
// (which may synchronise the device or fail under memory pressure) is not
// acceptable, or a plug-in that is handed its buffers and may not touch the
// CUDA allocator at all.  For them, skx_sort_by_count_noalloc runs the same
// sort kernels as skx_build_index_from_counts, but its scratch space is a
// fixed array in this library's device image instead of a stream-ordered
// allocation.  The caller passes the counts and receives perm and rank in
// its own buffers.
//
// The array holds the scratch of the largest supported domain,
// N <= kNoAllocMaxN ids (about 16 MiB).  A device reserves it when this
// file's module is first loaded there -- the first call on that device, or
// library load under CUDA_MODULE_LOADING=EAGER -- and keeps it until the
// process exits.  A call with N = 0 does only that set-up, so a caller can
// make it early, while memory is still free.
#include "skx_internal.cuh"

namespace skx {
namespace {

constexpr int32_t kNoAllocMaxN = 1 << 20;

// Scratch of the radix sort for kNoAllocMaxN ids (about 16 MiB).
constexpr size_t kNoAllocScratchBytes = sort_scratch_bound(size_t(kNoAllocMaxN));

static __device__ __align__(256) unsigned char g_sort_scratch[kNoAllocScratchBytes];

// The array's name in host code is only a host-side stand-in; its device
// address is looked up with the caller's device current, on every call.  The
// address is not cached: after cudaDeviceReset (or any teardown of the
// primary context) a cached one would no longer be mapped.  Once this file's
// module is loaded on the device the lookup is cheap; the first lookup loads
// it, and that is when the device reserves the array (CUDA loads modules
// lazily unless CUDA_MODULE_LOADING=EAGER, which reserves it at library
// load).
skx_status scratch_address(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess || p == nullptr) return cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    *out = p;
    return SKX_OK;
}

}  // namespace
}  // namespace skx

using namespace skx;

extern "C" skx_status skx_sort_by_count_noalloc(const uint32_t *d_counts, int32_t N, int64_t F, int32_t *d_perm,
                                                int32_t *d_rank, void *stream) {
    if (N < 0 || F < 0 || F >= (int64_t(1) << 32)) return SKX_EINVAL;
    if (N > kNoAllocMaxN) return SKX_EINVAL;  // beyond the fixed scratch array
    void *scratch = nullptr;
    skx_status s = scratch_address(&scratch);
    if (s != SKX_OK) return s;
    unsigned *err = device_error_word();  // a __device__ variable as well: no allocation
    if (!err) return SKX_ECUDA;
    if (N == 0) return SKX_OK;  // set-up only: the array and the error word are now resident
    if (!d_counts || !d_perm || !d_rank) return SKX_EINVAL;
    if (sort_scratch_bytes(N, F) > kNoAllocScratchBytes) return SKX_EINVAL;
    // Nothing in the scratch needs to start at zero: every pass fully writes
    // the digit counts, block sums and key/id arrays before it reads them.
    SKX_CUDA_TRY(launch_sort_by_count(d_counts, N, F, d_perm, d_rank, scratch, kNoAllocScratchBytes, err,
                                      static_cast<cudaStream_t>(stream)));
    return SKX_OK;
}

extern "C" int32_t skx_sort_by_count_noalloc_max_n(void) { return kNoAllocMaxN; }
