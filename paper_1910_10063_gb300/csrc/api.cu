// api.cu -- the extern "C" boundary of libskx (declared in include/skx.h).
// Argument checking, the index object, stream-ordered allocation and the
// per-device data-error word; every step of the path runs in the kernels of
// histogram.cu, sort.cu, remap.cu and probe.cu.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "skx_internal.cuh"

struct skx_index {
    int device;
    int32_t N;
    int64_t F;
    cudaStream_t stream;  // stream the arrays were allocated on (freed there)
    uint32_t *counts;
    int32_t *perm;
    int32_t *rank;
};

// Per-device data-error word (bits kErr*): a fixed 4-byte variable of this
// library's device image, so that no entry point has to allocate for it.
static __device__ unsigned g_err_word_dev = 0;

namespace skx {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int g_sms[kMaxDevices] = {};
int g_smem_optin[kMaxDevices] = {};
thread_local char g_last_cuda[256] = "no CUDA error";
std::atomic<uint64_t> g_launches{0};

int current_device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return 0;
    return d;
}

void query_device(int d) {
    if (g_sms[d] > 0) return;
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
    g_sms[d] = v > 0 ? v : 1;
    v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, d);
    g_smem_optin[d] = v > 0 ? v : 48 * 1024;
    // keep freed stream-ordered allocations in the device pool between calls
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
}

bool valid_stream_ptrs(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

cudaStream_t g_copy_stream[kMaxDevices] = {};

// A non-blocking stream per device for host-to-device copies that overlap the
// kernels of the host-buffer path (created on first use, kept for the process).
cudaStream_t copy_stream() {
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_copy_stream[d] && cudaStreamCreateWithFlags(&g_copy_stream[d], cudaStreamNonBlocking) != cudaSuccess)
        g_copy_stream[d] = nullptr;
    return g_copy_stream[d];
}

}  // namespace

void note_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

namespace {
std::set<std::pair<int, const void *>> g_smem_set;  // (device, kernel) with the limit raised
}  // namespace

cudaError_t set_smem_limit_once(const void *kernel, int dynamic_bytes) {
    const int d = current_device();
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_smem_set.count({d, kernel})) return cudaSuccess;
    }
    if (dynamic_bytes < 0) {
        cudaFuncAttributes fa{};
        const cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
        if (e != cudaSuccess) return e;
        dynamic_bytes = device_max_smem_optin() - (int)fa.sharedSizeBytes;
    }
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dynamic_bytes);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_mu);
        g_smem_set.insert({d, kernel});
    }
    return e;
}

skx_status cuda_status(cudaError_t e) {
    snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return SKX_ENOMEM;
    return SKX_ECUDA;
}

// The device address of the error word, looked up on every call with the
// caller's device current.  Not cached: after cudaDeviceReset (or any
// teardown of the primary context) a cached address would no longer be
// mapped, and a kernel given it would fault.  The word is zero when the
// module is loaded and is cleared by skx_stream_status.
unsigned *device_error_word() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_err_word_dev) != cudaSuccess) return nullptr;
    return static_cast<unsigned *>(p);
}

int device_sm_count() {
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    query_device(d);
    return g_sms[d];
}

int device_max_smem_optin() {
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    query_device(d);
    return g_smem_optin[d];
}

}  // namespace skx

using namespace skx;

namespace skx_rankcounts {
// out[k] = counts[perm[ranks[k]]]
__global__ void k_counts_at_ranks(const uint32_t *counts, const int32_t *perm, const int64_t *ranks, int64_t n,
                                  uint32_t *out) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        out[k] = counts[perm[ranks[k]]];
}
}  // namespace skx_rankcounts

namespace skx_append {
__global__ void k_append_tail(int32_t *perm, int32_t *rank, uint32_t *counts, int32_t N, int32_t n_new) {
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n_new; j += int64_t(gridDim.x) * blockDim.x) {
        perm[N + j] = N + (int32_t)j;
        rank[N + j] = N + (int32_t)j;
        counts[N + j] = 0;
    }
}
}  // namespace skx_append

namespace {

// Allocates an index whose counts are written by `fill` (a histogram or a copy),
// then sorts.  On failure everything is released.
template <typename Fill>
skx_status make_index(int32_t N, int64_t F, cudaStream_t st, skx_index **out, Fill fill) {
    skx_index *idx = new skx_index{};
    idx->device = 0;
    cudaGetDevice(&idx->device);
    idx->N = N;
    idx->F = F;
    idx->stream = st;
    const size_t nb = size_t(N) * 4;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&idx->counts), nb, st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&idx->perm), nb, st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&idx->rank), nb, st);
    void *scratch = nullptr;
    const size_t sb = sort_scratch_bytes(N, F);
    if (e == cudaSuccess && sb) e = cudaMallocAsync(&scratch, sb, st);
    if (e == cudaSuccess) e = fill(idx->counts);
    if (e == cudaSuccess)
        e = launch_sort_by_count(idx->counts, N, F, idx->perm, idx->rank, scratch, sb, device_error_word(), st);
    if (scratch) cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) {
        skx_status s = cuda_status(e);
        skx_index_destroy(idx);
        return s;
    }
    *out = idx;
    return SKX_OK;
}

}  // namespace

extern "C" {

const char *skx_strerror(skx_status s) {
    switch (s) {
        case SKX_OK: return "SKX_OK";
        case SKX_EINVAL: return "SKX_EINVAL: invalid argument";
        case SKX_ENOMEM: return "SKX_ENOMEM: out of memory";
        case SKX_EKEYRANGE: return "SKX_EKEYRANGE: foreign key outside [0, N)";
        case SKX_EGROUPRANGE: return "SKX_EGROUPRANGE: group key outside [0, G)";
        case SKX_ECUDA: return "SKX_ECUDA: CUDA error";
        case SKX_ETIMEOUT: return "SKX_ETIMEOUT: bounded wait expired";
        case SKX_EBUSY: return "SKX_EBUSY: resource busy";
        case SKX_ENOTSUP: return "SKX_ENOTSUP: not supported";
    }
    return "SKX_?: unknown status";
}

const char *skx_last_cuda_error(void) { return g_last_cuda; }

int32_t skx_version(void) { return (SKX_VERSION_MAJOR << 16) | SKX_VERSION_MINOR; }

uint64_t skx_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

skx_status skx_stream_status(void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SKX_CUDA_TRY(cudaStreamSynchronize(st));
    unsigned *w = device_error_word();
    if (!w) return SKX_ENOMEM;
    unsigned h = 0;
    SKX_CUDA_TRY(cudaMemcpyAsync(&h, w, sizeof(h), cudaMemcpyDeviceToHost, st));
    SKX_CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(unsigned), st));
    SKX_CUDA_TRY(cudaStreamSynchronize(st));
    if (h & kErrKeyRange) return SKX_EKEYRANGE;
    if (h & kErrGroupRange) return SKX_EGROUPRANGE;
    if (h & kErrTimeout) return SKX_ETIMEOUT;
    if (h & kErrCountBound) return SKX_EINVAL;
    return SKX_OK;
}

skx_status skx_count(const int32_t *d_fk, int64_t F, int32_t N, uint32_t *d_counts, void *stream) {
    if (N < 1 || F < 0 || F >= (int64_t(1) << 32) || (F > 0 && !d_fk) || !d_counts || !valid_stream_ptrs(d_fk) ||
        !valid_stream_ptrs(d_counts))
        return SKX_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned *err = device_error_word();
    if (!err) return SKX_ENOMEM;
    SKX_CUDA_TRY(launch_count(d_fk, F, N, d_counts, err, SKX_COUNT_AUTO, st));
    return SKX_OK;
}

skx_status skx_count_ex(const int32_t *d_fk, int64_t F, int32_t N, uint32_t *d_counts, int32_t method,
                        void *stream) {
    if (N < 1 || F < 0 || F >= (int64_t(1) << 32) || (F > 0 && !d_fk) || !d_counts || !valid_stream_ptrs(d_fk) ||
        !valid_stream_ptrs(d_counts) || method < SKX_COUNT_AUTO || method > SKX_COUNT_PARTITIONED)
        return SKX_EINVAL;
    if (method == SKX_COUNT_PARTITIONED && !histogram_partitioned_fits(N, F > 0 ? F : 1)) return SKX_ENOTSUP;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned *err = device_error_word();
    if (!err) return SKX_ENOMEM;
    SKX_CUDA_TRY(launch_count(d_fk, F, N, d_counts, err, method, st));
    return SKX_OK;
}

skx_status skx_build_index(const int32_t *d_fk, int64_t F, int32_t N, void *stream, skx_index **out) {
    if (!out) return SKX_EINVAL;
    *out = nullptr;
    if (N < 1 || F < 0 || F >= (int64_t(1) << 32) || (F > 0 && !d_fk) || !valid_stream_ptrs(d_fk)) return SKX_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned *err = device_error_word();
    if (!err) return SKX_ENOMEM;
    return make_index(N, F, st, out, [&](uint32_t *counts) {
        return launch_count(d_fk, F, N, counts, err, SKX_COUNT_AUTO, st);
    });
}

skx_status skx_build_index_from_counts(const uint32_t *d_counts, int32_t N, int64_t F, void *stream,
                                       skx_index **out) {
    if (!out) return SKX_EINVAL;
    *out = nullptr;
    if (N < 1 || F < 0 || F >= (int64_t(1) << 32) || !d_counts || !valid_stream_ptrs(d_counts)) return SKX_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return make_index(N, F, st, out, [&](uint32_t *counts) {
        return cudaMemcpyAsync(counts, d_counts, size_t(N) * 4, cudaMemcpyDeviceToDevice, st);
    });
}

skx_status skx_index_perm(const skx_index *idx, const int32_t **d_perm) {
    if (!idx || !d_perm) return SKX_EINVAL;
    *d_perm = idx->perm;
    return SKX_OK;
}

skx_status skx_index_rank(const skx_index *idx, const int32_t **d_rank) {
    if (!idx || !d_rank) return SKX_EINVAL;
    *d_rank = idx->rank;
    return SKX_OK;
}

skx_status skx_index_counts(const skx_index *idx, const uint32_t **d_counts) {
    if (!idx || !d_counts) return SKX_EINVAL;
    *d_counts = idx->counts;
    return SKX_OK;
}

int32_t skx_index_size(const skx_index *idx) { return idx ? idx->N : -1; }

skx_status skx_index_counts_at_ranks(const skx_index *idx, const int64_t *h_ranks, int64_t n, uint32_t *h_counts,
                                     void *stream) {
    if (!idx || n < 0 || (n > 0 && (!h_ranks || !h_counts))) return SKX_EINVAL;
    for (int64_t k = 0; k < n; ++k)
        if (h_ranks[k] < 0 || h_ranks[k] >= idx->N) return SKX_EINVAL;
    if (n == 0) return SKX_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t *d_r = nullptr;
    uint32_t *d_c = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d_r), size_t(n) * 8, st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&d_c), size_t(n) * 4, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_r, h_ranks, size_t(n) * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const int grid = (int)std::min<int64_t>((n + 255) / 256, int64_t(device_sm_count()) * 8);
        skx_rankcounts::k_counts_at_ranks<<<grid, 256, 0, st>>>(idx->counts, idx->perm, d_r, n, d_c);
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_counts, d_c, size_t(n) * 4, cudaMemcpyDeviceToHost, st);
    if (d_r) cudaFreeAsync(d_r, st);
    if (d_c) cudaFreeAsync(d_c, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? SKX_OK : cuda_status(e);
}

skx_status skx_index_drift(const skx_index *idx, const int32_t *d_fk_sample, int64_t n, int64_t t, double max_loss,
                           skx_drift *out, void *stream) {
    if (!idx || !d_fk_sample || !out || n < 1 || n >= (int64_t(1) << 32) || t < 1 || t > idx->N ||
        !(max_loss >= 0.0) || !valid_stream_ptrs(d_fk_sample))
        return SKX_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned *err = device_error_word();
    if (!err) return SKX_ECUDA;
    int32_t *d_r = nullptr;
    uint32_t *d_c = nullptr;
    std::vector<uint32_t> h(size_t(idx->N));
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d_r), size_t(n) * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&d_c), size_t(idx->N) * 4, st);
    if (e == cudaSuccess) e = launch_remap(idx->rank, idx->N, d_fk_sample, d_r, n, err, st);
    if (e == cudaSuccess) e = launch_count(d_r, n, idx->N, d_c, err, SKX_COUNT_AUTO, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_c, size_t(idx->N) * 4, cudaMemcpyDeviceToHost, st);
    if (d_r) cudaFreeAsync(d_r, st);
    if (d_c) cudaFreeAsync(d_c, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    return skx_drift_from_counts(h.data(), idx->N, t, max_loss, out);
}

void skx_index_destroy(skx_index *idx) {
    if (!idx) return;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != idx->device) cudaSetDevice(idx->device);
    if (idx->counts) cudaFreeAsync(idx->counts, idx->stream);
    if (idx->perm) cudaFreeAsync(idx->perm, idx->stream);
    if (idx->rank) cudaFreeAsync(idx->rank, idx->stream);
    if (prev != idx->device) cudaSetDevice(prev);
    delete idx;
}

skx_status skx_index_append(skx_index *idx, int32_t n_new, void *stream) {
    if (!idx || n_new < 0 || int64_t(idx->N) + n_new > INT32_MAX) return SKX_EINVAL;
    if (n_new == 0) return SKX_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t N = idx->N, N2 = N + n_new;
    uint32_t *c2 = nullptr;
    int32_t *p2 = nullptr, *r2 = nullptr;
    const size_t nb = size_t(N2) * 4, ob = size_t(N) * 4;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&c2), nb, st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&p2), nb, st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&r2), nb, st);
    // the index arrays were last written on the build stream: order against it first
    cudaEvent_t ev = nullptr;
    if (e == cudaSuccess && idx->stream != st) {
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, idx->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c2, idx->counts, ob, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p2, idx->perm, ob, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r2, idx->rank, ob, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        const int64_t g = std::min<int64_t>((n_new + 255) / 256, int64_t(device_sm_count()) * 8);
        skx_append::k_append_tail<<<(unsigned)std::max<int64_t>(g, 1), 256, 0, st>>>(p2, r2, c2, N, n_new);
        note_launches(1);
        e = cudaGetLastError();
    }
    if (ev) cudaEventDestroy(ev);
    if (e != cudaSuccess) {
        if (c2) cudaFreeAsync(c2, st);
        if (p2) cudaFreeAsync(p2, st);
        if (r2) cudaFreeAsync(r2, st);
        return cuda_status(e);
    }
    cudaFreeAsync(idx->counts, st);
    cudaFreeAsync(idx->perm, st);
    cudaFreeAsync(idx->rank, st);
    idx->counts = c2;
    idx->perm = p2;
    idx->rank = r2;
    idx->N = N2;
    idx->stream = st;
    return SKX_OK;
}

skx_status skx_remap(const skx_index *idx, const int32_t *d_fk_in, int32_t *d_fk_out, int64_t F, void *stream) {
    if (!idx || F < 0 || (F > 0 && (!d_fk_in || !d_fk_out))) return SKX_EINVAL;
    if (!valid_stream_ptrs(d_fk_in) || !valid_stream_ptrs(d_fk_out)) return SKX_EINVAL;
    if (F > 0 && d_fk_in != d_fk_out) {  // partial overlap is not allowed
        const char *a = reinterpret_cast<const char *>(d_fk_in), *b = reinterpret_cast<const char *>(d_fk_out);
        if (a < b + F * 4 && b < a + F * 4) return SKX_EINVAL;
    }
    unsigned *err = device_error_word();
    if (!err) return SKX_ENOMEM;
    SKX_CUDA_TRY(launch_remap(idx->rank, idx->N, d_fk_in, d_fk_out, F, err, static_cast<cudaStream_t>(stream)));
    return SKX_OK;
}

skx_status skx_materialize(const void *d_rows, int32_t N, int32_t row_bytes, int32_t col, const int32_t *d_fk,
                           int64_t F, int32_t *d_out, void *stream) {
    if (!d_rows || N < 1 || row_bytes <= 0 || row_bytes % 4 != 0 || col < 0 || col >= row_bytes / 4 || F < 0 ||
        F >= (int64_t(1) << 32) || (F > 0 && (!d_fk || !d_out)))
        return SKX_EINVAL;
    if (!valid_stream_ptrs(d_rows) || !valid_stream_ptrs(d_fk) || !valid_stream_ptrs(d_out)) return SKX_EINVAL;
    unsigned *err = device_error_word();
    if (!err) return SKX_ENOMEM;
    SKX_CUDA_TRY(launch_materialize(d_rows, N, row_bytes, col, d_fk, F, d_out, err, static_cast<cudaStream_t>(stream)));
    return SKX_OK;
}

skx_status skx_reorder(const skx_index *idx, const void *d_rows_in, void *d_rows_out, int32_t N, int32_t row_bytes,
                       void *stream) {
    if (!idx || N != idx->N || row_bytes <= 0 || row_bytes % 4 != 0 || !d_rows_in || !d_rows_out) return SKX_EINVAL;
    if (!valid_stream_ptrs(d_rows_in) || !valid_stream_ptrs(d_rows_out)) return SKX_EINVAL;
    const char *a = static_cast<const char *>(d_rows_in), *b = static_cast<const char *>(d_rows_out);
    const int64_t bytes = int64_t(N) * row_bytes;
    if (a < b + bytes && b < a + bytes) return SKX_EINVAL;
    SKX_CUDA_TRY(launch_reorder(idx->perm, N, d_rows_in, d_rows_out, row_bytes, static_cast<cudaStream_t>(stream)));
    return SKX_OK;
}

skx_status skx_reorder_columns(const skx_index *idx, const void *d_rows_in, int32_t N, int32_t row_bytes,
                               const int32_t *h_cols, int32_t ncols, void *d_out, void *stream) {
    if (N < 1 || row_bytes <= 0 || row_bytes % 4 != 0 || !d_rows_in || !d_out || !h_cols || ncols < 1 || ncols > 16)
        return SKX_EINVAL;
    if (idx && idx->N != N) return SKX_EINVAL;
    if (!valid_stream_ptrs(d_rows_in) || !valid_stream_ptrs(d_out)) return SKX_EINVAL;
    for (int i = 0; i < ncols; ++i)
        if (h_cols[i] < 0 || h_cols[i] >= row_bytes / 4) return SKX_EINVAL;
    const char *a = static_cast<const char *>(d_rows_in), *b = static_cast<const char *>(d_out);
    if (a < b + int64_t(N) * ncols * 4 && b < a + int64_t(N) * row_bytes) return SKX_EINVAL;
    SKX_CUDA_TRY(launch_reorder_columns(idx ? idx->perm : nullptr, N, d_rows_in, row_bytes, h_cols, ncols, d_out,
                                        static_cast<cudaStream_t>(stream)));
    return SKX_OK;
}

skx_status skx_reorder_query(const skx_index *idx, const void *d_rows_in, int32_t N, int32_t row_bytes,
                             const skx_query *q, void *d_out, void *stream) {
    skx_status s = validate_query(q, row_bytes);
    if (s != SKX_OK) return s;
    if (N < 1 || !d_rows_in || !d_out || (idx && idx->N != N)) return SKX_EINVAL;
    if (!valid_stream_ptrs(d_rows_in) || (reinterpret_cast<uintptr_t>(d_out) & 7u)) return SKX_EINVAL;
    const char *a = static_cast<const char *>(d_rows_in), *b = static_cast<const char *>(d_out);
    if (a < b + int64_t(N) * 8 && b < a + int64_t(N) * row_bytes) return SKX_EINVAL;
    unsigned *err = device_error_word();
    if (!err) return SKX_ENOMEM;
    SKX_CUDA_TRY(launch_reorder_query(idx ? idx->perm : nullptr, N, d_rows_in, row_bytes, *q, d_out, err,
                                      static_cast<cudaStream_t>(stream)));
    return SKX_OK;
}

skx_status skx_reorder_query_packed(const skx_index *idx, const void *d_rows_in, int32_t N, int32_t row_bytes,
                                    const skx_query *q, void *d_out8, uint32_t *d_out4, void *stream) {
    skx_status s = validate_query(q, row_bytes);
    if (s != SKX_OK) return s;
    if (N < 1 || !d_rows_in || !d_out8 || !d_out4 || (idx && idx->N != N)) return SKX_EINVAL;
    if (!valid_stream_ptrs(d_rows_in) || (reinterpret_cast<uintptr_t>(d_out8) & 7u) ||
        (reinterpret_cast<uintptr_t>(d_out4) & 3u))
        return SKX_EINVAL;
    const char *a = static_cast<const char *>(d_rows_in), *b = static_cast<const char *>(d_out8),
               *c = reinterpret_cast<const char *>(d_out4);
    const int64_t la = int64_t(N) * row_bytes, lb = int64_t(N) * 8, lc = int64_t(N) * 4;
    if ((a < b + lb && b < a + la) || (a < c + lc && c < a + la) || (b < c + lc && c < b + lb)) return SKX_EINVAL;
    unsigned *err = device_error_word();
    if (!err) return SKX_ENOMEM;
    SKX_CUDA_TRY(launch_reorder_query(idx ? idx->perm : nullptr, N, d_rows_in, row_bytes, *q, d_out8, err,
                                      static_cast<cudaStream_t>(stream), d_out4));
    return SKX_OK;
}

int32_t skx_query_packed_key_bits(const skx_query *q) {
    if (!q || q->agg < SKX_AGG_COUNT || q->agg > SKX_AGG_GROUPBY_SUM) return -1;
    if (q->agg == SKX_AGG_GROUPBY_SUM && (q->num_groups < 1 || q->num_groups > (1 << 24))) return -1;
    return packed_key_bits(*q);
}

skx_status skx_probe_packed(const uint32_t *d_rows4, const void *d_rows8, int32_t N, const int32_t *d_fk,
                            const int32_t *d_measure, int64_t F, const skx_query *q, int64_t *d_out,
                            const skx_tuning *tuning, void *stream) {
    if (skx_query_packed_key_bits(q) < 0) return SKX_EINVAL;
    if (N < 1 || F < 0 || F >= (int64_t(1) << 32) || !d_out || !d_rows4 || !d_rows8) return SKX_EINVAL;
    if (F > 0 && (!d_fk || (q->agg != SKX_AGG_COUNT && !d_measure))) return SKX_EINVAL;
    if (!valid_stream_ptrs(d_fk) || !valid_stream_ptrs(d_measure) || (reinterpret_cast<uintptr_t>(d_rows4) & 3u) ||
        (reinterpret_cast<uintptr_t>(d_rows8) & 7u) || (reinterpret_cast<uintptr_t>(d_out) & 7u))
        return SKX_EINVAL;
    unsigned *err = device_error_word();
    if (!err) return SKX_ENOMEM;
    ProbeArgs a{};
    a.rows = d_rows8;
    a.N = N;
    a.row_bytes = 8;
    a.fk = d_fk;
    a.measure = d_measure;
    a.F = F;
    a.q = *q;
    a.out = d_out;
    a.err = err;
    skx_tuning t{};
    if (tuning) t = *tuning;
    SKX_CUDA_TRY(launch_probe_packed(a, d_rows4, t, static_cast<cudaStream_t>(stream)));
    return SKX_OK;
}

skx_query skx_query_prefiltered(const skx_query *q) {
    skx_query r{};
    if (!q) return r;
    r.agg = q->agg;
    r.num_groups = q->agg == SKX_AGG_GROUPBY_SUM ? q->num_groups : 1;
    r.filter_col = 0;
    r.filter_lt = r.num_groups;  // the sentinel num_groups fails "key < num_groups"
    r.group_col = 0;
    r.payload_col = 1;
    return r;
}

skx_status skx_probe_default_tuning(int32_t N, int32_t row_bytes, int64_t F, const skx_query *q, int remapped,
                                    skx_tuning *out) {
    if (!out || N < 1 || F < 0) return SKX_EINVAL;
    skx_status s = validate_query(q, row_bytes);
    if (s != SKX_OK) return s;
    ProbeArgs a{};
    a.N = N;
    a.row_bytes = row_bytes;
    a.F = F;
    a.q = *q;
    skx_tuning t{};
    if (!cached_probe_tuning(N, row_bytes, *q, F, remapped, &t) && !remapped) t.hot_keys = -1;
    resolve_probe_tuning(a, t);
    *out = t;
    return SKX_OK;
}

skx_status skx_probe_resolve_tuning(int32_t N, int32_t row_bytes, int64_t F, const skx_query *q,
                                    const skx_tuning *in, skx_tuning *out) {
    if (!out || !in || N < 1 || F < 0) return SKX_EINVAL;
    skx_status s = validate_query(q, row_bytes);
    if (s != SKX_OK) return s;
    ProbeArgs a{};
    a.N = N;
    a.row_bytes = row_bytes;
    a.F = F;
    a.q = *q;
    skx_tuning t = *in;
    resolve_probe_tuning(a, t);
    *out = t;
    return SKX_OK;
}

skx_status skx_probe_aggregate(const void *d_rows, int32_t N, int32_t row_bytes, const int32_t *d_fk,
                               const int32_t *d_measure, int64_t F, const skx_query *q, int64_t *d_out,
                               const skx_tuning *tuning, void *stream) {
    skx_status s = validate_query(q, row_bytes);
    if (s != SKX_OK) return s;
    if (N < 1 || F < 0 || F >= (int64_t(1) << 32) || !d_out || !d_rows) return SKX_EINVAL;
    if (F > 0 && (!d_fk || (q->agg != SKX_AGG_COUNT && !d_measure))) return SKX_EINVAL;
    if (!valid_stream_ptrs(d_fk) || !valid_stream_ptrs(d_measure) || !valid_stream_ptrs(d_rows) ||
        (reinterpret_cast<uintptr_t>(d_out) & 7u))
        return SKX_EINVAL;
    unsigned *err = device_error_word();
    if (!err) return SKX_ENOMEM;
    ProbeArgs a{};
    a.rows = d_rows;
    a.N = N;
    a.row_bytes = row_bytes;
    a.fk = d_fk;
    a.measure = d_measure;
    a.F = F;
    a.q = *q;
    a.out = d_out;
    a.err = err;
    skx_tuning t{};
    if (tuning)
        t = *tuning;
    else
        cached_probe_tuning(N, row_bytes, *q, F, 1, &t);
    resolve_probe_tuning(a, t);
    SKX_CUDA_TRY(launch_probe(a, t, static_cast<cudaStream_t>(stream)));
    return SKX_OK;
}

skx_status skx_join_aggregate_host(const void *h_rows, int32_t N, int32_t row_bytes, const int32_t *h_fk,
                                   const int32_t *h_measure, int64_t F, const skx_query *q, int64_t *h_out,
                                   void *stream) {
    skx_status s = validate_query(q, row_bytes);
    if (s != SKX_OK) return s;
    if (N < 1 || F < 0 || F >= (int64_t(1) << 32) || !h_rows || !h_out) return SKX_EINVAL;
    if (F > 0 && (!h_fk || (q->agg != SKX_AGG_COUNT && !h_measure))) return SKX_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nout = q->agg == SKX_AGG_GROUPBY_SUM ? q->num_groups : 1;
    const size_t rows_b = size_t(N) * row_bytes, fk_b = size_t(F) * 4;
    // clear any stale error bits so this call reports only its own
    skx_status pre = skx_stream_status(stream);
    if (pre == SKX_ECUDA || pre == SKX_ENOMEM) return pre;
    unsigned *err = device_error_word();
    if (!err) return SKX_ENOMEM;
    cudaStream_t cs = copy_stream();
    if (!cs) return SKX_ECUDA;

    // The host link, not HBM, bounds this path, so copies run on their own
    // stream in the order the kernels need them -- fk, then the dimension
    // rows, then the measure column in chunks -- and each kernel waits only
    // for its inputs: the build and the remap overlap the copy of the rows,
    // the reorder and the probe of each measure chunk overlap the copy of the
    // next chunk.
    constexpr int kChunks = 8;
    const bool with_m = F > 0 && q->agg != SKX_AGG_COUNT;
    const int nm = with_m ? kChunks : 0;
    char *d_rows = nullptr, *d_rows2 = nullptr;
    uint32_t *d_rows4 = nullptr;
    int32_t *d_fk = nullptr, *d_m = nullptr;
    int64_t *d_out = nullptr;
    skx_index *idx = nullptr;
    cudaEvent_t ev_alloc = nullptr, ev_fk = nullptr, ev_rows = nullptr, ev_done = nullptr, ev_m[kChunks] = {};
    // the probe runs over the query's own permuted copy (Section III-B): {group or the
    // filter's sentinel, payload} packed in 32 bits per dimension row, with its 8-byte form
    // beside it for the rows that do not fit
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d_rows), rows_b, st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&d_rows2), size_t(N) * 8, st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&d_rows4), size_t(N) * 4, st);
    if (e == cudaSuccess && F > 0) e = cudaMallocAsync(reinterpret_cast<void **>(&d_fk), fk_b, st);
    if (e == cudaSuccess && with_m) e = cudaMallocAsync(reinterpret_cast<void **>(&d_m), fk_b, st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&d_out), size_t(nout) * 8, st);
    for (cudaEvent_t *ev : {&ev_alloc, &ev_fk, &ev_rows, &ev_done})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    for (int k = 0; k < nm && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev_m[k], cudaEventDisableTiming);
    // chunk k of the measure column: rows [cut(k), cut(k + 1)), cuts on 16-byte boundaries
    auto cut = [&](int k) { return k >= nm ? F : ((F * k / nm) & ~int64_t(3)); };
    bool copies = false;
    if (e == cudaSuccess) e = cudaEventRecord(ev_alloc, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_alloc, 0);
    if (e == cudaSuccess) {
        copies = true;
        if (d_fk) e = cudaMemcpyAsync(d_fk, h_fk, fk_b, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev_fk, cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_rows, h_rows, rows_b, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev_rows, cs);
        for (int k = 0; k < nm && e == cudaSuccess; ++k) {
            const int64_t a0 = cut(k), a1 = cut(k + 1);
            if (a1 > a0)
                e = cudaMemcpyAsync(d_m + a0, h_measure + a0, size_t(a1 - a0) * 4, cudaMemcpyHostToDevice, cs);
            if (e == cudaSuccess) e = cudaEventRecord(ev_m[k], cs);
        }
        const cudaError_t e2 = cudaEventRecord(ev_done, cs);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) s = cuda_status(e);
    if (s == SKX_OK) s = cudaStreamWaitEvent(st, ev_fk, 0) == cudaSuccess ? SKX_OK : SKX_ECUDA;
    if (s == SKX_OK) s = skx_build_index(d_fk, F, N, stream, &idx);
    if (s == SKX_OK) s = skx_remap(idx, d_fk, d_fk, F, stream);
    if (s == SKX_OK) s = cudaStreamWaitEvent(st, ev_rows, 0) == cudaSuccess ? SKX_OK : SKX_ECUDA;
    if (s == SKX_OK) s = skx_reorder_query_packed(idx, d_rows, N, row_bytes, q, d_rows2, d_rows4, stream);
    if (s == SKX_OK) {
        ProbeArgs a{};
        a.rows = d_rows2;
        a.N = N;
        a.row_bytes = 8;
        a.q = *q;
        a.out = d_out;
        a.err = err;
        skx_tuning t{};  // 512 threads, as many CTAs as fit
        const int parts = with_m ? nm : 1;
        for (int k = 0; k < parts && s == SKX_OK; ++k) {
            const int64_t a0 = with_m ? cut(k) : 0, a1 = with_m ? cut(k + 1) : F;
            if (with_m && cudaStreamWaitEvent(st, ev_m[k], 0) != cudaSuccess) s = SKX_ECUDA;
            a.fk = d_fk ? d_fk + a0 : nullptr;
            a.measure = d_m ? d_m + a0 : nullptr;
            a.F = a1 - a0;
            a.accumulate = k > 0;
            if (s == SKX_OK) {
                e = launch_probe_packed(a, d_rows4, t, st);
                if (e != cudaSuccess) s = cuda_status(e);
            }
        }
    }
    if (s == SKX_OK) {
        e = cudaMemcpyAsync(h_out, d_out, size_t(nout) * 8, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) s = cuda_status(e);
    }
    // the buffers are freed in the compute stream's order: it first waits for every copy
    if (copies) cudaStreamWaitEvent(st, ev_done, 0);
    skx_index_destroy(idx);
    if (d_rows) cudaFreeAsync(d_rows, st);
    if (d_rows2) cudaFreeAsync(d_rows2, st);
    if (d_rows4) cudaFreeAsync(d_rows4, st);
    if (d_fk) cudaFreeAsync(d_fk, st);
    if (d_m) cudaFreeAsync(d_m, st);
    if (d_out) cudaFreeAsync(d_out, st);
    skx_status fin = skx_stream_status(stream);
    for (cudaEvent_t ev : {ev_alloc, ev_fk, ev_rows, ev_done})
        if (ev) cudaEventDestroy(ev);
    for (int k = 0; k < nm; ++k)
        if (ev_m[k]) cudaEventDestroy(ev_m[k]);
    return s != SKX_OK ? s : fin;
}

}  // extern "C"
