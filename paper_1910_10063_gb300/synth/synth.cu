// synth.cu -- device twin of the seeded input generator (see include/skx_synth.h).
// Computes inputs only; shares nothing with the permutation-index kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/skx_synth.h"

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

__device__ __forceinline__ uint64_t draw(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * kGamma); }

__device__ __forceinline__ int32_t bounded(uint64_t x, int32_t lo, uint32_t range) {
    const uint64_t hi32 = x >> 32;
    if (range == 0) return (int32_t)(uint32_t)hi32;
    return (int32_t)((int64_t)lo + (int64_t)((hi32 * (uint64_t)range) >> 32));
}

__global__ void k_zipf(const double *__restrict__ cdf, const int32_t *__restrict__ r2id, int32_t n, uint64_t key,
                       int64_t start, int64_t count, int32_t *__restrict__ out) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
        const double u = (double)(draw(key, (uint64_t)(start + i)) >> 11) * 0x1.0p-53;
        // first r with cdf[r] > u (cdf[n-1] == 1 > u, so r < n)
        int32_t lo = 0, hi = n - 1;
        while (lo < hi) {
            const int32_t mid = lo + ((hi - lo) >> 1);
            if (__ldg(cdf + mid) > u) hi = mid;
            else lo = mid + 1;
        }
        out[i] = __ldg(r2id + lo);
    }
}

__global__ void k_uniform(uint64_t key, int64_t start, int64_t count, int32_t lo, uint32_t range,
                          int32_t *__restrict__ out) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = bounded(draw(key, (uint64_t)(start + i)), lo, range);
}

struct ColSpec {
    int32_t lo[64];
    uint32_t range[64];
};

__global__ void k_rows(uint64_t key, int64_t n, int32_t width, ColSpec spec, int32_t *__restrict__ out) {
    const int64_t total = n * width;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < total; j += int64_t(gridDim.x) * blockDim.x) {
        const int32_t c = (int32_t)(j % width);
        out[j] = bounded(draw(key, (uint64_t)j), spec.lo[c], spec.range[c]);
    }
}

unsigned grid_for(int64_t count) {
    int64_t g = (count + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

extern "C" {

int skx_synth_zipf(const double *d_cdf, const int32_t *d_r2id, int32_t n, uint64_t key, int64_t start, int64_t count,
                   int32_t *d_out, void *stream) {
    if (n < 1 || count < 0 || start < 0 || !d_cdf || !d_r2id || (count > 0 && !d_out)) return 1;
    if (count == 0) return 0;
    k_zipf<<<grid_for(count), 256, 0, static_cast<cudaStream_t>(stream)>>>(d_cdf, d_r2id, n, key, start, count, d_out);
    return cudaGetLastError() == cudaSuccess ? 0 : 5;
}

int skx_synth_uniform(uint64_t key, int64_t start, int64_t count, int32_t lo, uint32_t range, int32_t *d_out,
                      void *stream) {
    if (count < 0 || start < 0 || (count > 0 && !d_out)) return 1;
    if (count == 0) return 0;
    k_uniform<<<grid_for(count), 256, 0, static_cast<cudaStream_t>(stream)>>>(key, start, count, lo, range, d_out);
    return cudaGetLastError() == cudaSuccess ? 0 : 5;
}

int skx_synth_rows(uint64_t key, int64_t n, int32_t width, const int32_t *h_lo, const uint32_t *h_range,
                   int32_t *d_out, void *stream) {
    if (n < 0 || width < 1 || width > 64 || !h_lo || !h_range || (n > 0 && !d_out)) return 1;
    if (n == 0) return 0;
    ColSpec spec{};
    for (int c = 0; c < width; ++c) {
        spec.lo[c] = h_lo[c];
        spec.range[c] = h_range[c];
    }
    k_rows<<<grid_for(n * width), 256, 0, static_cast<cudaStream_t>(stream)>>>(key, n, width, spec, d_out);
    return cudaGetLastError() == cudaSuccess ? 0 : 5;
}

}  // extern "C"
