/*
 * skx_synth.h -- C ABI of libskx_synth.so, the seeded synthetic-input
 * generator used by the tests and the benchmark.  It computes inputs only
 * (none of the permutation index's arithmetic) and has a bit-identical host
 * twin in paper_1910_10063_gb300/synth/__init__.py.  The paper has no
 * counterpart beyond its skew model: Zipf frequencies proportional to r^-s
 * over ranks r counted from 1 (Section II-A), with the fact keys drawn
 * independently and shuffled over the ids (Section V-A).
 *
 * Element i of a stream with key k is x = mix64(k + (i + 1) * 0x9E3779B97F4A7C15),
 * mix64 being the SplitMix64 output function.  All pointers are device
 * pointers; calls are asynchronous on `stream` (cudaStream_t as void*).
 * Return value: 0 on success, 1 on a bad argument, 5 on a CUDA error.
 */
#ifndef SKX_SYNTH_H
#define SKX_SYNTH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* out[i] = r2id[min{r : cdf[r] > u_i}], u_i = (x_i >> 11) * 2^-53, i in [0, count),
 * for global element indices start + i.  cdf: float64[n] non-decreasing with
 * cdf[n-1] == 1; r2id: int32[n]. */
int skx_synth_zipf(const double *d_cdf, const int32_t *d_r2id, int32_t n, uint64_t key, int64_t start,
                   int64_t count, int32_t *d_out, void *stream);

/* out[i] = lo + (((x_i >> 32) * range) >> 32) for range > 0; int32(x_i >> 32) for range == 0. */
int skx_synth_uniform(uint64_t key, int64_t start, int64_t count, int32_t lo, uint32_t range, int32_t *d_out,
                      void *stream);

/* Row-major table int32[n][width]: element (v, c) is column c's bounded value
 * of draw v * width + c; lo[c], range[c] as in skx_synth_uniform (width <= 64). */
int skx_synth_rows(uint64_t key, int64_t n, int32_t width, const int32_t *h_lo, const uint32_t *h_range,
                   int32_t *d_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SKX_SYNTH_H */
