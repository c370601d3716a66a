// remap.cu -- apply the permutation index to both sides of the join.
//
//   remap    fk_out[i] = rank[fk_in[i]]        recode of column C into C'
//                                              (Section III-A)
//   reorder  rows_out[r] = rows_in[perm[r]]    permuted copy of the dimension
//                                              rows (Section III-B)
//   materialize  out[i] = rows[fk[i]][col]     query Q1 over either layout
//                                              (Sections I, IV-A)
//
// GB300 design: remap streams the fact column with 16-byte loads and stores
// marked L2 evict-first, so that rank[] (4 B per id) stays L2-resident for
// the random gathers; under skew most gathers hit a few hot lines.  Reorder
// gives every 16-byte chunk of the output its own lane, so stores are fully
// coalesced and each source row is read as one contiguous run.
#include "skx_internal.cuh"

namespace skx {
namespace {

constexpr int kRemapBlock = 512;
constexpr int kQueryRows = 4;  // rows per thread per step of the query copy
constexpr int kRemapUnroll = 2;

__device__ __forceinline__ int32_t remap_one(int32_t k, const int32_t *__restrict__ rank, int32_t N, unsigned *err) {
    if ((uint32_t)k < (uint32_t)N) return __ldg(rank + k);
    raise_error(err, kErrKeyRange);
    return k;
}

template <bool INPLACE>
__global__ void __launch_bounds__(kRemapBlock)
    k_remap(const int32_t *__restrict__ rank, int32_t N, const int32_t *in, int32_t *out, int64_t F, int64_t head,
            unsigned *err) {
    const uint64_t pol = policy_evict_first();
    const int4 *vin = reinterpret_cast<const int4 *>(in + head);
    int4 *vout = reinterpret_cast<int4 *>(out + head);
    const int64_t nvec = (F - head) >> 2;
    const int64_t tid = int64_t(blockIdx.x) * kRemapBlock + threadIdx.x;
    const int64_t nthr = int64_t(gridDim.x) * kRemapBlock;
    // software pipeline: the next vectors are in flight while this one's rank gathers resolve
    int4 nk[kRemapUnroll];
#pragma unroll
    for (int u = 0; u < kRemapUnroll; ++u) {
        const int64_t i = tid + u * nthr;
        if (i < nvec) nk[u] = INPLACE ? ld_stream16_rw(vin + i, pol) : ld_stream16(vin + i, pol);
    }
    for (int64_t base = tid; base < nvec; base += nthr * kRemapUnroll) {
        int4 k[kRemapUnroll];
#pragma unroll
        for (int u = 0; u < kRemapUnroll; ++u) k[u] = nk[u];
        int4 r[kRemapUnroll];
#pragma unroll
        for (int u = 0; u < kRemapUnroll; ++u) {
            if (base + u * nthr < nvec) {
                r[u].x = remap_one(k[u].x, rank, N, err);
                r[u].y = remap_one(k[u].y, rank, N, err);
                r[u].z = remap_one(k[u].z, rank, N, err);
                r[u].w = remap_one(k[u].w, rank, N, err);
            }
        }
#pragma unroll
        for (int u = 0; u < kRemapUnroll; ++u) {
            // in place: vector i + U*nthr is read before any thread writes it (each vector
            // is read and written by the same thread, in this order)
            const int64_t i = base + (kRemapUnroll + u) * nthr;
            if (i < nvec) nk[u] = INPLACE ? ld_stream16_rw(vin + i, pol) : ld_stream16(vin + i, pol);
        }
#pragma unroll
        for (int u = 0; u < kRemapUnroll; ++u) {
            const int64_t i = base + u * nthr;
            if (i < nvec) st_stream16(vout + i, r[u], pol);
        }
    }
    if (tid < 8) {  // unaligned head (< 4) and ragged tail (< 4)
        const int64_t tail0 = head + (nvec << 2);
        int64_t idx = -1;
        if (tid < head) idx = tid;
        else if (tid >= 4 && tail0 + (tid - 4) < F) idx = tail0 + (tid - 4);
        if (idx >= 0) out[idx] = remap_one(in[idx], rank, N, err);
    }
}

// Unaligned in/out pair (different offsets mod 16 bytes): plain 4-byte path.
__global__ void __launch_bounds__(kRemapBlock)
    k_remap_scalar(const int32_t *__restrict__ rank, int32_t N, const int32_t *in, int32_t *out, int64_t F,
                   unsigned *err) {
    for (int64_t i = int64_t(blockIdx.x) * kRemapBlock + threadIdx.x; i < F; i += int64_t(gridDim.x) * kRemapBlock)
        out[i] = remap_one(in[i], rank, N, err);
}

// Q1 materialisation (Sections I, IV-A): out[i] = column col of row fk[i]
// (int32).  The fact keys stream with 16-byte evict-first loads, one 4-byte
// gather per key, 16-byte evict-first stores; the next vectors' keys are in
// flight while this one's gathers resolve.  Keys outside [0, N) give 0 and
// are flagged.
__device__ __forceinline__ int32_t gather_col(const int32_t *__restrict__ rows, int64_t words, int32_t col, int32_t k,
                                              int32_t N, unsigned *err) {
    if ((uint32_t)k < (uint32_t)N) return __ldg(rows + int64_t(k) * words + col);
    raise_error(err, kErrKeyRange);
    return 0;
}

__global__ void __launch_bounds__(kRemapBlock)
    k_materialize(const int32_t *__restrict__ rows, int64_t words, int32_t col, int32_t N,
                  const int32_t *__restrict__ fk, int32_t *__restrict__ out, int64_t F, int64_t head,
                  unsigned *err) {
    const uint64_t pol = policy_evict_first();
    const int4 *vin = reinterpret_cast<const int4 *>(fk + head);
    int4 *vout = reinterpret_cast<int4 *>(out + head);
    const int64_t nvec = (F - head) >> 2;
    const int64_t tid = int64_t(blockIdx.x) * kRemapBlock + threadIdx.x;
    const int64_t nthr = int64_t(gridDim.x) * kRemapBlock;
    int4 nk[kRemapUnroll];
#pragma unroll
    for (int u = 0; u < kRemapUnroll; ++u) {
        const int64_t i = tid + u * nthr;
        if (i < nvec) nk[u] = ld_stream16(vin + i, pol);
    }
    for (int64_t base = tid; base < nvec; base += nthr * kRemapUnroll) {
        int4 k[kRemapUnroll], r[kRemapUnroll];
#pragma unroll
        for (int u = 0; u < kRemapUnroll; ++u) k[u] = nk[u];
#pragma unroll
        for (int u = 0; u < kRemapUnroll; ++u) {
            if (base + u * nthr < nvec) {
                r[u].x = gather_col(rows, words, col, k[u].x, N, err);
                r[u].y = gather_col(rows, words, col, k[u].y, N, err);
                r[u].z = gather_col(rows, words, col, k[u].z, N, err);
                r[u].w = gather_col(rows, words, col, k[u].w, N, err);
            }
        }
#pragma unroll
        for (int u = 0; u < kRemapUnroll; ++u) {
            const int64_t i = base + (kRemapUnroll + u) * nthr;
            if (i < nvec) nk[u] = ld_stream16(vin + i, pol);
        }
#pragma unroll
        for (int u = 0; u < kRemapUnroll; ++u) {
            const int64_t i = base + u * nthr;
            if (i < nvec) st_stream16(vout + i, r[u], pol);
        }
    }
    if (tid < 8) {  // unaligned head (< 4) and ragged tail (< 4)
        const int64_t tail0 = head + (nvec << 2);
        int64_t idx = -1;
        if (tid < head) idx = tid;
        else if (tid >= 4 && tail0 + (tid - 4) < F) idx = tail0 + (tid - 4);
        if (idx >= 0) out[idx] = gather_col(rows, words, col, fk[idx], N, err);
    }
}

// fk and out at different offsets mod 16 bytes: plain 4-byte path
__global__ void __launch_bounds__(kRemapBlock)
    k_materialize_scalar(const int32_t *__restrict__ rows, int64_t words, int32_t col, int32_t N,
                         const int32_t *__restrict__ fk, int32_t *__restrict__ out, int64_t F, unsigned *err) {
    for (int64_t i = int64_t(blockIdx.x) * kRemapBlock + threadIdx.x; i < F; i += int64_t(gridDim.x) * kRemapBlock)
        out[i] = gather_col(rows, words, col, fk[i], N, err);
}

// 16-byte read of a source row of 64 bytes or more through the read-only path,
// with the L2 told to fetch 64 bytes rather than a 128-byte line (half of
// which would be another, randomly placed row)
__device__ __forceinline__ int4 ld_row16_p64(const int4 *p) {
    int4 v;
    asm volatile("ld.global.nc.L2::64B.v4.s32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__global__ void __launch_bounds__(512)
    k_reorder16(const int32_t *__restrict__ perm, int32_t N, const int4 *__restrict__ in, int4 *__restrict__ out,
                int32_t chunks_per_row) {
    const int64_t total = int64_t(N) * chunks_per_row;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < total; j += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = j / chunks_per_row;
        const int64_t c = j - r * chunks_per_row;
        const int32_t src = __ldg(perm + r);
        if ((uint32_t)src < (uint32_t)N) out[j] = ld_row16_p64(in + int64_t(src) * chunks_per_row + c);
    }
}

template <typename Chunk>
__global__ void __launch_bounds__(512)
    k_reorder(const int32_t *__restrict__ perm, int32_t N, const Chunk *__restrict__ in, Chunk *__restrict__ out,
              int32_t chunks_per_row) {
    const int64_t total = int64_t(N) * chunks_per_row;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < total; j += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = j / chunks_per_row;
        const int64_t c = j - r * chunks_per_row;
        const int32_t src = __ldg(perm + r);
        if ((uint32_t)src < (uint32_t)N) out[j] = in[int64_t(src) * chunks_per_row + c];
    }
}

// Permuted copy of selected columns (Section III-B): out[r][c] = in[src(r)][cols[c]],
// src(r) = perm[r] (or r when perm is null: the identity-order copy of the plain layout).
struct ColList {
    int32_t c[16];
};

template <int NC>
__global__ void __launch_bounds__(512)
    k_reorder_cols(const int32_t *__restrict__ perm, int32_t N, const int32_t *__restrict__ in, int32_t words,
                   ColList cols, int32_t ncols, int32_t *__restrict__ out) {
    const bool wide = words >= 16;  // rows of 64 bytes or more: fetch 64 bytes per miss
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < N; r += int64_t(gridDim.x) * blockDim.x) {
        const int32_t src = perm ? __ldg(perm + r) : (int32_t)r;
        if ((uint32_t)src >= (uint32_t)N) continue;
        const int32_t *row = in + int64_t(src) * words;
        auto rd = [wide](const int32_t *q) { return wide ? ld_row4_p64(q) : __ldg(q); };
        if (NC == 4) {
            int4 v;
            v.x = rd(row + cols.c[0]);
            v.y = rd(row + cols.c[1]);
            v.z = rd(row + cols.c[2]);
            v.w = rd(row + cols.c[3]);
            reinterpret_cast<int4 *>(out)[r] = v;
        } else if (NC == 2) {
            int2 v;
            v.x = rd(row + cols.c[0]);
            v.y = rd(row + cols.c[1]);
            reinterpret_cast<int2 *>(out)[r] = v;
        } else {
            for (int c = 0; c < ncols; ++c) out[r * ncols + c] = rd(row + cols.c[c]);
        }
    }
}

// Query-specific copy (Sections I and III-B): the predicate is evaluated once per
// dimension row, as for the Q2 bitmap, and folded into the copy:
// out[r] = {passes ? group : sentinel, payload}.
// Each thread takes U rows per step (grid stride) and issues all of their perm
// loads, then all of their row loads, before it writes any, so U rows' latencies
// overlap.  VEC: the used columns lie in one aligned 16-byte chunk of a 16-byte
// aligned row (chunk index `chunk`), read with one load.
__device__ __forceinline__ int32_t pick4(const int4 &c, int i) {
    return i == 0 ? c.x : (i == 1 ? c.y : (i == 2 ? c.z : c.w));
}

// With out4, each row is also written packed in 32 bits (the query's two values in
// one word, so that twice as many rows share a cache line): key << (32 - kbits) |
// the payload's low 32 - kbits bits (0 for a filtered row), key = group or sentinel.  A row whose key is
// outside [0, sentinel] or whose payload needs more bits gets the escape code
// (key field all ones); its values stay in the 8-byte copy.
template <int U, bool VEC>
__global__ void __launch_bounds__(512, VEC ? 4 : 2)
    k_reorder_query(const int32_t *__restrict__ perm, int32_t N, const int32_t *__restrict__ in, int32_t words,
                    int32_t fcol, int32_t flt, int32_t gcol, int32_t pcol, int32_t sentinel, int32_t chunk,
                    int2 *__restrict__ out, uint32_t *__restrict__ out4, int32_t kbits, unsigned *err) {
    const bool wide = words >= 16;  // rows of 64 bytes or more: fetch 64 bytes per miss
    const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
    for (int64_t r0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r0 < N; r0 += nthr * U) {
        int32_t src[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = r0 + u * nthr;
            src[u] = r < N ? (perm ? __ldg(perm + r) : (int32_t)r) : -1;
        }
        int32_t fv[U], gv[U], pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            fv[u] = 0;
            gv[u] = 0;
            pv[u] = 1;
            if ((uint32_t)src[u] >= (uint32_t)N) continue;
            const int32_t *row = in + int64_t(src[u]) * words;
            if (VEC) {
                const int4 *q = reinterpret_cast<const int4 *>(row) + chunk;
                const int4 c = wide ? ld_row16_p64(q) : __ldg(q);
                if (fcol >= 0) fv[u] = pick4(c, fcol & 3);
                if (gcol >= 0) gv[u] = pick4(c, gcol & 3);
                if (pcol >= 0) pv[u] = pick4(c, pcol & 3);
            } else {
                auto rd = [wide](const int32_t *a) { return wide ? ld_row4_p64(a) : __ldg(a); };
                if (fcol >= 0) fv[u] = rd(row + fcol);
                if (gcol >= 0) gv[u] = rd(row + gcol);
                if (pcol >= 0) pv[u] = rd(row + pcol);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = r0 + u * nthr;
            if (r >= N || (uint32_t)src[u] >= (uint32_t)N) continue;
            const bool pass = fcol < 0 || fv[u] < flt;
            // a passing row's group must lie in [0, G) (G = sentinel); the probe over the copy
            // could not tell a group >= G from a filtered row
            if (pass && gcol >= 0 && (uint32_t)gv[u] >= (uint32_t)sentinel) raise_error(err, kErrGroupRange);
            const int32_t key = pass ? gv[u] : sentinel;
            out[r] = make_int2(key, pv[u]);
            if (out4) {  // a filtered row's payload is never used: it is packed as 0
                const int pb = 32 - kbits;
                const int32_t half = int32_t(1) << (pb - 1);
                const int32_t pay = pass ? pv[u] : 0;
                const bool fits = (uint32_t)key <= (uint32_t)sentinel && pay >= -half && pay < half;
                const uint32_t esc = (1u << kbits) - 1u;
                out4[r] = fits ? ((uint32_t)key << pb) | ((uint32_t)pay & ((1u << pb) - 1u)) : esc << pb;
            }
        }
    }
}

int grid_for(int64_t work_items, int block, int per_sm) {
    const int sms = device_sm_count();
    int64_t want = (work_items + block - 1) / block;
    int64_t cap = (int64_t)sms * per_sm;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

cudaError_t launch_remap(const int32_t *d_rank, int32_t N, const int32_t *d_in, int32_t *d_out, int64_t F,
                         unsigned *d_err, cudaStream_t st) {
    if (F <= 0) return cudaSuccess;
    const uintptr_t ai = reinterpret_cast<uintptr_t>(d_in) & 15u, ao = reinterpret_cast<uintptr_t>(d_out) & 15u;
    if (ai != ao) {
        k_remap_scalar<<<grid_for(F, kRemapBlock, 4), kRemapBlock, 0, st>>>(d_rank, N, d_in, d_out, F, d_err);
        note_launches(1);
        return cudaGetLastError();
    }
    const int64_t mis = (int64_t)(ai >> 2);
    const int64_t head = mis ? (F < 4 - mis ? F : 4 - mis) : 0;
    const int64_t nvec = (F - head) >> 2;
    int grid = grid_for((nvec + kRemapUnroll - 1) / kRemapUnroll, kRemapBlock, 2048 / kRemapBlock);
    if (d_in == d_out)
        k_remap<true><<<grid, kRemapBlock, 0, st>>>(d_rank, N, d_in, d_out, F, head, d_err);
    else
        k_remap<false><<<grid, kRemapBlock, 0, st>>>(d_rank, N, d_in, d_out, F, head, d_err);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_materialize(const void *d_rows, int32_t N, int32_t row_bytes, int32_t col, const int32_t *d_fk,
                               int64_t F, int32_t *d_out, unsigned *d_err, cudaStream_t st) {
    if (F <= 0) return cudaSuccess;
    const int32_t *rows = static_cast<const int32_t *>(d_rows);
    const int64_t words = row_bytes / 4;
    const uintptr_t ai = reinterpret_cast<uintptr_t>(d_fk) & 15u, ao = reinterpret_cast<uintptr_t>(d_out) & 15u;
    if (ai != ao) {
        k_materialize_scalar<<<grid_for(F, kRemapBlock, 4), kRemapBlock, 0, st>>>(rows, words, col, N, d_fk, d_out, F,
                                                                                  d_err);
        note_launches(1);
        return cudaGetLastError();
    }
    const int64_t mis = (int64_t)(ai >> 2);
    const int64_t head = mis ? (F < 4 - mis ? F : 4 - mis) : 0;
    const int64_t nvec = (F - head) >> 2;
    const int grid = grid_for((nvec + kRemapUnroll - 1) / kRemapUnroll, kRemapBlock, 2048 / kRemapBlock);
    k_materialize<<<grid, kRemapBlock, 0, st>>>(rows, words, col, N, d_fk, d_out, F, head, d_err);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_reorder_columns(const int32_t *d_perm, int32_t N, const void *d_in, int32_t row_bytes,
                                   const int32_t *cols, int32_t ncols, void *d_out, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    ColList cl{};
    for (int i = 0; i < ncols; ++i) cl.c[i] = cols[i];
    const int32_t words = row_bytes / 4;
    const int grid = grid_for(N, 512, 4);
    const int32_t *in = static_cast<const int32_t *>(d_in);
    int32_t *out = static_cast<int32_t *>(d_out);
    if (ncols == 4 && aligned16(d_out))
        k_reorder_cols<4><<<grid, 512, 0, st>>>(d_perm, N, in, words, cl, ncols, out);
    else if (ncols == 2 && (reinterpret_cast<uintptr_t>(d_out) & 7u) == 0)
        k_reorder_cols<2><<<grid, 512, 0, st>>>(d_perm, N, in, words, cl, ncols, out);
    else
        k_reorder_cols<0><<<grid, 512, 0, st>>>(d_perm, N, in, words, cl, ncols, out);
    note_launches(1);
    return cudaGetLastError();
}

int32_t packed_key_bits(const skx_query &q) {
    const int64_t G = q.agg == SKX_AGG_GROUPBY_SUM ? q.num_groups : 1;
    int32_t b = 1;
    while ((int64_t(1) << b) < G + 2) ++b;
    return b;
}

cudaError_t launch_reorder_query(const int32_t *d_perm, int32_t N, const void *d_in, int32_t row_bytes,
                                 const skx_query &q, void *d_out, unsigned *d_err, cudaStream_t st,
                                 uint32_t *d_out4) {
    if (N <= 0) return cudaSuccess;
    const bool grp = q.agg == SKX_AGG_GROUPBY_SUM;
    const int32_t sentinel = grp ? q.num_groups : 1;
    const int32_t words = row_bytes / 4, fcol = q.filter_col, gcol = grp ? q.group_col : -1,
                  pcol = q.agg == SKX_AGG_COUNT ? -1 : q.payload_col;
    // one 16-byte load per row when every used column is in the same aligned chunk
    int32_t chunk = -1;
    bool vec = words % 4 == 0 && aligned16(d_in);
    for (int32_t c : {fcol, gcol, pcol}) {
        if (c < 0) continue;
        if (chunk < 0) chunk = c / 4;
        vec = vec && c / 4 == chunk;
    }
    if (chunk < 0) chunk = 0;
    const int32_t *in = static_cast<const int32_t *>(d_in);
    int2 *out = static_cast<int2 *>(d_out);
    // four 512-thread CTAs per SM with one vector load a row (at most 32 registers), two otherwise
    const int grid = grid_for((N + kQueryRows - 1) / kQueryRows, 512, vec ? 4 : 2);
    const int32_t kbits = packed_key_bits(q);
    if (vec)
        k_reorder_query<kQueryRows, true><<<grid, 512, 0, st>>>(d_perm, N, in, words, fcol, q.filter_lt, gcol, pcol,
                                                                sentinel, chunk, out, d_out4, kbits, d_err);
    else
        k_reorder_query<kQueryRows, false><<<grid, 512, 0, st>>>(d_perm, N, in, words, fcol, q.filter_lt, gcol,
                                                                 pcol, sentinel, chunk, out, d_out4, kbits, d_err);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_reorder(const int32_t *d_perm, int32_t N, const void *d_in, void *d_out, int32_t row_bytes,
                           cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    if (row_bytes % 16 == 0 && aligned16(d_in) && aligned16(d_out)) {
        const int32_t w = row_bytes / 16;
        if (row_bytes >= 64)  // wide rows: fetch 64 bytes per missed row, not a 128-byte line
            k_reorder16<<<grid_for(int64_t(N) * w, 512, 4), 512, 0, st>>>(d_perm, N, static_cast<const int4 *>(d_in),
                                                                          static_cast<int4 *>(d_out), w);
        else
            k_reorder<int4><<<grid_for(int64_t(N) * w, 512, 4), 512, 0, st>>>(
                d_perm, N, static_cast<const int4 *>(d_in), static_cast<int4 *>(d_out), w);
    } else {
        const int32_t w = row_bytes / 4;
        k_reorder<int32_t><<<grid_for(int64_t(N) * w, 512, 4), 512, 0, st>>>(
            d_perm, N, static_cast<const int32_t *>(d_in), static_cast<int32_t *>(d_out), w);
    }
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace skx
