// probe_core.cuh -- per-row logic of the FK-join probe, shared by the single
// probe (probe.cu) and the batched persistent probe (batch.cu): the gather of
// the needed dimension columns, the filter, the group/SUM/COUNT fold and the
// exact 32-bit hot-key sums of threshold-based processing (Section IV-B).
#pragma once

#include "skx_internal.cuh"

namespace skx {
namespace pcore {

constexpr int kMaxSmemGroups = 4096;
// dynamic shared memory of the split probe's first pass beside groups and hot
// prefix: 4096 staged rows of 10 bytes and two words per bucket (<= 512)
constexpr int64_t kSplitSmemBytes = 4096 * 10 + 512 * 8;

struct PP {
    const int32_t *fk, *measure;
    int64_t F, head;
    const char *rows;
    int32_t N, row_bytes;
    int32_t fcol, flt, gcol, G, pcol;
    int32_t t_hot, t_lane;
    int32_t gather_policy;
    unsigned long long *out;
    unsigned *err;
};

__device__ __forceinline__ int sel4(const int4 &v, int c) {
    return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

__device__ __forceinline__ int2 ld_gather8(const int2 *p, uint64_t pol) {
    int2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.s32 {%0,%1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ int sel2(const int2 &v, int c) { return c == 0 ? v.x : v.y; }

// Row access paths: 16-byte rows (or wider, columns in the first 16 bytes),
// 8-byte rows, or one 4-byte load per needed column.
enum RowPath { kRowGeneric = 0, kRow16 = 1, kRow8 = 2 };

// Gathered values of one dimension row: x = filter column, y = group column, z = payload.
template <int PATH, int AGG>
__device__ __forceinline__ int4 fetch_row(const PP &p, int32_t k, uint64_t pol) {
    const char *r = p.rows + size_t(k) * size_t(p.row_bytes);
    int4 v;
    if (PATH == kRow8) {
        const int2 raw = ld_gather8(reinterpret_cast<const int2 *>(r), pol);
        v.x = p.fcol >= 0 ? sel2(raw, p.fcol) : 0;
        v.y = AGG == SKX_AGG_GROUPBY_SUM ? sel2(raw, p.gcol) : 0;
        v.z = p.pcol >= 0 ? sel2(raw, p.pcol) : 1;
    } else if (PATH == kRow16) {
        const int4 raw = ld_gather16(reinterpret_cast<const int4 *>(r), pol);
        v.x = p.fcol >= 0 ? sel4(raw, p.fcol) : 0;
        v.y = AGG == SKX_AGG_GROUPBY_SUM ? sel4(raw, p.gcol) : 0;
        v.z = p.pcol >= 0 ? sel4(raw, p.pcol) : 1;
    } else {
        const int *ri = reinterpret_cast<const int *>(r);
        v.x = p.fcol >= 0 ? ld_gather4(ri + p.fcol, pol) : 0;
        v.y = AGG == SKX_AGG_GROUPBY_SUM ? ld_gather4(ri + p.gcol, pol) : 0;
        v.z = (AGG != SKX_AGG_COUNT && p.pcol >= 0) ? ld_gather4(ri + p.pcol, pol) : 1;
    }
    v.w = 0;
    return v;
}

__device__ __forceinline__ bool passes(const PP &p, const int4 &v) { return p.fcol < 0 || v.x < p.flt; }

// Hot-key sums are kept exactly in two 32-bit shared words (32-bit shared
// atomics run about 4x faster than 64-bit ones on this part): lo accumulates
// the measures as unsigned 32-bit values, hi counts the wrap-arounds of lo
// minus the number of negative measures.  Then sum = lo + 2^32 * hi exactly,
// because a measure m < 0 enters lo as m + 2^32.
struct HotRef {
    uint32_t *lo;
    int32_t *hi;
};

template <int AGG>
__device__ __forceinline__ void hot_add(HotRef h, int32_t m) {
    if (AGG == SKX_AGG_COUNT) {
        atomicAdd(h.lo, 1u);  // a CTA sees fewer than 2^32 rows
        return;
    }
    const uint32_t u = (uint32_t)m;
    const uint32_t old = atomicAdd(h.lo, u);
    const int d = (int)(old + u < old) - (int)(m < 0);
    if (d) atomicAdd(h.hi, d);
}

__device__ __forceinline__ unsigned long long hot_value(uint32_t lo, int32_t hi) {
    return (unsigned long long)lo + ((unsigned long long)(long long)hi << 32);
}

// Group sums of one CTA as two 32-bit shared words per group (32-bit shared
// atomics are native; a 64-bit shared add is several times slower): lo takes
// the low words of the 64-bit products, hi their high words plus one for each
// carry out of lo, which the returning add on lo reveals exactly.  So
// sum = lo + 2^32 * hi (mod 2^64), bit for bit.
struct GrpRef {
    uint32_t *lo, *hi;  // G each
};

__device__ __forceinline__ void add64_split(uint32_t *lo, uint32_t *hi, unsigned long long x) {
    const uint32_t xl = (uint32_t)x, xh = (uint32_t)(x >> 32);
    const uint32_t old = atomicAdd(lo, xl);
    const uint32_t inc = xh + (old + xl < old ? 1u : 0u);
    if (inc) atomicAdd(hi, inc);
}

// Fold of one fact row (measure m) whose gathered values are v: the product is
// formed as one signed 32 x 32 -> 64 multiply.
template <int AGG, bool GSMEM>
__device__ __forceinline__ void fold_row(const PP &p, const int4 &v, int32_t m, unsigned long long &acc, GrpRef g) {
    if (!passes(p, v)) return;
    if (AGG == SKX_AGG_COUNT) {
        acc += 1ull;
        return;
    }
    const unsigned long long prod = (unsigned long long)((long long)m * (long long)v.z);
    if (AGG == SKX_AGG_SUM) {
        acc += prod;
        return;
    }
    if ((uint32_t)v.y < (uint32_t)p.G) {
        if (GSMEM)
            add64_split(g.lo + v.y, g.hi + v.y, prod);
        else
            atomicAdd(p.out + v.y, prod);
    } else {
        raise_error(p.err, kErrGroupRange);
    }
}

// Fold of a hot row's 64-bit measure sum (or count) s.
template <int AGG, bool GSMEM>
__device__ __forceinline__ void fold_sum(const PP &p, const int4 &v, unsigned long long s, unsigned long long &acc,
                                         GrpRef g) {
    if (!passes(p, v)) return;
    if (AGG == SKX_AGG_COUNT) {
        acc += s;
        return;
    }
    const unsigned long long prod = s * (unsigned long long)(long long)v.z;
    if (AGG == SKX_AGG_SUM) {
        acc += prod;
        return;
    }
    if ((uint32_t)v.y < (uint32_t)p.G) {
        if (GSMEM)
            add64_split(g.lo + v.y, g.hi + v.y, prod);
        else
            atomicAdd(p.out + v.y, prod);
    } else {
        raise_error(p.err, kErrGroupRange);
    }
}

// CTA epilogue: shared group sums into the output (one global add per nonzero
// group), or the register sum of COUNT / SUM reduced per warp.
template <int AGG, bool GSMEM>
__device__ __forceinline__ void flush_groups(const PP &p, unsigned long long acc, GrpRef g) {
    if (AGG == SKX_AGG_GROUPBY_SUM) {
        if (GSMEM) {
            __syncthreads();
            for (int k = threadIdx.x; k < p.G; k += blockDim.x) {
                const unsigned long long v = (unsigned long long)g.lo[k] + ((unsigned long long)g.hi[k] << 32);
                if (v) atomicAdd(p.out + k, v);
            }
        }
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31u) == 0 && acc) atomicAdd(p.out, acc);
    }
}

// Four rows at once: their shared atomics are issued back to back and only
// then are the returned words inspected, so the atomics' latencies overlap
// instead of each row waiting for its own before the next one starts.
template <int AGG, bool GSMEM>
__device__ __forceinline__ void fold4(const PP &p, const int4 (&v)[4], const int32_t (&m)[4], const bool (&use)[4],
                                      unsigned long long &acc, GrpRef g) {
    bool ok[4];
    unsigned long long prod[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        ok[j] = use[j] && passes(p, v[j]);
        prod[j] = (unsigned long long)((long long)m[j] * (long long)v[j].z);
    }
    if (AGG == SKX_AGG_COUNT) {
#pragma unroll
        for (int j = 0; j < 4; ++j) acc += ok[j] ? 1ull : 0ull;
        return;
    }
    if (AGG == SKX_AGG_SUM) {
#pragma unroll
        for (int j = 0; j < 4; ++j) acc += ok[j] ? prod[j] : 0ull;
        return;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (ok[j] && (uint32_t)v[j].y >= (uint32_t)p.G) {
            raise_error(p.err, kErrGroupRange);
            ok[j] = false;
        }
    if (!GSMEM) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j]) atomicAdd(p.out + v[j].y, prod[j]);
        return;
    }
    uint32_t old[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) old[j] = ok[j] ? atomicAdd(g.lo + v[j].y, (uint32_t)prod[j]) : 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t xl = (uint32_t)prod[j];
        const uint32_t inc = (uint32_t)(prod[j] >> 32) + (old[j] + xl < old[j] ? 1u : 0u);
        if (ok[j] && inc) atomicAdd(g.hi + v[j].y, inc);
    }
}

struct HotArrays {
    uint32_t *lo, *lane_lo;
    int32_t *hi, *lane_hi;
};

// Hot-key adds of four rows (use[j]: key[j] < t_hot), batched like fold4.
template <int AGG>
__device__ __forceinline__ void hot_add4(const PP &p, const HotArrays &h, const int32_t (&k)[4],
                                         const int32_t (&m)[4], const bool (&use)[4], unsigned lane) {
    uint32_t *lo[4];
    int32_t *hi[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool ln = (uint32_t)k[j] < (uint32_t)p.t_lane;
        const size_t li = (size_t(k[j]) << 5) + lane;
        lo[j] = ln ? h.lane_lo + li : h.lo + k[j];
        hi[j] = ln ? h.lane_hi + li : h.hi + k[j];
    }
    if (AGG == SKX_AGG_COUNT) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (use[j]) atomicAdd(lo[j], 1u);
        return;
    }
    uint32_t old[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) old[j] = use[j] ? atomicAdd(lo[j], (uint32_t)m[j]) : 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t u = (uint32_t)m[j];
        const int d = (int)(old[j] + u < old[j]) - (int)(m[j] < 0);
        if (use[j] && d) atomicAdd(hi[j], d);
    }
}

// One fact row: a hot key's measure goes to its shared per-key sum, any other
// key's row (already gathered) is folded into the group sums (the single,
// split and batched probes).
template <int AGG, int PATH, bool GSMEM>
__device__ __forceinline__ void handle_row(const PP &p, int32_t k, int32_t m, const int4 &row, unsigned long long &acc,
                                           GrpRef g, const HotArrays &h, unsigned lane) {
    if ((uint32_t)k < (uint32_t)p.t_hot) {
        if ((uint32_t)k < (uint32_t)p.t_lane) {
            const size_t i = (size_t(k) << 5) + lane;
            hot_add<AGG>(HotRef{h.lane_lo + i, h.lane_hi + i}, m);
        } else {
            hot_add<AGG>(HotRef{h.lo + k, h.hi + k}, m);
        }
    } else if ((uint32_t)k < (uint32_t)p.N) {
        fold_row<AGG, GSMEM>(p, row, m, acc, g);
    } else {
        raise_error(p.err, kErrKeyRange);
    }
}


}  // namespace pcore

// The probe with the split of Section IV-B (probe_split.cu): both passes
// enqueued on st with their stream-ordered scratch.  *ran is false when the
// tuning asks for no split or the scratch could not be allocated; nothing was
// enqueued then and the caller runs the unsplit probe.  Needs the 16-byte
// vector path (fk and measure at the same offset mod 16).
cudaError_t launch_probe_split(const pcore::PP &p, int agg, int path, bool gsmem, const skx_tuning &t,
                               cudaStream_t st, bool *ran);

}  // namespace skx
