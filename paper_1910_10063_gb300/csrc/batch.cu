// batch.cu -- many FK-join probes in one persistent launch.
//
// A batch is a list of probe descriptors (fact keys, measures, query, output)
// against one dimension table.  The fact rows of all queries are cut into
// tiles of `tile_rows` rows; tile t of the whole batch belongs to the query
// whose tile range contains t (a prefix table of tiles per query).  A
// persistent grid pulls tiles from one global atomic counter, so queries of
// very different sizes (lognormal batch sizes from 1K to 20M rows) balance
// across the SMs without any host involvement.  Each tile is processed with
// the same row logic as the single probe (probe_core.cuh), including the
// shared-memory hot prefix of threshold-based processing (Section IV-B), and
// flushes its group partials with global atomics at its end, so no state
// carries from one tile to the next and COUNT, SUM and GROUP BY queries mix
// freely.  A small prologue kernel clears every output and the tile counter;
// the two launches can be captured once in a CUDA graph and replayed.
#include <algorithm>
#include <vector>

#include "probe_core.cuh"

struct skx_batch_plan;

namespace skx {
namespace {

using namespace pcore;

struct BatchArgs {
    const BatchDesc *desc;
    const uint32_t *tile_start;  // n + 1 entries
    uint32_t *counter;
    int32_t n;
    uint32_t total_tiles;
    int32_t tile_rows;
    const char *rows;
    int32_t N, row_bytes;
    int32_t max_groups;  // shared-memory group slots
    int32_t t_hot, t_lane, gather_policy;
    unsigned *err;
};

__global__ void k_batch_clear(const BatchDesc *__restrict__ desc, int32_t n, uint32_t *counter, int clear_outputs) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
    if (!clear_outputs) return;
    for (int q = blockIdx.x; q < n; q += gridDim.x) {
        const BatchDesc d = desc[q];
        for (int g = threadIdx.x; g < d.nout; g += blockDim.x) d.out[g] = 0;
    }
}

template <int AGG, int PATH>
__device__ __forceinline__ void batch_rows(const PP &p, unsigned long long &acc, GrpRef g,
                                           const HotArrays &h, uint64_t pol_s, uint64_t pol_g, bool vec) {
    const unsigned lane = lane_id();
    if (vec) {
        const int4 *fk4 = reinterpret_cast<const int4 *>(p.fk);
        const int4 *m4 = reinterpret_cast<const int4 *>(AGG == SKX_AGG_COUNT ? p.fk : p.measure);
        const int64_t nvec = p.F >> 2;
        int4 nk = make_int4(0, 0, 0, 0), nm = make_int4(0, 0, 0, 0);
        int64_t v = threadIdx.x;
        if (v < nvec) {
            nk = ld_stream16(fk4 + v, pol_s);
            if (AGG != SKX_AGG_COUNT) nm = ld_stream16(m4 + v, pol_s);
        }
        for (; v < nvec; v += blockDim.x) {
            const int32_t key[4] = {nk.x, nk.y, nk.z, nk.w};
            const int32_t mea[4] = {nm.x, nm.y, nm.z, nm.w};
            int4 row[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t k = (uint32_t)key[j];
                row[j] = make_int4(0, 0, 0, 0);
                if (k >= (uint32_t)p.t_hot && k < (uint32_t)p.N) row[j] = fetch_row<PATH, AGG>(p, key[j], pol_g);
            }
            const int64_t nv = v + blockDim.x;
            if (nv < nvec) {
                nk = ld_stream16(fk4 + nv, pol_s);
                if (AGG != SKX_AGG_COUNT) nm = ld_stream16(m4 + nv, pol_s);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) handle_row<AGG, PATH, true>(p, key[j], mea[j], row[j], acc, g, h, lane);
        }
        const int64_t tail0 = nvec << 2;
        if (threadIdx.x < p.F - tail0) {
            const int64_t i = tail0 + threadIdx.x;
            const int32_t k = p.fk[i];
            const int32_t m = AGG == SKX_AGG_COUNT ? 0 : p.measure[i];
            int4 row = make_int4(0, 0, 0, 0);
            if ((uint32_t)k >= (uint32_t)p.t_hot && (uint32_t)k < (uint32_t)p.N) row = fetch_row<PATH, AGG>(p, k, pol_g);
            handle_row<AGG, PATH, true>(p, k, m, row, acc, g, h, lane);
        }
    } else {
        for (int64_t i = threadIdx.x; i < p.F; i += blockDim.x) {
            const int32_t k = ld_stream4(p.fk + i, pol_s);
            const int32_t m = AGG == SKX_AGG_COUNT ? 0 : ld_stream4(p.measure + i, pol_s);
            int4 row = make_int4(0, 0, 0, 0);
            if ((uint32_t)k >= (uint32_t)p.t_hot && (uint32_t)k < (uint32_t)p.N) row = fetch_row<PATH, AGG>(p, k, pol_g);
            handle_row<AGG, PATH, true>(p, k, m, row, acc, g, h, lane);
        }
    }
}

template <int AGG, int PATH>
__device__ __forceinline__ void batch_epilogue(const PP &p, unsigned long long acc, GrpRef g,
                                               const HotArrays &h, uint64_t pol_g, unsigned long long *s_red) {
    for (int k = threadIdx.x; k < p.t_hot; k += blockDim.x) {
        unsigned long long s = hot_value(h.lo[k], h.hi[k]);
        if (k < p.t_lane) {
#pragma unroll 8
            for (int l = 0; l < 32; ++l) s += hot_value(h.lane_lo[(size_t(k) << 5) + l], h.lane_hi[(size_t(k) << 5) + l]);
        }
        if (s == 0) continue;
        fold_sum<AGG, true>(p, fetch_row<PATH, AGG>(p, k, pol_g), s, acc, g);
    }
    if (AGG == SKX_AGG_GROUPBY_SUM) {
        __syncthreads();
        for (int k = threadIdx.x; k < p.G; k += blockDim.x) {
            const unsigned long long v = (unsigned long long)g.lo[k] + ((unsigned long long)g.hi[k] << 32);
            if (v) atomicAdd(p.out + k, v);
        }
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane_id() == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
            if (t) atomicAdd(p.out, t);
        }
    }
}

template <int PATH>
__global__ void __launch_bounds__(512) k_probe_batch(BatchArgs a) {
    extern __shared__ unsigned long long smem[];
    __shared__ uint32_t s_tile;
    __shared__ int32_t s_q;
    __shared__ BatchDesc s_d;
    __shared__ unsigned long long s_red[16];
    // group sums: two 32-bit words per group slot (low word, and high word with the carries)
    GrpRef g;
    g.lo = reinterpret_cast<uint32_t *>(smem);
    g.hi = g.lo + a.max_groups;
    HotArrays h;
    h.lo = reinterpret_cast<uint32_t *>(smem + a.max_groups);
    h.hi = reinterpret_cast<int32_t *>(h.lo + a.t_hot);
    h.lane_lo = reinterpret_cast<uint32_t *>(h.hi + a.t_hot);
    h.lane_hi = reinterpret_cast<int32_t *>(h.lane_lo + (a.t_lane << 5));
    const int nsm = a.max_groups + a.t_hot + (a.t_lane << 5);
    const uint64_t pol_s = policy_evict_first();
    const uint64_t pol_g = policy_by_code(a.gather_policy);

    while (true) {
        if (threadIdx.x == 0) {
            const uint32_t t = atomicAdd(a.counter, 1u);
            s_tile = t;
            if (t < a.total_tiles) {
                // last query whose first tile is <= t
                int lo = 0, hi = a.n - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.tile_start[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                s_q = lo;
                s_d = a.desc[lo];
            }
        }
        for (int i = threadIdx.x; i < nsm; i += blockDim.x) smem[i] = 0;
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= a.total_tiles) break;
        const BatchDesc d = s_d;
        const int64_t lo = int64_t(t - a.tile_start[s_q]) * a.tile_rows;
        const int64_t hi = min(lo + int64_t(a.tile_rows), d.F);
        PP p{};
        p.fk = d.fk + lo;
        p.measure = d.measure ? d.measure + lo : nullptr;
        p.F = hi - lo;
        p.head = 0;
        p.rows = a.rows;
        p.N = a.N;
        p.row_bytes = a.row_bytes;
        p.fcol = d.fcol;
        p.flt = d.flt;
        p.gcol = d.gcol;
        p.G = d.G;
        p.pcol = d.pcol;
        p.t_hot = a.t_hot;
        p.t_lane = a.t_lane;
        p.gather_policy = a.gather_policy;
        p.out = d.out;
        p.err = a.err;
        unsigned long long acc = 0;
        const bool vec = d.vec != 0;
        switch (d.agg) {
            case SKX_AGG_COUNT:
                batch_rows<SKX_AGG_COUNT, PATH>(p, acc, g, h, pol_s, pol_g, vec);
                __syncthreads();
                batch_epilogue<SKX_AGG_COUNT, PATH>(p, acc, g, h, pol_g, s_red);
                break;
            case SKX_AGG_SUM:
                batch_rows<SKX_AGG_SUM, PATH>(p, acc, g, h, pol_s, pol_g, vec);
                __syncthreads();
                batch_epilogue<SKX_AGG_SUM, PATH>(p, acc, g, h, pol_g, s_red);
                break;
            default:
                batch_rows<SKX_AGG_GROUPBY_SUM, PATH>(p, acc, g, h, pol_s, pol_g, vec);
                __syncthreads();
                batch_epilogue<SKX_AGG_GROUPBY_SUM, PATH>(p, acc, g, h, pol_g, s_red);
                break;
        }
        __syncthreads();
    }
}

constexpr int kBatchMaxGroups = 4096;

}  // namespace

int batch_row_path(const void *rows, int32_t row_bytes, bool cols_beyond16, bool cols_beyond8) {
    if (row_bytes % 16 == 0 && aligned16(rows) && !cols_beyond16) return kRow16;
    if (row_bytes == 8 && (reinterpret_cast<uintptr_t>(rows) & 7u) == 0 && !cols_beyond8) return kRow8;
    return kRowGeneric;
}

cudaError_t launch_batch_items(const BatchDesc *d_desc, const uint32_t *d_tile_start, int32_t n,
                               uint32_t total_tiles, int32_t tile_rows, const void *rows, int32_t N,
                               int32_t row_bytes, int path, int32_t max_groups, const skx_tuning &t,
                               bool clear_outputs, uint32_t *d_counter, cudaStream_t st) {
    unsigned *err = device_error_word();
    if (!err) return cudaErrorMemoryAllocation;
    const int32_t t_hot = t.hot_keys > 0 ? t.hot_keys : 0;
    const int32_t t_lane = t.lane_keys > 0 ? t.lane_keys : 0;
    BatchArgs a{};
    a.desc = d_desc;
    a.tile_start = d_tile_start;
    a.counter = d_counter;
    a.n = n;
    a.total_tiles = total_tiles;
    a.tile_rows = tile_rows;
    a.rows = static_cast<const char *>(rows);
    a.N = N;
    a.row_bytes = row_bytes;
    a.max_groups = max_groups;
    a.t_hot = t_hot;
    a.t_lane = t_lane;
    a.gather_policy = t.gather_policy;
    a.err = err;
    const size_t smem = size_t(max_groups + t_hot + t_lane * 32) * 8;
    const int optin = device_max_smem_optin();
    if (smem + 1024 > (size_t)optin) return cudaErrorInvalidValue;
    const int block = t.block_threads;
    int per_sm = 0;
    auto go = [&](auto kern) -> cudaError_t {
        // dynamic + static shared memory must fit the per-block limit
        cudaError_t e2 = set_smem_limit_once(reinterpret_cast<const void *>(kern), -1);
        if (e2 != cudaSuccess) return e2;
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
        if (e2 != cudaSuccess) return e2;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        if (t.ctas_per_sm > 0 && t.ctas_per_sm < per_sm) per_sm = t.ctas_per_sm;
        int64_t grid = int64_t(device_sm_count()) * per_sm;
        if (grid > int64_t(total_tiles)) grid = std::max<int64_t>(1, total_tiles);
        k_batch_clear<<<std::max(1, std::min(n, 1024)), 256, 0, st>>>(d_desc, n, d_counter, clear_outputs ? 1 : 0);
        kern<<<(unsigned)grid, block, smem, st>>>(a);
        note_launches(2);
        return cudaGetLastError();
    };
    if (path == kRow16) return go(k_probe_batch<kRow16>);
    if (path == kRow8) return go(k_probe_batch<kRow8>);
    return go(k_probe_batch<kRowGeneric>);
}

}  // namespace skx

using namespace skx;

struct skx_batch_plan {
    int device;
    const void *rows;
    int32_t N, row_bytes, n, path, max_groups;
    int32_t tile_rows;
    uint32_t total_tiles;
    skx_tuning t;
    std::vector<skx_probe_desc> descs;
    BatchDesc *d_desc;
    uint32_t *d_tile_start;
    uint32_t *d_counter;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool graph_ready;
};

namespace {

skx_status plan_tiles(skx_batch_plan *p, int32_t tile_rows, cudaStream_t st) {
    if (tile_rows <= 0) tile_rows = 65536;
    tile_rows = (tile_rows + 3) & ~3;
    std::vector<uint32_t> start(p->n + 1, 0);
    uint64_t total = 0;
    for (int q = 0; q < p->n; ++q) {
        start[q] = (uint32_t)total;
        total += (uint64_t)((p->descs[q].F + tile_rows - 1) / tile_rows);
        if (total >= (uint64_t(1) << 31)) return SKX_EINVAL;
    }
    start[p->n] = (uint32_t)total;
    p->tile_rows = tile_rows;
    p->total_tiles = (uint32_t)total;
    SKX_CUDA_TRY(cudaMemcpyAsync(p->d_tile_start, start.data(), sizeof(uint32_t) * (p->n + 1), cudaMemcpyHostToDevice, st));
    SKX_CUDA_TRY(cudaStreamSynchronize(st));  // `start` is a host temporary
    return SKX_OK;
}

skx_status plan_launch(skx_batch_plan *p, cudaStream_t st) {
    SKX_CUDA_TRY(launch_batch_items(p->d_desc, p->d_tile_start, p->n, p->total_tiles, p->tile_rows, p->rows, p->N,
                                    p->row_bytes, p->path, p->max_groups, p->t, true, p->d_counter, st));
    return SKX_OK;
}

void release_graph(skx_batch_plan *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
    p->graph_ready = false;
}

}  // namespace

extern "C" {

skx_status skx_batch_plan_create(const void *d_rows, int32_t N, int32_t row_bytes, const skx_probe_desc *h_descs,
                                 int32_t n, const skx_tuning *tuning, int32_t tile_rows, void *stream,
                                 skx_batch_plan **out) {
    if (!out) return SKX_EINVAL;
    *out = nullptr;
    if (!d_rows || N < 1 || row_bytes <= 0 || row_bytes % 4 || !h_descs || n < 1 || n > (1 << 24)) return SKX_EINVAL;
    int32_t max_groups = 1;
    bool any_col_beyond16 = false, any_col_beyond8 = false;
    std::vector<BatchDesc> dd(n);
    for (int q = 0; q < n; ++q) {
        const skx_probe_desc &d = h_descs[q];
        skx_status s = validate_query(&d.q, row_bytes);
        if (s != SKX_OK) return s;
        if (d.F < 0 || d.F >= (int64_t(1) << 32) || !d.out || (d.F > 0 && !d.fk) ||
            (d.F > 0 && d.q.agg != SKX_AGG_COUNT && !d.measure))
            return SKX_EINVAL;
        if ((reinterpret_cast<uintptr_t>(d.fk) & 3u) || (reinterpret_cast<uintptr_t>(d.measure) & 3u) ||
            (reinterpret_cast<uintptr_t>(d.out) & 7u))
            return SKX_EINVAL;
        const bool grp = d.q.agg == SKX_AGG_GROUPBY_SUM;
        if (grp && d.q.num_groups > kBatchMaxGroups) return SKX_ENOTSUP;
        const int32_t nout = grp ? d.q.num_groups : 1;
        max_groups = std::max(max_groups, nout);
        const int32_t cols[3] = {d.q.filter_col, grp ? d.q.group_col : -1, d.q.payload_col};
        for (int32_t c : cols) {
            any_col_beyond16 |= c >= 4;
            any_col_beyond8 |= c >= 2;
        }
        BatchDesc b{};
        b.fk = d.fk;
        b.measure = d.q.agg == SKX_AGG_COUNT ? nullptr : d.measure;
        b.out = reinterpret_cast<unsigned long long *>(d.out);
        b.F = d.F;
        b.agg = d.q.agg;
        b.fcol = d.q.filter_col;
        b.flt = d.q.filter_lt;
        b.gcol = d.q.group_col;
        b.G = nout;
        b.pcol = d.q.payload_col;
        b.nout = nout;
        b.vec = aligned16(d.fk) && (d.q.agg == SKX_AGG_COUNT || aligned16(d.measure));
        dd[q] = b;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    skx_batch_plan *p = new skx_batch_plan{};
    cudaGetDevice(&p->device);
    p->rows = d_rows;
    p->N = N;
    p->row_bytes = row_bytes;
    p->n = n;
    p->max_groups = max_groups;
    p->descs.assign(h_descs, h_descs + n);
    p->path = batch_row_path(d_rows, row_bytes, any_col_beyond16, any_col_beyond8);
    skx_tuning t{};
    if (tuning) t = *tuning;
    ProbeArgs pa{};
    pa.N = N;
    pa.row_bytes = row_bytes;
    pa.q = h_descs[0].q;
    pa.q.agg = SKX_AGG_GROUPBY_SUM;
    pa.q.num_groups = max_groups;
    if (t.hot_keys == 0) t.hot_keys = std::min(N, 1024);  // per-tile hot epilogues favour a short prefix
    resolve_probe_tuning(pa, t);
    p->t = t;
    cudaError_t e = cudaMalloc(&p->d_desc, sizeof(BatchDesc) * n);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tile_start, sizeof(uint32_t) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_counter, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_desc, dd.data(), sizeof(BatchDesc) * n, cudaMemcpyHostToDevice, st);
    skx_status s = e == cudaSuccess ? plan_tiles(p, tile_rows, st) : cuda_status(e);
    if (s != SKX_OK) {
        skx_batch_plan_destroy(p);
        return s;
    }
    *out = p;
    return SKX_OK;
}

skx_status skx_batch_plan_launch(skx_batch_plan *plan, int use_graph, void *stream) {
    if (!plan) return SKX_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!use_graph) return plan_launch(plan, st);
    if (!plan->graph_ready) {
        cudaStream_t cap;
        SKX_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        // device set-up (error word, attributes) happens outside the capture
        if (!device_error_word()) {
            cudaStreamDestroy(cap);
            return SKX_ENOMEM;
        }
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        skx_status s = e == cudaSuccess ? plan_launch(plan, cap) : cuda_status(e);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (s != SKX_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return cuda_status(e);
        plan->graph = g;
        e = cudaGraphInstantiate(&plan->exec, g, 0);
        if (e != cudaSuccess) {
            release_graph(plan);
            return cuda_status(e);
        }
        plan->graph_ready = true;
    }
    SKX_CUDA_TRY(cudaGraphLaunch(plan->exec, st));
    note_launches(2);
    return SKX_OK;
}

skx_status skx_batch_plan_autotune(skx_batch_plan *plan, void *stream, skx_tuning *out, int32_t *tile_rows_out,
                                   float *best_ms) {
    if (!plan) return SKX_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    SKX_CUDA_TRY(cudaEventCreate(&e0));
    SKX_CUDA_TRY(cudaEventCreate(&e1));
    const skx_tuning keep = plan->t;
    const int32_t keep_tile = plan->tile_rows;
    float best = 1e30f;
    skx_tuning best_t = keep;
    int32_t best_tile = keep_tile;
    ProbeArgs pa{};
    pa.N = plan->N;
    pa.row_bytes = plan->row_bytes;
    pa.q.agg = SKX_AGG_GROUPBY_SUM;
    pa.q.num_groups = plan->max_groups;
    pa.q.group_col = 0;
    for (int32_t tile : {32768, 65536, 131072}) {
        if (plan_tiles(plan, tile, st) != SKX_OK) continue;
        for (int b : {256, 512})
            for (int cps : {0, -1})
                for (int hot : {-1, 256, 1024, 4096}) {
                    if (hot > plan->N) continue;
                    skx_tuning t{};
                    t.block_threads = b;
                    t.ctas_per_sm = cps;
                    t.hot_keys = hot;
                    t.lane_keys = hot == -1 ? -1 : 0;
                    resolve_probe_tuning(pa, t);
                    plan->t = t;
                    float ms_min = 1e30f;
                    bool ok = true;
                    for (int rep = 0; rep < 2 && ok; ++rep) {
                        cudaEventRecord(e0, st);
                        ok = plan_launch(plan, st) == SKX_OK;
                        cudaEventRecord(e1, st);
                        ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
                        float ms = 0;
                        cudaEventElapsedTime(&ms, e0, e1);
                        ms_min = std::min(ms_min, ms);
                    }
                    cudaGetLastError();
                    if (ok && ms_min < best) {
                        best = ms_min;
                        best_t = t;
                        best_tile = tile;
                    }
                }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    plan->t = best_t;
    skx_status s = plan_tiles(plan, best_tile, st);
    release_graph(plan);  // a captured graph holds the old launch shape
    if (s != SKX_OK) return s;
    if (out) *out = best_t;
    if (tile_rows_out) *tile_rows_out = best_tile;
    if (best_ms) *best_ms = best;
    return best < 1e30f ? SKX_OK : SKX_ECUDA;
}

void skx_batch_plan_destroy(skx_batch_plan *plan) {
    if (!plan) return;
    release_graph(plan);
    if (plan->d_desc) cudaFree(plan->d_desc);
    if (plan->d_tile_start) cudaFree(plan->d_tile_start);
    if (plan->d_counter) cudaFree(plan->d_counter);
    delete plan;
}

skx_status skx_probe_batch(const void *d_rows, int32_t N, int32_t row_bytes, const skx_probe_desc *h_descs,
                           int32_t n, const skx_tuning *tuning, void *stream) {
    skx_batch_plan *p = nullptr;
    skx_status s = skx_batch_plan_create(d_rows, N, row_bytes, h_descs, n, tuning, 0, stream, &p);
    if (s != SKX_OK) return s;
    s = plan_launch(p, static_cast<cudaStream_t>(stream));
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    skx_batch_plan_destroy(p);
    if (s != SKX_OK) return s;
    SKX_CUDA_TRY(e);
    return SKX_OK;
}

}  // extern "C"
