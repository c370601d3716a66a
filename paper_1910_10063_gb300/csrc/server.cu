// server.cu -- a request loop with continuous batching over a resident
// permutation index.
//
// The reordered dimension table and the rank array (the index's old -> new
// map, Section III) stay resident on the device.  Each request brings a fact
// batch with original keys in host memory.  A server thread:
//   1. admits pending requests in arrival order while an in-flight slot and
//      room in a fixed device arena (the memory budget) are free: the keys and
//      measures are copied to the device on a copy stream that carries copies
//      only; once copied, the keys are recoded through the resident rank array
//      (the recode C' = Rank(C) of Section III-A) on a recode stream;
//   2. forms a round from the remaining rows of every admitted, ready request
//      (oldest first, up to `round_rows` rows) and runs it as one persistent
//      batched probe (batch.cu) on a compute stream, two rounds in flight;
//   3. returns each finished result to the caller's host buffer.
// Requests that arrive while others are on the GPU join the next round, and
// their copies overlap with the running rounds: continuous batching.  Every
// host-side wait polls CUDA events against a deadline; no kernel waits on
// anything.
#include <pthread.h>
#include <sched.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "skx_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double seconds(Clock::time_point t) { return std::chrono::duration<double>(t.time_since_epoch()).count(); }

constexpr int32_t kMaxOut = 4096;  // groups per request (shared-memory groups of the batch kernel)

enum State { kPending = 0, kCopying, kReady, kFinishing, kDone, kFailed };

struct Req {
    uint64_t ticket = 0;
    skx_request r{};
    int32_t nout = 1;
    bool cols16 = false, cols8 = false;  // a needed column beyond the first 16 / 8 bytes
    size_t off = 0, bytes = 0;
    int32_t *d_fk = nullptr, *d_m = nullptr;
    int64_t *d_out = nullptr;
    int slot = -1;
    int64_t next_row = 0;
    int state = kPending;
    uint64_t round_seq = 0;  // the round whose completion delivers the result (kFinishing)
    skx_status status = SKX_OK;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

// First-fit allocator over [0, size) of the device arena.
class Arena {
   public:
    void init(size_t size) {
        free_.clear();
        free_[0] = size;
    }
    bool alloc(size_t bytes, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

   private:
    std::map<size_t, size_t> free_;
};

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// The CPUs next to a device (its PCI function's local_cpulist in sysfs), so
// that the server thread, which polls the device and copies results, does
// not run across a socket from it.  Returns false when they cannot be read.
bool device_local_cpus(int device, cpu_set_t *set) {
    char bus[64] = {0};
    if (cudaDeviceGetPCIBusId(bus, sizeof(bus), device) != cudaSuccess) return false;
    for (char *c = bus; *c; ++c)
        if (*c >= 'A' && *c <= 'F') *c = char(*c - 'A' + 'a');
    char path[160];
    snprintf(path, sizeof(path), "/sys/bus/pci/devices/%s/local_cpulist", bus);
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[4096] = {0};
    const bool got = fgets(line, sizeof(line), f) != nullptr;
    fclose(f);
    if (!got) return false;
    CPU_ZERO(set);
    int n = 0;
    for (char *p = line; *p && *p != '\n';) {
        char *end = nullptr;
        const long lo = strtol(p, &end, 10);
        if (end == p) break;
        long hi = lo;
        p = end;
        if (*p == '-') {
            hi = strtol(p + 1, &end, 10);
            p = end;
        }
        for (long c = lo; c <= hi && c < CPU_SETSIZE; ++c) {
            CPU_SET((int)c, set);
            ++n;
        }
        if (*p == ',') ++p;
    }
    return n > 0;
}

}  // namespace

using namespace skx;

struct skx_server {
    int device = 0;
    const void *rows = nullptr;
    int32_t N = 0, row_bytes = 0;
    const int32_t *rank = nullptr;
    skx_server_config cfg{};
    char *arena_base = nullptr;
    Arena arena;
    cudaStream_t s_copy = nullptr, s_recode = nullptr, s_comp = nullptr;
    BatchDesc *d_desc[2] = {}, *h_desc[2] = {};
    uint32_t *d_tile[2] = {}, *h_tile[2] = {}, *d_counter[2] = {};
    cudaEvent_t ev_round[2] = {};
    bool round_used[2] = {false, false};
    double round_t0[2] = {0.0, 0.0};  // host time the round was enqueued (for the deadline)
    uint64_t round_seq_of[2] = {0, 0};  // sequence number of the round in each buffer
    uint64_t rounds_enqueued = 0, rounds_done = 0;  // rounds are completed in sequence order
    uint64_t loops = 0;
    int64_t *h_stage = nullptr;  // pinned, kMaxOut per slot
    std::vector<cudaEvent_t> ev_copied, ev_ready;
    std::vector<int> free_slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::vector<Req *> active;
    std::map<uint64_t, Req *> reqs;
    std::thread th;
    bool stop = false;
    bool broken = false;
    uint64_t next_ticket = 1;
    uint64_t rounds = 0, round_rows_total = 0, max_active = 0;
    int round_idx = 0;
};

namespace {

void fail_all(skx_server *s, skx_status st) {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Req *q : s->active) {
        q->state = kFailed;
        q->status = st;
    }
    for (Req *q : s->pending) {
        q->state = kFailed;
        q->status = st;
    }
    s->active.clear();
    s->pending.clear();
    s->broken = true;
    s->cv_done.notify_all();
}

// Host bookkeeping of an admission (called with s->mu held): room in the
// device arena and an in-flight slot.  False when the arena is short.
bool reserve(skx_server *s, Req *q) {
    // device memory: keys, measures, output
    const size_t fk_b = up256(size_t(q->r.F) * 4), m_b = q->r.h_measure ? fk_b : 0, out_b = up256(size_t(q->nout) * 8);
    const size_t need = fk_b + m_b + out_b;
    size_t off = 0;
    if (!s->arena.alloc(need, &off)) return false;
    q->off = off;
    q->bytes = need;
    char *base = s->arena_base + off;
    q->d_fk = reinterpret_cast<int32_t *>(base);
    q->d_m = m_b ? reinterpret_cast<int32_t *>(base + fk_b) : nullptr;
    q->d_out = reinterpret_cast<int64_t *>(base + fk_b + m_b);
    q->slot = s->free_slots.back();
    s->free_slots.pop_back();
    q->next_row = 0;
    q->t_admit = seconds(Clock::now());
    q->state = kCopying;
    return true;
}

// The CUDA work of an admission, enqueued without holding s->mu (the lock is
// what submitters wait for).  Only copies go on the copy stream: a kernel
// there would wait for SMs held by a running round, and every later copy
// would wait behind it.  The recode C' = Rank(C) and the cleared output
// follow on a recode stream once the copy is done.
void enqueue_admission(skx_server *s, Req *q) {
    unsigned *err = device_error_word();
    cudaError_t e = err ? cudaSuccess : cudaErrorInvalidSymbol;
    if (e == cudaSuccess && q->r.F > 0) {
        e = cudaMemcpyAsync(q->d_fk, q->r.h_fk, size_t(q->r.F) * 4, cudaMemcpyHostToDevice, s->s_copy);
        if (e == cudaSuccess && q->d_m)
            e = cudaMemcpyAsync(q->d_m, q->r.h_measure, size_t(q->r.F) * 4, cudaMemcpyHostToDevice, s->s_copy);
    }
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_copied[q->slot], s->s_copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->s_recode, s->ev_copied[q->slot], 0);
    if (e == cudaSuccess && q->r.F > 0 && s->rank)
        e = launch_remap(s->rank, s->N, q->d_fk, q->d_fk, q->r.F, err, s->s_recode);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->d_out, 0, size_t(q->nout) * 8, s->s_recode);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_ready[q->slot], s->s_recode);
    if (e != cudaSuccess) {
        cuda_status(e);
        std::lock_guard<std::mutex> lk(s->mu);
        q->status = SKX_ECUDA;
        q->state = kFailed;
    }
}

void finish(skx_server *s, Req *q, int state, skx_status st) {
    q->state = state;
    q->status = st;
    q->t_done = seconds(Clock::now());
    if (q->bytes) s->arena.release(q->off, q->bytes);
    q->bytes = 0;
    if (q->slot >= 0) s->free_slots.push_back(q->slot);
    q->slot = -1;
}

void server_loop(skx_server *s) {
    cudaSetDevice(s->device);
    if (s->cfg.cpu_affinity == 0) {
        cpu_set_t set;
        if (device_local_cpus(s->device, &set)) pthread_setaffinity_np(pthread_self(), sizeof(set), &set);
    }
    const double wait_limit = s->cfg.timeout_ms / 1e3;
    while (true) {
        std::vector<Req *> to_admit;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->active.empty() && s->pending.empty())
                s->cv_work.wait_for(lk, std::chrono::milliseconds(2), [&] { return s->stop || !s->pending.empty(); });
            if (s->stop && s->active.empty() && s->pending.empty()) break;
            if (s->stop && s->broken) break;
        }
        bool progressed = false;
        // 1. admission (arrival order; a request waits while memory or slots are short).  The
        //    lock covers only host bookkeeping; the copies are enqueued after it is released.
        std::vector<Req *> admitted;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            while (!s->pending.empty() && !s->free_slots.empty() &&
                   (int32_t)s->active.size() < s->cfg.max_inflight) {
                Req *q = s->pending.front();
                if (!reserve(s, q)) break;
                s->pending.pop_front();
                s->active.push_back(q);
                admitted.push_back(q);
            }
            s->max_active = std::max<uint64_t>(s->max_active, s->active.size());
        }
        for (Req *q : admitted) enqueue_admission(s, q);
        progressed |= !admitted.empty();
        // 2. a round over every ready request's remaining rows
        std::vector<Req *> last_chunk;
        std::vector<BatchDesc> items;
        int32_t max_groups = 1;
        bool any16 = false, any8 = false;
        int64_t budget = s->cfg.round_rows;
        // the round buffer to fill next must be free; while its previous round runs the loop
        // keeps admitting and completing requests instead of waiting (with a deadline)
        const int rb = s->round_idx & 1;
        bool round_free = true;
        bool failed = false;
        // Rounds run in order on the compute stream, so the oldest round in flight is the
        // only one worth asking about; when it is done, so are the results it carried.
        for (int k = 0; k < 2 && !failed; ++k) {
            const int b = (s->round_idx + k) & 1;  // oldest first
            if (!s->round_used[b] || s->round_seq_of[b] <= s->rounds_done) continue;
            const cudaError_t qe = cudaEventQuery(s->ev_round[b]);
            if (qe == cudaSuccess) {
                s->rounds_done = s->round_seq_of[b];
                continue;
            }
            if (qe != cudaErrorNotReady) {
                cuda_status(qe);
                fail_all(s, SKX_ECUDA);
                failed = true;
            } else if (seconds(Clock::now()) - s->round_t0[b] > wait_limit) {
                fail_all(s, SKX_ETIMEOUT);
                failed = true;
            }
            break;  // a later round cannot be done before this one
        }
        if (failed) break;
        if (s->round_used[rb] && s->round_seq_of[rb] > s->rounds_done) round_free = false;
        // Copies and recodes run in admission order on their streams, so readiness is asked
        // of the oldest copying request only, and of the next ones while they are ready.
        bool copies_pending = true;
        for (Req *q : s->active) {
            if (q->state == kCopying && copies_pending) {
                if (cudaEventQuery(s->ev_ready[q->slot]) == cudaSuccess) q->state = kReady;
                else copies_pending = false;
            }
            if (q->state != kReady || budget <= 0 || !round_free) continue;
            const int64_t take = std::min<int64_t>(q->r.F - q->next_row, budget);
            if (take > 0) {
                BatchDesc b{};
                b.fk = q->d_fk + q->next_row;
                b.measure = q->d_m ? q->d_m + q->next_row : nullptr;
                b.out = reinterpret_cast<unsigned long long *>(q->d_out);
                b.F = take;
                b.agg = q->r.q.agg;
                b.fcol = q->r.q.filter_col;
                b.flt = q->r.q.filter_lt;
                b.gcol = q->r.q.group_col;
                b.G = q->nout;
                b.pcol = q->r.q.payload_col;
                b.nout = q->nout;
                b.vec = aligned16(b.fk) && (b.measure == nullptr || aligned16(b.measure));
                items.push_back(b);
                max_groups = std::max(max_groups, q->nout);
                any16 |= q->cols16;
                any8 |= q->cols8;
                q->next_row += take;
                budget -= take;
            }
            if (q->next_row >= q->r.F) last_chunk.push_back(q);
        }
        if (round_free && (!last_chunk.empty() || !items.empty())) {
            const int b = rb;
            cudaError_t e = cudaSuccess;
            if (!items.empty()) {
                const int32_t tile = s->cfg.tile_rows;
                uint64_t tiles = 0;
                for (size_t i = 0; i < items.size(); ++i) {
                    s->h_desc[b][i] = items[i];
                    s->h_tile[b][i] = (uint32_t)tiles;
                    tiles += (uint64_t)((items[i].F + tile - 1) / tile);
                }
                s->h_tile[b][items.size()] = (uint32_t)tiles;
                e = cudaMemcpyAsync(s->d_desc[b], s->h_desc[b], sizeof(BatchDesc) * items.size(),
                                    cudaMemcpyHostToDevice, s->s_comp);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(s->d_tile[b], s->h_tile[b], sizeof(uint32_t) * (items.size() + 1),
                                        cudaMemcpyHostToDevice, s->s_comp);
                if (e == cudaSuccess)
                    e = launch_batch_items(s->d_desc[b], s->d_tile[b], (int32_t)items.size(), (uint32_t)tiles, tile,
                                           s->rows, s->N, s->row_bytes,
                                           batch_row_path(s->rows, s->row_bytes, any16, any8), max_groups,
                                           s->cfg.tuning, false,
                                           s->d_counter[b], s->s_comp);
                s->rounds++;
                for (const BatchDesc &d : items) s->round_rows_total += (uint64_t)d.F;
            }
            const uint64_t seq = ++s->rounds_enqueued;
            for (Req *q : last_chunk) {
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(s->h_stage + size_t(q->slot) * kMaxOut, q->d_out, size_t(q->nout) * 8,
                                        cudaMemcpyDeviceToHost, s->s_comp);
                q->round_seq = seq;
                q->state = kFinishing;
            }
            if (e == cudaSuccess) e = cudaEventRecord(s->ev_round[b], s->s_comp);
            s->round_seq_of[b] = seq;
            if (e != cudaSuccess) {
                cuda_status(e);
                fail_all(s, SKX_ECUDA);
                break;
            }
            s->round_used[b] = true;
            s->round_t0[b] = seconds(Clock::now());
            s->round_idx++;
            progressed = true;
        }
        // 3. completions: the device is polled without the lock; the lock is taken once, only
        //    when results are ready to hand over
        {
            std::vector<std::pair<Req *, skx_status>> ended;
            for (Req *q : s->active) {
                if (q->state == kFinishing && q->round_seq <= s->rounds_done) ended.push_back({q, SKX_OK});
                else if (q->state == kFailed) ended.push_back({q, q->status});
            }
            if (!ended.empty()) {
                std::lock_guard<std::mutex> lk(s->mu);
                for (auto &x : ended) {
                    Req *q = x.first;
                    if (x.second == SKX_OK) {
                        std::memcpy(q->r.h_out, s->h_stage + size_t(q->slot) * kMaxOut, size_t(q->nout) * 8);
                        finish(s, q, kDone, SKX_OK);
                    } else {
                        finish(s, q, kFailed, x.second);
                    }
                    s->active.erase(std::find(s->active.begin(), s->active.end(), q));
                }
                s->cv_done.notify_all();
                progressed = true;
            }
        }
        ++s->loops;
        // Nothing moved: the device is busy.  Yield rather than sleep -- a sleep of a few
        // microseconds lasts the kernel's timer slack (tens of microseconds), which every
        // request waiting for its round or its copy would pay again.
        if (!progressed) std::this_thread::yield();
    }
}

}  // namespace

extern "C" {

skx_status skx_server_create(const void *d_rows, int32_t N, int32_t row_bytes, const int32_t *d_rank,
                             const skx_server_config *cfg, skx_server **out) {
    if (!out) return SKX_EINVAL;
    *out = nullptr;
    if (!d_rows || N < 1 || row_bytes <= 0 || row_bytes % 4) return SKX_EINVAL;
    skx_server *s = new skx_server{};
    cudaGetDevice(&s->device);
    s->rows = d_rows;
    s->N = N;
    s->row_bytes = row_bytes;
    s->rank = d_rank;
    if (cfg) s->cfg = *cfg;
    if (s->cfg.max_inflight <= 0) s->cfg.max_inflight = 128;
    if (s->cfg.tile_rows <= 0) s->cfg.tile_rows = 65536;
    s->cfg.tile_rows = (s->cfg.tile_rows + 3) & ~3;
    if (s->cfg.round_rows <= 0) s->cfg.round_rows = int64_t(64) << 20;
    if (s->cfg.timeout_ms <= 0) s->cfg.timeout_ms = 10000;
    if (s->cfg.memory_budget <= 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        s->cfg.memory_budget = (int64_t)std::min<size_t>(fr / 2, size_t(16) << 30);
    }
    ProbeArgs pa{};
    pa.N = N;
    pa.row_bytes = row_bytes;
    pa.q.agg = SKX_AGG_GROUPBY_SUM;
    pa.q.num_groups = kMaxOut;
    if (s->cfg.tuning.hot_keys == 0) s->cfg.tuning.hot_keys = std::min(N, 1024);
    resolve_probe_tuning(pa, s->cfg.tuning);
    const int32_t slots = s->cfg.max_inflight;
    cudaError_t e = cudaMalloc(&s->arena_base, (size_t)s->cfg.memory_budget);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_recode, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaMalloc(&s->d_desc[b], sizeof(BatchDesc) * slots);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_tile[b], sizeof(uint32_t) * (slots + 1));
        if (e == cudaSuccess) e = cudaMalloc(&s->d_counter[b], sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_desc[b], sizeof(BatchDesc) * slots);
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_tile[b], sizeof(uint32_t) * (slots + 1));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_round[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_stage, sizeof(int64_t) * kMaxOut * slots);
    s->ev_copied.assign(slots, nullptr);
    s->ev_ready.assign(slots, nullptr);
    for (int i = 0; i < slots && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&s->ev_ready[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_copied[i], cudaEventDisableTiming);
        s->free_slots.push_back(slots - 1 - i);
    }
    if (e == cudaSuccess && !device_error_word()) e = cudaErrorMemoryAllocation;
    if (e != cudaSuccess) {
        skx_status st = cuda_status(e);
        skx_server_destroy(s);
        return st;
    }
    s->arena.init((size_t)s->cfg.memory_budget);
    s->th = std::thread(server_loop, s);
    *out = s;
    return SKX_OK;
}

skx_status skx_server_submit(skx_server *s, const skx_request *req, uint64_t *ticket) {
    if (!s || !req || !ticket) return SKX_EINVAL;
    skx_status st = validate_query(&req->q, s->row_bytes);
    if (st != SKX_OK) return st;
    const bool grp = req->q.agg == SKX_AGG_GROUPBY_SUM;
    if (grp && req->q.num_groups > kMaxOut) return SKX_ENOTSUP;
    if (req->F < 0 || req->F >= (int64_t(1) << 32) || !req->h_out || (req->F > 0 && !req->h_fk) ||
        (req->F > 0 && req->q.agg != SKX_AGG_COUNT && !req->h_measure))
        return SKX_EINVAL;
    const size_t need = up256(size_t(req->F) * 4) * 2 + up256(size_t(kMaxOut) * 8);
    if (need > (size_t)s->cfg.memory_budget) return SKX_ENOMEM;  // can never be admitted
    Req *q = new Req{};
    q->r = *req;
    if (q->r.q.agg == SKX_AGG_COUNT) q->r.h_measure = nullptr;
    q->nout = grp ? req->q.num_groups : 1;
    const int32_t cols[3] = {req->q.filter_col, grp ? req->q.group_col : -1,
                             req->q.agg == SKX_AGG_COUNT ? -1 : req->q.payload_col};
    for (int32_t c : cols) {
        q->cols16 |= c >= 4;
        q->cols8 |= c >= 2;
    }
    q->t_submit = seconds(Clock::now());
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->broken) {
        delete q;
        return SKX_ECUDA;
    }
    q->ticket = s->next_ticket++;
    s->reqs[q->ticket] = q;
    s->pending.push_back(q);
    *ticket = q->ticket;
    s->cv_work.notify_one();
    return SKX_OK;
}

skx_status skx_server_wait(skx_server *s, uint64_t ticket, int32_t timeout_ms) {
    if (!s) return SKX_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return SKX_EINVAL;
    Req *q = it->second;
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                        [&] { return q->state == kDone || q->state == kFailed; });
    if (!ok) return SKX_ETIMEOUT;
    return q->status;
}

skx_status skx_server_request_times(skx_server *s, uint64_t ticket, double *submit_s, double *admit_s,
                                    double *done_s) {
    if (!s) return SKX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return SKX_EINVAL;
    Req *q = it->second;
    if (submit_s) *submit_s = q->t_submit;
    if (admit_s) *admit_s = q->t_admit;
    if (done_s) *done_s = q->t_done;
    return q->state == kDone ? SKX_OK : (q->state == kFailed ? q->status : SKX_EBUSY);
}

skx_status skx_server_release(skx_server *s, uint64_t ticket) {
    if (!s) return SKX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return SKX_EINVAL;
    if (it->second->state != kDone && it->second->state != kFailed) return SKX_EBUSY;
    delete it->second;
    s->reqs.erase(it);
    return SKX_OK;
}

skx_status skx_server_replay(skx_server *s, const skx_request *reqs, const double *arrival_s, int32_t n,
                             int32_t timeout_ms, double *latency_s) {
    if (!s || !reqs || !arrival_s || n < 0 || !latency_s) return SKX_EINVAL;
    std::vector<uint64_t> tickets(n);
    const double t0 = seconds(Clock::now());
    for (int32_t i = 0; i < n; ++i) {
        while (seconds(Clock::now()) - t0 < arrival_s[i]) {  // open-loop schedule
        }
        skx_status st = skx_server_submit(s, &reqs[i], &tickets[i]);
        if (st != SKX_OK) return st;
    }
    skx_status worst = SKX_OK;
    for (int32_t i = 0; i < n; ++i) {
        const double left_ms = std::max(0.0, timeout_ms - (seconds(Clock::now()) - t0) * 1e3);
        skx_status st = skx_server_wait(s, tickets[i], (int32_t)left_ms);
        double done = 0;
        skx_server_request_times(s, tickets[i], nullptr, nullptr, &done);
        latency_s[i] = st == SKX_OK ? done - (t0 + arrival_s[i]) : -1.0;
        if (st != SKX_OK && worst == SKX_OK) worst = st;
        skx_server_release(s, tickets[i]);
    }
    return worst;
}

skx_status skx_server_stats(skx_server *s, uint64_t *rounds, uint64_t *rows, uint64_t *max_active) {
    if (!s) return SKX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (rounds) *rounds = s->rounds;
    if (rows) *rows = s->round_rows_total;
    if (max_active) *max_active = s->max_active;
    return SKX_OK;
}

void skx_server_destroy(skx_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    if (s->s_copy) cudaStreamSynchronize(s->s_copy);
    if (s->s_recode) cudaStreamSynchronize(s->s_recode);
    if (s->s_comp) cudaStreamSynchronize(s->s_comp);
    for (auto &kv : s->reqs) delete kv.second;
    for (int b = 0; b < 2; ++b) {
        if (s->d_desc[b]) cudaFree(s->d_desc[b]);
        if (s->d_tile[b]) cudaFree(s->d_tile[b]);
        if (s->d_counter[b]) cudaFree(s->d_counter[b]);
        if (s->h_desc[b]) cudaFreeHost(s->h_desc[b]);
        if (s->h_tile[b]) cudaFreeHost(s->h_tile[b]);
        if (s->ev_round[b]) cudaEventDestroy(s->ev_round[b]);
    }
    for (cudaEvent_t e : s->ev_ready)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : s->ev_copied)
        if (e) cudaEventDestroy(e);
    if (s->h_stage) cudaFreeHost(s->h_stage);
    if (s->arena_base) cudaFree(s->arena_base);
    if (s->s_copy) cudaStreamDestroy(s->s_copy);
    if (s->s_recode) cudaStreamDestroy(s->s_recode);
    if (s->s_comp) cudaStreamDestroy(s->s_comp);
    delete s;
}

}  // extern "C"
