// K6 -- the serving loop: admission by memory budget, continuous batching of
// request parts into steps, concurrent steps on several CUDA streams.
//
// Every request is a processing element with its own slice of its own stream
// (paper Sec. 2.1); positions are reserved at submission, in submission
// order, so a result never depends on which step or which neighbours it ran
// with.  A step is the batch kernel (batch.cu) over the request parts of the
// step: one set-up kernel (each part's start state by jump-ahead, Sec. 2.3)
// and one persistent generation kernel, enqueued on the step's slot stream.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <sys/prctl.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace srng_impl {
namespace {

using Clock = std::chrono::steady_clock;

double now_s()
{
    return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t stream = 0, pos = 0, n = 0;
    srng_out type = SRNG_OUT_U32;
    uint32_t esz = 4;
    uint64_t pool_off = 0;      // bytes
    uint64_t scheduled = 0, done = 0;
    int state = 0;              // 0 queued, 1 admitted, 2 complete
    bool auto_release = false;
    double t_submit = 0, t_done = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    // one host-to-device copy per step: the step's descriptors, then (16-byte
    // aligned) its work items, in one page-locked buffer and its device twin
    BatchInst *h_inst = nullptr, *d_inst = nullptr;
    uint2 *h_items = nullptr;  // work items as the step is gathered
    uint32_t *d_item_state = nullptr;  // MRG32k3a items' first-chunk states (6 words each)
    uint32_t *d_counter = nullptr;
    std::vector<std::pair<uint64_t, uint64_t>> parts;  // (ticket, draws) of the step in flight
};

// First-fit allocator over [0, size) in 256-byte units.
struct Pool {
    std::map<uint64_t, uint64_t> free_;  // offset -> size
    uint64_t used = 0, peak = 0;
    void init(uint64_t size) { free_.clear(); free_[0] = size; used = peak = 0; }
    bool alloc(uint64_t want, uint64_t *off)
    {
        want = (want + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= want) {
                *off = it->first;
                const uint64_t rest = it->second - want, start = it->first + want;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used += want;
                peak = std::max(peak, used);
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t size)
    {
        size = (size + 255) / 256 * 256;
        used -= size;
        auto it = free_.emplace(off, size).first;
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
};

}  // namespace
}  // namespace srng_impl

using namespace srng_impl;

// MRG32k3a lane chunks of a step: its jump table (A^(chunk 2^k)) and lane table
// (A^(chunk l), l < 32, on the device).
struct ChunkCfg {
    uint64_t chunk = 0;
    JumpTable tab;
    uint32_t *d_lane_tab = nullptr;
};
// Default chunks by the draws a step can take: below kStepDraws[0] 128-draw
// chunks, below kStepDraws[1] 256, else 1024 -- more lanes for a small step
// (lower latency), fewer work items for a large one (higher throughput).
// Serving workload, 20k req/s, one chunk for every step: 128 p50 62 us /
// saturation 763 Guniforms/s; 256: 67 us / 790; 512: 83 us / 805; 1024:
// 120 us / 810.
constexpr int kChunks = 3;
// MRG32k3a steps of at most this many work items set up their item states in
// one kernel straight from the stream states
constexpr uint32_t kDirectItemStates = 4096;
constexpr uint64_t kDefaultChunk[kChunks] = {128, 256, 1024};
constexpr uint64_t kStepDraws[kChunks - 1] = {1ull << 23, 1ull << 27};

struct srng_server {
    srng_set *set = nullptr;
    srng_server_config cfg;
    int device = 0;
    unsigned grid[3] = {0, 0, 0};
    char *pool_mem = nullptr;
    Pool pool;
    ChunkCfg ck[kChunks];            // by step size, smallest first ([0] only: a configured chunk)
    int n_ck = 1;
    std::vector<Slot> slots;
    uint32_t cap_items = 0;

    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::unordered_map<uint64_t, Req> reqs;
    std::deque<uint64_t> pending;   // submitted, waiting for pool memory
    std::deque<uint64_t> active;    // admitted with unscheduled draws
    std::unordered_map<uint64_t, uint64_t> next_pos;
    uint64_t next_ticket = 1;
    std::thread th;
    bool stop = false;
    srng_status fault = SRNG_OK;
    std::string fault_msg;

    // statistics
    std::vector<double> lat_us;
    uint64_t submitted = 0, completed = 0, rejected = 0, draws_completed = 0, steps = 0, kernels = 0;
    double t_first = 0, t_last = 0;
    uint64_t peak_base = 0;
};

namespace srng_impl {
namespace {

// Mark the parts of a finished step; completes requests.  Caller holds mu.
void finish_step(srng_server *srv, Slot &sl)
{
    const double t = now_s();
    for (auto &p : sl.parts) {
        auto it = srv->reqs.find(p.first);
        if (it == srv->reqs.end()) continue;
        Req &r = it->second;
        r.done += p.second;
        if (r.done == r.n) {
            r.state = 2;
            r.t_done = t;
            srv->lat_us.push_back((t - r.t_submit) * 1e6);
            srv->completed++;
            srv->draws_completed += r.n;
            srv->t_last = t;
            if (r.auto_release) {
                srv->pool.release(r.pool_off, r.n * r.esz);
                srv->reqs.erase(it);
            }
        }
    }
    sl.parts.clear();
    sl.busy = false;
    srv->cv_done.notify_all();
}

// Build and enqueue one step on a free slot.  Caller holds mu.
srng_status launch_step(srng_server *srv, Slot &sl)
{
    const srng_set *set = srv->set;
    uint64_t budget = srv->cfg.max_step_draws;
    uint32_t n_inst = 0, n_items = 0;
    int type = -1;
    // the step's chunk, by the draws it can take (capped once past the last threshold)
    int ci = 0;
    if (srv->n_ck > 1) {
        uint64_t want = 0;
        uint32_t parts = 0;
        int t0 = -1;
        for (uint64_t id : srv->active) {
            if (want >= kStepDraws[kChunks - 2] || parts >= srv->cfg.max_step_requests) break;
            const Req &r = srv->reqs[id];
            if (t0 < 0) t0 = r.type;
            if ((int)r.type != t0) continue;
            want += r.n - r.scheduled;
            ++parts;
        }
        want = std::min(want, srv->cfg.max_step_draws);
        while (ci < srv->n_ck - 1 && want >= kStepDraws[ci]) ++ci;
    }
    const ChunkCfg &ck = srv->ck[ci];
    const uint64_t chunk = ck.chunk, lane_blocks = srv->cfg.lane_blocks;
    for (auto it = srv->active.begin(); it != srv->active.end() && budget && n_inst < srv->cfg.max_step_requests;) {
        Req &r = srv->reqs[*it];
        if (type < 0) type = r.type;
        if ((int)r.type != type) { ++it; continue; }
        uint64_t take = std::min(r.n - r.scheduled, budget);
        // work items this part needs, bounded by the slot's item buffer
        auto items_for = [&](uint64_t len) -> uint64_t {
            if (set->gen == SRNG_MRG32K3A) return ((len + chunk - 1) / chunk + 31) / 32;
            const uint64_t per = 32 * lane_blocks;
            return ((len + 3) / 4 + 1 + per - 1) / per;
        };
        if (n_items + items_for(take) > srv->cap_items) {
            const uint64_t room = srv->cap_items - n_items;
            if (room == 0) break;
            take = set->gen == SRNG_MRG32K3A ? std::min(take, room * 32 * chunk)
                                              : std::min(take, (room * 32 * lane_blocks - 1) * 4);
            if (take == 0) break;
        }
        BatchInst &b = sl.h_inst[n_inst];
        memset(&b, 0, sizeof b);
        b.gen = inst_gen(set);
        const uint64_t gs = set->stream_base + r.stream;  // stream number
        b.key0 = set->keyed ? (uint32_t)gs : set->key0;
        b.key1 = set->keyed ? (uint32_t)(gs >> 32) : set->key1;
        b.ctr_hi = set->keyed ? ((uint64_t)set->key1 << 32 | set->key0) : gs;
        b.stream = r.stream;
        b.offset = r.pos + r.scheduled;
        b.length = take;
        b.out_offset = r.pool_off / r.esz + r.scheduled;
        b.src_state = set->d_state;
        b.src_ns = set->n_streams;
        b.src_pos = set->d_pos;
        if (set->gen == SRNG_MRG32K3A) {
            const uint64_t nch = (take + chunk - 1) / chunk;
            for (uint64_t c = 0; c < nch; c += 32) sl.h_items[n_items++] = make_uint2(n_inst, (uint32_t)c);
        } else {
            const uint64_t nb = (take + 3) / 4 + 1, per = 32 * lane_blocks;
            for (uint64_t g = 0; g * per < nb; ++g) sl.h_items[n_items++] = make_uint2(n_inst, (uint32_t)g);
        }
        sl.parts.emplace_back(*it, take);
        ++n_inst;
        r.scheduled += take;
        budget -= take;
        if (r.scheduled == r.n) it = srv->active.erase(it);
        else ++it;
    }
    if (n_inst == 0) return SRNG_OK;
    const size_t items_off = (n_inst * sizeof(BatchInst) + 15) / 16 * 16;
    memcpy(reinterpret_cast<char *>(sl.h_inst) + items_off, sl.h_items, n_items * sizeof(uint2));
    SRNG_CUDA_TRY(cudaMemcpyAsync(sl.d_inst, sl.h_inst, items_off + n_items * sizeof(uint2), cudaMemcpyHostToDevice,
                                  sl.stream));
    uint2 *const d_items = reinterpret_cast<uint2 *>(reinterpret_cast<char *>(sl.d_inst) + items_off);
    const bool mrg = set->gen == SRNG_MRG32K3A;
    // each MRG32k3a item's first-chunk state, so a lane reaches its chunk with one
    // jump: for a small step straight from the stream states in one kernel (the
    // set-up kernel's launch saved), else after a set-up kernel per instance
    // (each instance's offset jump done once); both zero the work counter
    const bool direct = mrg && n_items <= kDirectItemStates;
    if (direct) {
        SRNG_CUDA_TRY(launch_batch_item_states_direct(sl.d_inst, d_items, n_items, ck.tab, sl.d_item_state,
                                                      sl.d_counter, sl.stream));
    } else {
        SRNG_CUDA_TRY(launch_batch_setup(sl.d_inst, n_inst, sl.stream, sl.d_counter));
        if (mrg)
            SRNG_CUDA_TRY(launch_batch_item_states(sl.d_inst, d_items, n_items, ck.tab, sl.d_item_state,
                                                   sl.stream));
    }
    BatchArgs a;
    memset(&a, 0, sizeof a);
    a.inst = sl.d_inst;
    a.items = d_items;
    a.counter = sl.d_counter;
    a.n_items = n_items;
    a.chunk = chunk;
    a.lane_blocks = (uint32_t)lane_blocks;
    a.mode = SRNG_BATCH_WRITE;
    a.out = srv->pool_mem;
    a.item_state = mrg ? sl.d_item_state : nullptr;
    a.lane_tab = mrg ? ck.d_lane_tab : nullptr;
    const unsigned grid = std::max(1u, std::min(srv->grid[type], (n_items + 7) / 8));
    SRNG_CUDA_TRY(launch_batch(a, (srng_out)type, batch_family(set), ck.tab, grid, sl.stream));
    SRNG_CUDA_TRY(cudaEventRecord(sl.ev, sl.stream));
    sl.busy = true;
    srv->steps++;
    srv->kernels += mrg && !direct ? 3 : 2;
    return SRNG_OK;
}

void dispatcher(srng_server *srv)
{
    cudaSetDevice(srv->device);
#ifdef PR_SET_TIMERSLACK
    // this thread's sleeps end within 1 us of their time: the 5 us polls of
    // steps in flight are not stretched to the default 50 us timer slack
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
#endif
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        bool progress = false;
        bool any_busy = false;
        for (Slot &sl : srv->slots) {
            if (!sl.busy) continue;
            const cudaError_t e = cudaEventQuery(sl.ev);
            if (e == cudaSuccess) {
                finish_step(srv, sl);
                progress = true;
            } else if (e != cudaErrorNotReady) {
                srv->fault = cuda_fail(e, "server step");
                srv->fault_msg = srng_last_error();
                sl.busy = false;
                srv->cv_done.notify_all();
            } else {
                any_busy = true;
            }
        }
        // admission in arrival order, as memory frees up
        while (!srv->pending.empty()) {
            Req &r = srv->reqs[srv->pending.front()];
            uint64_t off;
            if (!srv->pool.alloc(r.n * r.esz, &off)) break;
            r.pool_off = off;
            r.state = 1;
            srv->active.push_back(srv->pending.front());
            srv->pending.pop_front();
            progress = true;
        }
        // fill every free slot with a step
        for (Slot &sl : srv->slots) {
            if (sl.busy || srv->active.empty() || srv->fault) continue;
            const srng_status st = launch_step(srv, sl);
            if (st) {
                srv->fault = st;
                srv->fault_msg = srng_last_error();
                srv->cv_done.notify_all();
                break;
            }
            if (sl.busy) {
                progress = true;
                any_busy = true;
            }
        }
        if (srv->stop && !any_busy) break;
        if (!progress) {
            if (any_busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(5));
                lk.lock();
            } else {
                srv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
    }
}

srng_status check_type(srng_out t)
{
    if (t != SRNG_OUT_U32 && t != SRNG_OUT_F32 && t != SRNG_OUT_F64) return fail(SRNG_ERR_ARG, "unknown output type");
    return SRNG_OK;
}

srng_status submit_common(srng_server *srv, uint64_t stream, bool explicit_pos, uint64_t pos, uint64_t n,
                          srng_out type, bool auto_release, uint64_t *ticket)
{
    if (!srv || (!ticket && !auto_release)) return fail(SRNG_ERR_ARG, "NULL argument");
    srng_status st = check_type(type);
    if (st) return st;
    if (stream >= srv->set->n_streams) return fail(SRNG_ERR_RANGE, "stream outside the set");
    if (n == 0) return fail(SRNG_ERR_ARG, "n must be positive");
    const uint32_t esz = type == SRNG_OUT_F64 ? 8 : 4;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->fault) return fail(srv->fault, "server stopped after an error: " + srv->fault_msg);
    if (n > srv->cfg.budget_bytes / esz) {
        srv->rejected++;
        return fail(SRNG_ERR_BUDGET, "request larger than the server's memory budget");
    }
    uint64_t &np = srv->next_pos[stream];
    const uint64_t p = explicit_pos ? pos : np;
    if (n > UINT64_MAX - p) return fail(SRNG_ERR_RANGE, "position would pass 2^64 - 1");
    if (srv->set->gen == SRNG_PHILOX4X32_10 && p + n > UINT64_MAX - srv->set->max_pos)
        return fail(SRNG_ERR_RANGE, "Philox position would pass 2^64 - 1");
    if (!explicit_pos) np = p + n;
    const uint64_t t = srv->next_ticket++;
    Req r;
    r.stream = stream;
    r.pos = p;
    r.n = n;
    r.type = type;
    r.esz = esz;
    r.auto_release = auto_release;
    r.t_submit = now_s();
    if (srv->submitted == 0 || srv->t_first == 0) srv->t_first = r.t_submit;
    srv->reqs.emplace(t, r);
    srv->pending.push_back(t);
    srv->submitted++;
    if (ticket) *ticket = t;
    srv->cv_work.notify_one();
    return SRNG_OK;
}

void fill_stats(srng_server *srv, srng_server_stats *out)
{
    memset(out, 0, sizeof *out);
    out->submitted = srv->submitted;
    out->completed = srv->completed;
    out->rejected = srv->rejected;
    out->draws_completed = srv->draws_completed;
    out->steps = srv->steps;
    out->kernels = srv->kernels;
    std::vector<double> l = srv->lat_us;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) { return l[std::min(l.size() - 1, (size_t)(q * (l.size() - 1) + 0.5))]; };
        out->p50_us = pct(0.50);
        out->p99_us = pct(0.99);
        double s = 0;
        for (double x : l) s += x;
        out->mean_us = s / l.size();
        out->max_us = l.back();
    }
    out->wall_s = srv->t_last > srv->t_first ? srv->t_last - srv->t_first : 0;
    out->peak_pool_bytes = srv->pool.peak;
}

void server_free(srng_server *srv)
{
    for (Slot &sl : srv->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_inst) cudaFreeHost(sl.h_inst);
        if (sl.h_items) cudaFreeHost(sl.h_items);
        if (sl.d_inst) cudaFree(sl.d_inst);
        if (sl.d_item_state) cudaFree(sl.d_item_state);
        if (sl.d_counter) cudaFree(sl.d_counter);
    }
    for (ChunkCfg &k : srv->ck)
        if (k.d_lane_tab) cudaFree(k.d_lane_tab);
    if (srv->pool_mem) cudaFree(srv->pool_mem);
    delete srv;
}

}  // namespace
}  // namespace srng_impl

extern "C" {

srng_status srng_server_create(srng_server **out, srng_set *set, const srng_server_config *cfg)
{
    clear_error();
    if (!out || !set) return fail(SRNG_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (set->gen == SRNG_TINYMT32) return fail(SRNG_ERR_UNSUPPORTED, "TinyMT32 sets are not served");
    srng_server_config c;
    memset(&c, 0, sizeof c);
    if (cfg) c = *cfg;
    if (!c.budget_bytes) c.budget_bytes = 16ull << 30;
    if (!c.max_inflight) c.max_inflight = 4;
    if (!c.max_step_requests) c.max_step_requests = 4096;
    // steps of up to 2^30 draws: the serving workload's saturation throughput
    // grows with the step (2^25: 535 Guniforms/s, 2^27: 723, 2^30: 806) and
    // its latency at the offered load does not suffer (p99 356 -> 285 us)
    if (!c.max_step_draws) c.max_step_draws = 1ull << 30;
    if (!c.lane_blocks) c.lane_blocks = 64;
    if (c.max_inflight > 8 || c.max_step_requests > 65536 || c.chunk % 32 || c.lane_blocks > 4096 ||
        c.max_step_draws > (1ull << 34))
        return fail(SRNG_ERR_ARG, "server configuration out of range");
    srng_server *srv = new (std::nothrow) srng_server();
    if (!srv) return fail(SRNG_ERR_OOM, "host allocation failed");
    srv->set = set;
    srv->cfg = c;
    cudaGetDevice(&srv->device);
    srng_status st = SRNG_OK;
    cudaError_t e;
    int sms = 0;
#define SRV_TRY(expr)                                                \
    do {                                                             \
        e = (expr);                                                  \
        if (e != cudaSuccess) { st = cuda_fail(e, #expr); goto bad; } \
    } while (0)
    SRV_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, srv->device));
    for (int t = 0; t < 3; ++t)
        srv->grid[t] = (unsigned)(sms * batch_blocks_per_sm((srng_out)t, batch_family(set)));
    SRV_TRY(cudaMalloc(&srv->pool_mem, c.budget_bytes));
    srv->pool.init(c.budget_bytes / 256 * 256);
    srv->n_ck = c.chunk ? 1 : kChunks;
    for (int k = 0; k < kChunks; ++k) srv->ck[k].chunk = c.chunk ? c.chunk : kDefaultChunk[k];
    for (int k = 0; k < srv->n_ck; ++k) chunk_jump_table(srv->ck[k].chunk, &srv->ck[k].tab);
    {
        // item buffers sized for the smallest chunk over a whole step
        const uint64_t per_item = set->gen == SRNG_MRG32K3A ? 32ull * srv->ck[0].chunk : 32ull * c.lane_blocks * 4;
        srv->cap_items = (uint32_t)(c.max_step_draws / per_item + 2ull * c.max_step_requests + 2);
    }
    srv->slots.resize(c.max_inflight);
    for (Slot &sl : srv->slots) {
        SRV_TRY(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
        SRV_TRY(cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming));
        const size_t desc_bytes = (c.max_step_requests * sizeof(BatchInst) + 15) / 16 * 16 +
                                  srv->cap_items * sizeof(uint2);
        SRV_TRY(cudaMallocHost(&sl.h_inst, desc_bytes));
        SRV_TRY(cudaMallocHost(&sl.h_items, srv->cap_items * sizeof(uint2)));
        SRV_TRY(cudaMalloc(&sl.d_inst, desc_bytes));
        SRV_TRY(cudaMalloc(&sl.d_counter, sizeof(uint32_t)));
        if (set->gen == SRNG_MRG32K3A)
            SRV_TRY(cudaMalloc(&sl.d_item_state, srv->cap_items * 6 * sizeof(uint32_t)));
    }
    if (set->gen == SRNG_MRG32K3A) {
        for (int k = 0; k < srv->n_ck; ++k) {
            uint32_t lane_tab[32 * 18];
            lane_jump_table(srv->ck[k].chunk, lane_tab);
            SRV_TRY(cudaMalloc(&srv->ck[k].d_lane_tab, sizeof lane_tab));
            SRV_TRY(cudaMemcpy(srv->ck[k].d_lane_tab, lane_tab, sizeof lane_tab, cudaMemcpyHostToDevice));
        }
    }
#undef SRV_TRY
    try {
        srv->th = std::thread(dispatcher, srv);
    } catch (...) {
        st = fail(SRNG_ERR_OOM, "cannot start the dispatcher thread");
        goto bad;
    }
    *out = srv;
    return SRNG_OK;
bad:
    server_free(srv);
    return st;
}

srng_status srng_server_submit(srng_server *srv, uint64_t stream, uint64_t n, srng_out type, uint64_t *ticket)
{
    clear_error();
    return submit_common(srv, stream, false, 0, n, type, false, ticket);
}

srng_status srng_server_submit_at(srng_server *srv, uint64_t stream, uint64_t pos, uint64_t n, srng_out type,
                                  uint64_t *ticket)
{
    clear_error();
    return submit_common(srv, stream, true, pos, n, type, false, ticket);
}

srng_status srng_server_poll(srng_server *srv, uint64_t ticket, int *done, const void **out_dev)
{
    clear_error();
    if (!srv || !done) return fail(SRNG_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(SRNG_ERR_CLOSED, "unknown ticket");
    *done = it->second.state == 2;
    if (out_dev) *out_dev = *done ? srv->pool_mem + it->second.pool_off : nullptr;
    if (srv->fault && !*done) return fail(srv->fault, "server stopped after an error: " + srv->fault_msg);
    return SRNG_OK;
}

srng_status srng_server_wait(srng_server *srv, uint64_t ticket, uint32_t timeout_ms, const void **out_dev)
{
    clear_error();
    if (!srv) return fail(SRNG_ERR_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(srv->mu);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        auto it = srv->reqs.find(ticket);
        if (it == srv->reqs.end()) return fail(SRNG_ERR_CLOSED, "unknown ticket");
        if (it->second.state == 2) {
            if (out_dev) *out_dev = srv->pool_mem + it->second.pool_off;
            return SRNG_OK;
        }
        if (srv->fault) return fail(srv->fault, "server stopped after an error: " + srv->fault_msg);
        if (srv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto it2 = srv->reqs.find(ticket);
            if (it2 != srv->reqs.end() && it2->second.state == 2) continue;
            return fail(SRNG_ERR_TIMEOUT, "request not complete within the timeout");
        }
    }
}

srng_status srng_server_release(srng_server *srv, uint64_t ticket)
{
    clear_error();
    if (!srv) return fail(SRNG_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(SRNG_ERR_CLOSED, "unknown ticket");
    if (it->second.state != 2) return fail(SRNG_ERR_ARG, "request not complete");
    srv->pool.release(it->second.pool_off, it->second.n * it->second.esz);
    srv->reqs.erase(it);
    srv->cv_work.notify_one();
    return SRNG_OK;
}

srng_status srng_server_read(srng_server *srv, uint64_t ticket, void *dst, int dst_is_host)
{
    clear_error();
    if (!srv || !dst) return fail(SRNG_ERR_ARG, "NULL argument");
    const char *src;
    uint64_t bytes;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->reqs.find(ticket);
        if (it == srv->reqs.end()) return fail(SRNG_ERR_CLOSED, "unknown ticket");
        if (it->second.state != 2) return fail(SRNG_ERR_ARG, "request not complete");
        src = srv->pool_mem + it->second.pool_off;
        bytes = it->second.n * it->second.esz;
    }
    SRNG_CUDA_TRY(cudaMemcpy(dst, src, bytes, dst_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice));
    return SRNG_OK;
}

srng_status srng_server_get_stats(srng_server *srv, srng_server_stats *out)
{
    clear_error();
    if (!srv || !out) return fail(SRNG_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    fill_stats(srv, out);
    return SRNG_OK;
}

srng_status srng_server_reset_stats(srng_server *srv)
{
    clear_error();
    if (!srv) return fail(SRNG_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->lat_us.clear();
    srv->submitted = srv->completed = srv->rejected = srv->draws_completed = srv->steps = srv->kernels = 0;
    srv->t_first = srv->t_last = 0;
    srv->pool.peak = srv->pool.used;
    return SRNG_OK;
}

srng_status srng_server_destroy(srng_server *srv)
{
    clear_error();
    if (!srv) return SRNG_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->pending.clear();
        srv->active.clear();
    }
    srv->cv_work.notify_all();
    if (srv->th.joinable()) srv->th.join();
    server_free(srv);
    return SRNG_OK;
}

srng_status srng_server_replay(srng_server *srv, const srng_request *req, uint64_t n_req, srng_out type,
                               double time_scale, uint32_t timeout_ms, srng_server_stats *out)
{
    clear_error();
    if (!srv || (n_req && !req)) return fail(SRNG_ERR_ARG, "NULL argument");
    srng_status st = check_type(type);
    if (st) return st;
    if ((st = srng_server_reset_stats(srv))) return st;
    const auto t0 = Clock::now();
    uint64_t ok = 0;
    for (uint64_t i = 0; i < n_req; ++i) {
        if (time_scale > 0) {
            const auto due = t0 + std::chrono::duration_cast<Clock::duration>(
                                      std::chrono::duration<double>(req[i].arrival_s * time_scale));
            std::this_thread::sleep_until(due);
        }
        st = submit_common(srv, req[i].stream, false, 0, req[i].n, type, true, nullptr);
        if (st == SRNG_OK) ++ok;
        else if (st != SRNG_ERR_BUDGET) return st;
    }
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
        while (srv->completed < ok && !srv->fault) {
            if (srv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && srv->completed < ok)
                return fail(SRNG_ERR_TIMEOUT, "replay did not complete within the timeout");
        }
        if (srv->fault) return fail(srv->fault, "server stopped after an error: " + srv->fault_msg);
        if (out) fill_stats(srv, out);
    }
    return SRNG_OK;
}

}  // extern "C"
