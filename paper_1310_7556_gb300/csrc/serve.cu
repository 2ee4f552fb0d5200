// Served mode: a trigger-style request loop with continuous batching.
//
// Events arrive one at a time (hough_serve_submit) and are appended to the batch that is filling.
// A dispatcher thread launches the filling batch as soon as fewer than max_in_flight batches are
// on the GPU, so events that arrive while others run are admitted into the next launch, and
// launches of different lanes overlap on the device (one stream per lane).  Each lane is a
// hough_batch (device buffers for max_batch_events accumulators, candidate lists and member
// pools, allocated once and kept resident) plus pinned host staging for its hits and results.
// Admission is bounded by those lanes, which the caller's device-memory budget sizes: when the
// filling batch is full and no lane is free to take the next one, an event is refused with
// HOUGH_EBUSY -- a trigger's dead time.
//
// Results come back without blocking the dispatcher: after the batch's graph the lane packs the
// candidates straight into mapped pinned host memory (up to its capacity) and copies the per-event
// offsets and counters; a batch with more candidates than that copies the rest once the offsets
// announce them.  Stream completions reach the dispatcher through
// host functions enqueued on the lane's stream; the dispatcher itself only polls flags, so a lane
// that never completes is caught by its watchdog (lane_timeout_us) instead of blocking the loop.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <ctime>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hough_internal.cuh"

using namespace hough;

namespace {

int64_t clock_ns()
{
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (int64_t)ts.tv_sec * 1000000000LL + ts.tv_nsec;
}

enum class LaneState { Free, Filling, Sealed, Running, Copying, Retired };

}  // namespace

struct hough_server;

namespace {

// The host buffers of one batch's candidates: a mapped pinned part the pack kernel writes the first
// `cap` candidates to, and a pinned overflow the rest of a larger batch is copied to.  A finished
// batch hands its block to its events' tickets (shared ownership) and the lane takes a spare block
// for its next launch, so the dispatcher copies no candidate: a poll copies its event's range
// straight to the caller, and the last ticket released returns the block to the pool.
struct ResultBlock {
    hough_candidate *host = nullptr;
    hough_candidate *dev = nullptr;    // its device address
    int64_t cap = 0;
    hough_candidate *over = nullptr;   // candidates cap.. of the batch
    int64_t over_cap = 0;
};

// Copy candidates [a, a + n) of a block's batch to `out`.
void copy_candidates(const ResultBlock &b, int64_t a, int64_t n, hough_candidate *out)
{
    const int64_t split = std::min(std::max(a, b.cap), a + n);   // [a, split) mapped, [split, a + n) overflow
    if (split > a) std::memcpy(out, b.host + a, sizeof(hough_candidate) * (split - a));
    if (a + n > split) std::memcpy(out + (split - a), b.over + (split - b.cap), sizeof(hough_candidate) * (a + n - split));
}

struct BlockPool {
    std::mutex mu;
    std::vector<ResultBlock *> free;
    int total = 0;       // blocks allocated
    int limit = 0;       // at most this many; beyond it results are copied out of the lane's block
    int64_t cap = 0;     // candidates in a block's mapped part
    int64_t over0 = 0;   // and in a new block's overflow (grown on demand)
    // overflows replaced by larger ones: freed only with the pool, since freeing pinned memory
    // synchronises the device and would stall the lanes in flight
    std::vector<hough_candidate *> retired;
    ~BlockPool()
    {
        for (ResultBlock *b : free) {
            cudaFreeHost(b->host);
            cudaFreeHost(b->over);
            delete b;
        }
        for (hough_candidate *p : retired) cudaFreeHost(p);
    }
};

// A free block of the pool, or a new one while the pool is below its limit; null otherwise (or when
// the allocation fails).  Never blocks on the device.
std::shared_ptr<ResultBlock> take_block(const std::shared_ptr<BlockPool> &pool)
{
    ResultBlock *b = nullptr;
    {
        std::lock_guard<std::mutex> g(pool->mu);
        if (!pool->free.empty()) {
            b = pool->free.back();
            pool->free.pop_back();
        } else if (pool->total < pool->limit) {
            ++pool->total;
        } else {
            return nullptr;
        }
    }
    if (!b) {
        b = new (std::nothrow) ResultBlock();
        bool ok = b && cudaHostAlloc(&b->host, sizeof(hough_candidate) * pool->cap, cudaHostAllocMapped) == cudaSuccess;
        ok = ok && cudaHostGetDevicePointer(reinterpret_cast<void **>(&b->dev), b->host, 0) == cudaSuccess;
        ok = ok && cudaHostAlloc(&b->over, sizeof(hough_candidate) * pool->over0, cudaHostAllocDefault) == cudaSuccess;
        if (ok) {
            b->cap = pool->cap;
            b->over_cap = pool->over0;
        } else {
            if (b) {
                if (b->host) cudaFreeHost(b->host);
                if (b->over) cudaFreeHost(b->over);
                delete b;
            }
            std::lock_guard<std::mutex> g(pool->mu);
            --pool->total;
            return nullptr;
        }
    }
    return std::shared_ptr<ResultBlock>(b, [pool](ResultBlock *x) {
        std::lock_guard<std::mutex> g(pool->mu);
        pool->free.push_back(x);
    });
}

struct Ticket {
    int64_t arrival_ns = 0, submit_ns = 0, launch_ns = 0, done_ns = 0;
    int32_t status = HOUGH_ENOTREADY;
    int32_t batch_events = 0;
    uint64_t votes = 0;
    uint32_t device_error = 0;
    int64_t n_candidates = 0;
    std::shared_ptr<ResultBlock> block;   // the candidates are [block_off, + n_candidates) of the block ...
    int64_t block_off = 0;
    std::vector<hough_candidate> cands;   // ... or, without a block, here
    bool done = false;
};

struct Lane {
    int index = 0;
    hough_server *server = nullptr;   // the host functions' argument is the lane itself
    hough_batch *b = nullptr;
    cudaStream_t stream = nullptr;
    // pinned staging of the filling batch's hits, and of the results
    float *r = nullptr, *phi = nullptr, *z = nullptr;
    uint8_t *layer = nullptr;
    int64_t *hit_start = nullptr;
    int32_t *offsets = nullptr;
    DevStats *stats = nullptr;
    std::shared_ptr<ResultBlock> blk;       // the pack kernel writes the first mcap candidates here
    int64_t mcap = 0;
    // the batch being filled or processed
    std::vector<Ticket *> tickets;
    int n_events = 0;          // events reserved (copies may still be in progress)
    int64_t n_hits = 0;        // hits reserved
    int copying = 0;           // submitters still copying into the staging
    LaneState state = LaneState::Free;
    int64_t launch_ns = 0;
    // set by host functions on the lane's stream
    std::atomic<int> phase_done{0};   // 1: offsets and counters are on the host; 2: candidates too
    int phase_wanted = 0;
};

void CUDART_CB lane_phase_done(void *p);

}  // namespace

struct hough_server {
    int device = 0;
    hough_serve_config cfg{};
    Axes ax{};
    std::vector<std::unique_ptr<Lane>> lanes;
    std::shared_ptr<BlockPool> pool = std::make_shared<BlockPool>();
    size_t device_bytes = 0;
    std::mutex mu;
    std::condition_variable cv_dispatch;   // wakes the dispatcher
    std::condition_variable cv_done;       // wakes pollers and drain
    std::thread dispatcher;
    bool stop = false;
    std::unordered_map<uint64_t, std::unique_ptr<Ticket>> tickets;
    uint64_t next_ticket = 1;
    Lane *filling = nullptr;
    std::deque<Lane *> sealed;             // full batches waiting for a launch, oldest first
    int running = 0;                       // lanes in Running or Copying
    // faults injected on the host side (hough_serve_inject)
    bool hold = false, stall = false, fail_alloc = false;
    hough_serve_stats st{};
    std::string last_error;

    ~hough_server();
    int live_lanes() const
    {
        int n = 0;
        for (auto &l : lanes) n += l->state != LaneState::Retired;
        return n;
    }
    int in_flight_limit() const { return std::max(1, std::min(cfg.max_in_flight, live_lanes() - 1)); }
    void run();
    int enqueue_batch(Lane *l);
    int enqueue_candidates(Lane *l, bool injected_alloc_failure);
    void fill_results(Lane *l);
    void complete_lane(Lane *l);
    void fail_lane(Lane *l, int status, bool retire, const char *why);
};

namespace {

void CUDART_CB lane_phase_done(void *p)
{
    // host function on the lane's stream: no CUDA calls here, only a flag and a wake-up
    Lane *l = static_cast<Lane *>(p);
    hough_server *s = l->server;
    {
        std::lock_guard<std::mutex> g(s->mu);
        l->phase_done.fetch_add(1);
    }
    s->cv_dispatch.notify_one();
}

}  // namespace

hough_server::~hough_server()
{
    {
        std::lock_guard<std::mutex> g(mu);
        stop = true;
    }
    cv_dispatch.notify_all();
    if (dispatcher.joinable()) dispatcher.join();
    cudaSetDevice(device);
    for (auto &l : lanes) {
        if (l->stream) cudaStreamSynchronize(l->stream);
        hough_batch_destroy(l->b);
        if (l->stream) cudaStreamDestroy(l->stream);
        cudaFreeHost(l->r);
        cudaFreeHost(l->phi);
        cudaFreeHost(l->z);
        cudaFreeHost(l->layer);
        cudaFreeHost(l->hit_start);
        cudaFreeHost(l->offsets);
        cudaFreeHost(l->stats);
    }
}

// Lanes in Running or Copying belong to the dispatcher alone: submitters only turn a Free lane
// into the Filling one and seal it, so the dispatcher may enqueue work and read results of its
// lanes without the mutex, and takes it only to publish state.

// Enqueue a batch: hit copies, the graph, the counters and offsets, then the phase-1 host
// function.  Unlocked; returns a status.
int hough_server::enqueue_batch(Lane *l)
{
    const int n = l->n_events;
    l->hit_start[0] = 0;   // the running offsets were written at submission
    l->phase_done.store(0);
    l->phase_wanted = 1;
    int rc = batch_run(l->b, l->r, l->phi, l->z, l->layer, l->hit_start, n, HOUGH_HOST, l->stream, false);
    if (!rc) rc = batch_enqueue_stats(l->b, l->stats, n, l->stream);
    if (!rc) rc = batch_enqueue_offsets_mapped(l->b, l->offsets, l->blk->dev, l->mcap, l->stream);
    if (!rc && cudaLaunchHostFunc(l->stream, lane_phase_done, l) != cudaSuccess)
        rc = set_last_error(HOUGH_ECUDA, "cudaLaunchHostFunc failed");
    return rc;
}

// Offsets and counters are on the host, and the first mcap candidates in the mapped buffer: enqueue
// the copy of the rest, growing the pinned overflow buffer first if needed.  Unlocked; returns a
// status.
int hough_server::enqueue_candidates(Lane *l, bool injected_alloc_failure)
{
    const int64_t total = l->offsets[l->n_events];
    const int64_t rest = total - l->mcap;
    ResultBlock &blk = *l->blk;
    if (rest > blk.over_cap || injected_alloc_failure) {
        int64_t cap = std::max<int64_t>(blk.over_cap, 1);
        while (cap < rest) cap *= 2;
        hough_candidate *grown = nullptr;
        if (injected_alloc_failure)
            return set_last_error(HOUGH_ENOMEM, "injected result-buffer allocation failure");
        if (cudaHostAlloc(&grown, sizeof(hough_candidate) * cap, cudaHostAllocDefault) != cudaSuccess)
            return set_last_error(HOUGH_ENOMEM, "pinned result buffer allocation failed");
        {
            std::lock_guard<std::mutex> g(pool->mu);
            pool->retired.push_back(blk.over);
        }
        blk.over = grown;
        blk.over_cap = cap;
    }
    l->phase_wanted = 2;
    int rc = batch_enqueue_candidates(l->b, blk.over, total, l->stream, l->mcap);
    if (!rc && cudaLaunchHostFunc(l->stream, lane_phase_done, l) != cudaSuccess)
        rc = set_last_error(HOUGH_ECUDA, "cudaLaunchHostFunc failed");
    return rc;
}

// Everything of the lane's batch is on the host: fill each event's result (unlocked; pollers
// look at a ticket only once `done` is published under the mutex).  With a spare block the
// events share the lane's block and the lane moves on to the spare; without one (the pollers lag
// and the pool is at its limit) each event's candidates are copied out and the lane keeps it.
void hough_server::fill_results(Lane *l)
{
    std::shared_ptr<ResultBlock> spare = take_block(pool);
    for (int e = 0; e < l->n_events; ++e) {
        Ticket *k = l->tickets[e];
        const int64_t a = l->offsets[e], b = l->offsets[e + 1];
        if (spare) {
            k->block = l->blk;
            k->block_off = a;
        } else {
            k->cands.resize((size_t)(b - a));
            copy_candidates(*l->blk, a, b - a, k->cands.data());
        }
        k->n_candidates = b - a;
        const DevStats &d = l->stats[e];
        uint64_t v = 0;
        for (int q = 0; q < HOUGH_MAX_LAYERS; ++q) v += d.votes_by_layer[q];
        k->votes = v;
        k->device_error = d.device_error;
        k->status = d.device_error ? HOUGH_EDEVICE : HOUGH_OK;
    }
    if (spare) l->blk = std::move(spare);
}

// Publish the lane's results and free it (mutex held).
void hough_server::complete_lane(Lane *l)
{
    const int64_t t = clock_ns();
    for (Ticket *k : l->tickets) {
        k->done_ns = t;
        k->done = true;
    }
    st.completed += l->n_events;
    l->tickets.clear();
    l->n_events = 0;
    l->n_hits = 0;
    l->state = LaneState::Free;
    --running;
}

// Give every event of the lane `status` and free the lane, or retire it when its stream cannot be
// trusted any more (its device buffers may still be in use).  Mutex held.
void hough_server::fail_lane(Lane *l, int status, bool retire, const char *why)
{
    const int64_t t = clock_ns();
    last_error = why;
    for (Ticket *k : l->tickets) {
        k->status = status;
        k->done_ns = t;
        k->done = true;
    }
    st.failed += (int64_t)l->tickets.size();
    l->tickets.clear();
    l->n_events = 0;
    l->n_hits = 0;
    if (l->state == LaneState::Running || l->state == LaneState::Copying) --running;
    l->state = retire ? LaneState::Retired : LaneState::Free;
    if (retire) st.retired_lanes += 1;
}

void hough_server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> g(mu);
    while (!stop) {
        bool progressed = false;
        // completions; a stalled stream is simulated by not looking at them
        for (auto &lp : lanes) {
            Lane *l = lp.get();
            if (l->state != LaneState::Running && l->state != LaneState::Copying) continue;
            if (!stall && l->phase_done.load() >= l->phase_wanted) {
                progressed = true;
                if (l->state == LaneState::Running) {
                    const bool inject = fail_alloc;
                    fail_alloc = false;
                    const bool fits = l->offsets[l->n_events] <= l->mcap;
                    g.unlock();
                    int rc = HOUGH_OK;
                    if (inject || !fits) rc = enqueue_candidates(l, inject);
                    else fill_results(l);   // every candidate is already in the mapped buffer
                    std::string why = rc ? hough_last_error() : "";
                    g.lock();
                    if (rc) {
                        if (rc == HOUGH_ENOMEM) st.alloc_failures += 1;
                        fail_lane(l, rc, rc != HOUGH_ENOMEM, why.c_str());
                    } else if (inject || !fits) {
                        l->state = LaneState::Copying;
                    } else {
                        complete_lane(l);
                    }
                } else {
                    g.unlock();
                    fill_results(l);
                    g.lock();
                    complete_lane(l);
                }
            } else if (cfg.lane_timeout_us > 0 && clock_ns() - l->launch_ns > cfg.lane_timeout_us * 1000) {
                progressed = true;
                st.timeouts += 1;
                fail_lane(l, HOUGH_ETIMEDOUT, true, "a launch did not finish within lane_timeout_us; its lane is retired");
            }
        }
        // launches: full batches first, then the filling one, while the in-flight limit allows
        while (!hold && running < in_flight_limit()) {
            Lane *l = nullptr;
            if (!sealed.empty() && sealed.front()->copying == 0) {
                l = sealed.front();
                sealed.pop_front();
            } else if (sealed.empty() && filling && filling->n_events > 0 && filling->copying == 0) {
                l = filling;
                filling = nullptr;
            }
            if (!l) break;
            progressed = true;
            l->state = LaneState::Running;
            ++running;
            st.max_in_flight = std::max<int64_t>(st.max_in_flight, running);
            st.launches += 1;
            st.launched_events += l->n_events;
            const int64_t t = clock_ns();
            l->launch_ns = t;
            for (Ticket *k : l->tickets) {
                k->launch_ns = t;
                k->batch_events = l->n_events;
            }
            g.unlock();
            const int rc = enqueue_batch(l);
            std::string why = rc ? hough_last_error() : "";
            g.lock();
            // a failed enqueue may have left work on the stream: retire the lane
            if (rc) fail_lane(l, rc, true, why.c_str());
        }
        if (progressed) {
            cv_done.notify_all();
            continue;
        }
        cv_dispatch.wait_for(g, std::chrono::microseconds(running > 0 ? 200 : 5000));
    }
}

extern "C" {

int hough_serve_create(const hough_geometry *geometry, const hough_binning *binning, const hough_serve_config *config,
                       int device, hough_server **out)
{
    if (!out || !config) return set_last_error(HOUGH_EINVAL, "config and out are required");
    *out = nullptr;
    int rc = check_geometry_binning(geometry, binning);
    if (rc) return rc;
    hough_serve_config c = *config;
    if (c.lanes < 0 || c.lanes == 1 || c.max_in_flight < 0 || c.max_batch_events < 1 || c.max_batch_hits < 1 ||
        c.max_batch_hits > (1LL << 31) - 1 || c.max_candidates < 1 || c.max_members < 1 || c.memory_budget < 0 ||
        c.lane_timeout_us < 0 || c.reserved != 0)
        return set_last_error(HOUGH_EINVAL, "serve config out of range");
    if (c.lanes > 0 && c.max_in_flight >= c.lanes)
        return set_last_error(HOUGH_EINVAL, "max_in_flight must be below lanes (one lane fills while the others run)");
    auto s = std::unique_ptr<hough_server>(new (std::nothrow) hough_server());
    if (!s) return set_last_error(HOUGH_ENOMEM, "host allocation failed");
    s->device = device;
    s->ax = make_axes(geometry, binning);
    const int want = c.lanes > 0 ? c.lanes : 4;
    if (cudaSetDevice(device) != cudaSuccess) return set_last_error(HOUGH_EINVAL, "cudaSetDevice failed");
    hough_batch_limits lim{c.max_batch_events, c.max_candidates, c.max_batch_hits, c.max_members, 0};
    const int E = c.max_batch_events;
    const int64_t H = c.max_batch_hits;
    for (int i = 0; i < want; ++i) {
        auto l = std::make_unique<Lane>();
        l->index = i;
        l->server = s.get();
        hough_batch *b = nullptr;
        rc = hough_batch_create(geometry, binning, &lim, device, &b);
        if (rc) {
            if (rc == HOUGH_ENOMEM && c.lanes == 0 && i >= 2) break;   // as many as fit
            return rc;
        }
        l->b = b;
        const size_t bytes = batch_device_bytes(b);
        if (c.memory_budget > 0 && s->device_bytes + bytes > (size_t)c.memory_budget) {
            hough_batch_destroy(b);
            l->b = nullptr;
            if (i >= 2 && c.lanes == 0) break;
            return set_last_error(HOUGH_ENOMEM, c.lanes == 0 || i < 2
                                                    ? "the memory budget does not hold two lanes"
                                                    : "the memory budget does not hold the requested lanes");
        }
        s->device_bytes += bytes;
        bool ok = cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking) == cudaSuccess;
        l->mcap = std::max<int64_t>(1 << 14, (int64_t)E * 1024);
        ok = ok && cudaHostAlloc(&l->r, sizeof(float) * H, cudaHostAllocDefault) == cudaSuccess;
        ok = ok && cudaHostAlloc(&l->phi, sizeof(float) * H, cudaHostAllocDefault) == cudaSuccess;
        ok = ok && cudaHostAlloc(&l->z, sizeof(float) * H, cudaHostAllocDefault) == cudaSuccess;
        ok = ok && cudaHostAlloc(&l->layer, H, cudaHostAllocDefault) == cudaSuccess;
        ok = ok && cudaHostAlloc(&l->hit_start, sizeof(int64_t) * (E + 1), cudaHostAllocDefault) == cudaSuccess;
        ok = ok && cudaHostAlloc(&l->offsets, sizeof(int32_t) * (E + 1), cudaHostAllocDefault) == cudaSuccess;
        ok = ok && cudaHostAlloc(&l->stats, sizeof(DevStats) * E, cudaHostAllocDefault) == cudaSuccess;
        if (i == 0) {
            // every lane's block, as many spares, and room for as many again while pollers lag
            s->pool->cap = l->mcap;
            s->pool->over0 = std::max<int64_t>(1 << 14, (int64_t)E * 256);
            s->pool->limit = 3 * want;
        }
        l->blk = ok ? take_block(s->pool) : nullptr;
        ok = ok && l->blk;
        s->lanes.push_back(std::move(l));
        if (!ok) return set_last_error(HOUGH_ENOMEM, "lane allocation failed");
    }
    if (s->lanes.size() < 2) return set_last_error(HOUGH_ENOMEM, "fewer than two lanes fit");
    {
        // a spare result block per lane now, so that no completion in service waits on an allocation
        std::vector<std::shared_ptr<ResultBlock>> spares;
        for (size_t i = 0; i < s->lanes.size(); ++i)
            if (auto b = take_block(s->pool)) spares.push_back(std::move(b));
    }
    c.lanes = (int)s->lanes.size();
    if (c.max_in_flight == 0) c.max_in_flight = c.lanes - 1;
    s->cfg = c;
    s->st.lanes = c.lanes;
    s->st.device_bytes = (int64_t)s->device_bytes;
    // capture every batch size's graph now (empty events), so that no launch in service pays it
    for (auto &l : s->lanes) {
        for (int n = 1; n <= E; ++n) {
            for (int e = 0; e <= n; ++e) l->hit_start[e] = 0;
            rc = batch_run(l->b, l->r, l->phi, l->z, l->layer, l->hit_start, n, HOUGH_HOST, l->stream, false);
            if (rc) return rc;
        }
        if (cudaStreamSynchronize(l->stream) != cudaSuccess) return set_last_error(HOUGH_ECUDA, "warm-up failed");
    }
    s->dispatcher = std::thread([p = s.get()] { p->run(); });
    *out = s.release();
    return HOUGH_OK;
}

void hough_serve_destroy(hough_server *s) { delete s; }

int64_t hough_serve_clock_ns(void) { return clock_ns(); }

int hough_serve_submit(hough_server *s, const float *r, const float *phi, const float *z, const uint8_t *layer,
                       int64_t n_hits, int64_t arrival_ns, uint64_t *ticket)
{
    const int64_t t_submit = clock_ns();
    if (!s || !ticket) return set_last_error(HOUGH_EINVAL, "server and ticket are required");
    if (n_hits < 0 || (n_hits > 0 && (!r || !phi || !z || !layer))) return set_last_error(HOUGH_EINVAL, "bad hit arrays");
    if (n_hits > s->cfg.max_batch_hits) return set_last_error(HOUGH_ECAPACITY, "the event has more hits than max_batch_hits");
    auto fits = [&](const Lane *x) {
        return x->n_events < s->cfg.max_batch_events && x->n_hits + n_hits <= s->cfg.max_batch_hits;
    };
    auto room = [&] {
        if (s->filling && fits(s->filling)) return true;
        for (auto &lp : s->lanes)
            if (lp->state == LaneState::Free) return true;
        return false;
    };
    {
        // refusing an event in dead time costs no pass over its hits
        std::lock_guard<std::mutex> g(s->mu);
        if (!room()) {
            s->st.submitted += 1;
            s->st.rejected_busy += 1;
            return set_last_error(HOUGH_EBUSY, "every lane is full or on the GPU");
        }
    }
    // a malformed event is refused here and never reaches a batch
    int rc = check_host_hits_for(s->ax, r, phi, z, layer, n_hits);
    if (rc) {
        std::lock_guard<std::mutex> g(s->mu);
        s->st.submitted += 1;
        s->st.rejected_invalid += 1;
        return rc;
    }
    Lane *l = nullptr;
    int64_t at = 0;
    int slot = 0;
    Ticket *k = nullptr;
    uint64_t id = 0;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->st.submitted += 1;
        if (s->filling && !fits(s->filling)) {
            s->filling->state = LaneState::Sealed;
            s->sealed.push_back(s->filling);
            s->filling = nullptr;
        }
        if (!s->filling) {
            for (auto &lp : s->lanes)
                if (lp->state == LaneState::Free) {
                    s->filling = lp.get();
                    s->filling->state = LaneState::Filling;
                    break;
                }
        }
        if (!s->filling) {
            s->st.rejected_busy += 1;
            return set_last_error(HOUGH_EBUSY, "every lane is full or on the GPU");
        }
        l = s->filling;
        slot = l->n_events++;
        at = l->n_hits;
        l->n_hits += n_hits;
        l->hit_start[slot + 1] = at + n_hits;
        l->copying += 1;
        id = s->next_ticket++;
        auto t = std::make_unique<Ticket>();
        k = t.get();
        k->arrival_ns = arrival_ns > 0 ? arrival_ns : t_submit;
        k->submit_ns = t_submit;
        l->tickets.push_back(k);
        s->tickets.emplace(id, std::move(t));
        s->st.admitted += 1;
    }
    if (n_hits > 0) {
        std::memcpy(l->r + at, r, sizeof(float) * n_hits);
        std::memcpy(l->phi + at, phi, sizeof(float) * n_hits);
        std::memcpy(l->z + at, z, sizeof(float) * n_hits);
        std::memcpy(l->layer + at, layer, n_hits);
    }
    {
        std::lock_guard<std::mutex> g(s->mu);
        l->copying -= 1;
    }
    s->cv_dispatch.notify_one();
    *ticket = id;
    return HOUGH_OK;
}

int hough_serve_poll(hough_server *s, uint64_t ticket, hough_candidate *out, int64_t cap, hough_serve_result *result,
                     int64_t timeout_us)
{
    if (!s || cap < 0 || (cap > 0 && !out) || timeout_us < 0) return set_last_error(HOUGH_EINVAL, "bad arguments");
    std::unique_lock<std::mutex> g(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return set_last_error(HOUGH_EINVAL, "unknown ticket");
    Ticket *k = it->second.get();
    if (!k->done) {
        s->cv_done.wait_for(g, std::chrono::microseconds(timeout_us), [&] { return k->done; });
        if (!k->done) return set_last_error(HOUGH_ETIMEDOUT, "the event has not finished within the timeout");
    }
    std::unique_ptr<Ticket> t = std::move(it->second);
    s->tickets.erase(it);
    std::string why = k->status == HOUGH_OK ? std::string() : s->last_error;
    g.unlock();
    if (result) {
        result->ticket = ticket;
        result->arrival_ns = t->arrival_ns;
        result->submit_ns = t->submit_ns;
        result->launch_ns = t->launch_ns;
        result->done_ns = t->done_ns;
        result->n_candidates = t->n_candidates;
        result->votes = t->votes;
        result->status = t->status;
        result->batch_events = t->batch_events;
        result->device_error = t->device_error;
        result->reserved = 0;
    }
    if (cap > 0 && t->n_candidates > 0) {
        const int64_t n = std::min<int64_t>(cap, t->n_candidates);
        if (t->block) copy_candidates(*t->block, t->block_off, n, out);
        else std::memcpy(out, t->cands.data(), sizeof(hough_candidate) * n);
    }
    if (t->status != HOUGH_OK)
        return set_last_error(t->status, why.empty() ? "the event failed" : why.c_str());
    if (t->n_candidates > cap && cap >= 0 && out != nullptr)
        return set_last_error(HOUGH_ETRUNC, "more candidates than the capacity");
    return HOUGH_OK;
}

int hough_serve_drain(hough_server *s, int64_t timeout_us)
{
    if (!s || timeout_us < 0) return set_last_error(HOUGH_EINVAL, "bad arguments");
    std::unique_lock<std::mutex> g(s->mu);
    s->cv_dispatch.notify_one();
    const bool ok = s->cv_done.wait_for(g, std::chrono::microseconds(timeout_us), [&] {
        bool idle = s->running == 0 && s->sealed.empty() && (!s->filling || s->filling->n_events == 0);
        return idle;
    });
    if (!ok) return set_last_error(HOUGH_ETIMEDOUT, "the server did not drain within the timeout");
    return HOUGH_OK;
}

int hough_serve_get_stats(hough_server *s, hough_serve_stats *out)
{
    if (!s || !out) return set_last_error(HOUGH_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->st;
    out->lanes = s->live_lanes();
    out->in_flight = s->running;
    out->pending_tickets = (int64_t)s->tickets.size();
    return HOUGH_OK;
}

int hough_serve_replay(hough_server *s, const hough_event_view *pool, int32_t n_pool, const int64_t *arrival_ns,
                       int64_t n, int32_t threads, hough_serve_result *results)
{
    if (!s || !pool || n_pool < 1 || !arrival_ns || n < 0 || threads < 1 || threads > 64 || !results)
        return set_last_error(HOUGH_EINVAL, "bad arguments");
    for (int32_t q = 0; q < n_pool; ++q)
        if (pool[q].n_hits < 0 || (pool[q].n_hits > 0 && (!pool[q].r || !pool[q].phi || !pool[q].z || !pool[q].layer)))
            return set_last_error(HOUGH_EINVAL, "bad pool event");
    // ticket of arrival i once submitted: kPending until then, 0 when refused
    constexpr uint64_t kPending = ~0ull;
    std::vector<std::atomic<uint64_t>> ticket(n);
    for (int64_t i = 0; i < n; ++i) ticket[i].store(kPending, std::memory_order_relaxed);
    std::vector<int32_t> refused(n, 0);
    auto submitter = [&](int t) {
        for (int64_t i = t; i < n; i += threads) {
            const int64_t a = arrival_ns[i];
            for (int64_t now = clock_ns(); now < a; now = clock_ns())
                if (a - now > 200000) std::this_thread::sleep_for(std::chrono::nanoseconds(a - now - 100000));
            const hough_event_view &ev = pool[i % n_pool];
            uint64_t id = 0;
            const int rc = hough_serve_submit(s, ev.r, ev.phi, ev.z, ev.layer, ev.n_hits, a, &id);
            refused[i] = rc;
            ticket[i].store(rc == HOUGH_OK ? id : 0ull, std::memory_order_release);
        }
    };
    int consumer_rc = HOUGH_OK;
    auto consumer = [&] {
        for (int64_t i = 0; i < n; ++i) {
            uint64_t id;
            while ((id = ticket[i].load(std::memory_order_acquire)) == kPending) std::this_thread::yield();
            hough_serve_result &r = results[i];
            std::memset(&r, 0, sizeof(r));
            if (id == 0) {
                r.arrival_ns = arrival_ns[i];
                r.status = refused[i];
                continue;
            }
            int rc = HOUGH_ETIMEDOUT;
            // a result arrives within a few launches; the bound keeps a stalled server from blocking
            for (int k = 0; k < 600 && rc == HOUGH_ETIMEDOUT; ++k) {
                rc = hough_serve_poll(s, id, nullptr, 0, &r, 100000);
                if (rc == HOUGH_ETIMEDOUT && r.ticket == id) break;   // finished with status ETIMEDOUT
            }
            if (rc == HOUGH_ETIMEDOUT && r.ticket != id) {
                r.ticket = id;
                r.arrival_ns = arrival_ns[i];
                r.status = HOUGH_ETIMEDOUT;
                consumer_rc = HOUGH_ETIMEDOUT;
            }
        }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < threads; ++t) th.emplace_back(submitter, t);
    std::thread cons(consumer);
    for (auto &x : th) x.join();
    cons.join();
    if (consumer_rc) return set_last_error(consumer_rc, "some events had no result within 60 s");
    return HOUGH_OK;
}

int hough_serve_inject(hough_server *s, int fault, int on)
{
    if (!s) return set_last_error(HOUGH_EINVAL, "server is required");
    {
        std::lock_guard<std::mutex> g(s->mu);
        switch (fault) {
        case HOUGH_SERVE_FAULT_HOLD: s->hold = on != 0; break;
        case HOUGH_SERVE_FAULT_STALL: s->stall = on != 0; break;
        case HOUGH_SERVE_FAULT_ALLOC: s->fail_alloc = on != 0; break;
        default: return set_last_error(HOUGH_EINVAL, "unknown fault");
        }
    }
    s->cv_dispatch.notify_one();
    return HOUGH_OK;
}

}  // extern "C"
