// Batched processing: many events of uneven size through the whole path in one launch sequence.
//
// Every kernel of the path already works on a batch (hits of all events concatenated, per-event
// accumulators and lists at fixed strides, grids spanning all events' tiles, bands and
// candidates), so a batch costs the same dozen launches as a single event.  The launch sequence
// is captured once per batch size into a CUDA graph and replayed: the kernels read the hit total
// and the hit pointers from device memory, so the same graph serves every batch of that size.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "hough_internal.cuh"

using namespace hough;

namespace {

int bfail(int code, const char *msg) { return set_last_error(code, msg); }

#define BCU(call, what)                                                                       \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bfail(e_ == cudaErrorMemoryAllocation ? HOUGH_ENOMEM : HOUGH_ECUDA, what); \
    } while (0)

}  // namespace

struct hough_batch {
    int device = 0;
    int sms = 0;
    Axes ax{};
    Tiling tiling{};
    float refine_eps = 0.f;
    hough_batch_limits limits{};
    Workspace w{};
    std::vector<void *> allocations;
    int64_t *hit_start = nullptr;        // device, max_events + 1
    HitInputs *inputs_dev = nullptr;     // device copy of the current hit pointers
    HitInputs inputs_host{};
    HitInputs inputs_on_device{};        // what inputs_dev holds (copied only when it changes)
    float *in_r = nullptr, *in_phi = nullptr, *in_z = nullptr;
    uint8_t *in_layer = nullptr;
    hough_candidate *packed = nullptr;   // all events' candidates, concatenated
    cudaStream_t capture_stream = nullptr;
    std::map<int, cudaGraphExec_t> graphs;   // by batch size
    int n_events = 0;                        // of the last run
    bool ran = false;
    size_t device_bytes = 0;                 // everything allocated above

    ~hough_batch()
    {
        cudaSetDevice(device);
        cudaDeviceSynchronize();
        for (auto &g : graphs) cudaGraphExecDestroy(g.second);
        if (capture_stream) cudaStreamDestroy(capture_stream);
        for (void *p : allocations) cudaFree(p);
    }

    template <typename T>
    cudaError_t alloc(T **p, size_t count)
    {
        void *q = nullptr;
        const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e == cudaSuccess) {
            allocations.push_back(q);
            device_bytes += bytes;
        }
        *p = static_cast<T *>(q);
        return e;
    }

    // The whole path on the current batch, enqueued on `s` (also the body of the captured graph).
    cudaError_t enqueue(cudaStream_t s)
    {
        cudaError_t e;
        if ((e = launch_stage(ax, w, s))) return e;
        if (tiling.vote_mode != HOUGH_VOTE_SCATTER && (e = launch_gather(ax, w, tiling, s))) return e;
        if ((e = launch_scatter(ax, w, tiling, refine_eps, tiling.vote_mode != HOUGH_VOTE_SCATTER, s))) return e;
        if ((e = launch_band_peaks(ax, w, tiling, s))) return e;
        if ((e = launch_compact(ax, w, s))) return e;
        return launch_stage2(ax, w, sms, refine_eps, s);
    }
};

extern "C" {

int hough_batch_create(const hough_geometry *geometry, const hough_binning *binning, const hough_batch_limits *limits,
                       int device, hough_batch **out)
{
    if (!out) return bfail(HOUGH_EINVAL, "out is required");
    *out = nullptr;
    int rc = check_geometry_binning(geometry, binning);
    if (rc) return rc;
    if (!limits || limits->max_events < 1 || limits->max_hits < 1 || limits->max_hits > (1LL << 31) - 1 ||
        limits->max_candidates < 1 || limits->max_members < 1 || limits->reserved != 0)
        return bfail(HOUGH_EINVAL, "batch limits: max_events, max_hits (< 2^31), max_candidates, max_members >= 1");
    int ndev = 0;
    BCU(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount failed");
    if (device < 0 || device >= ndev) return bfail(HOUGH_EINVAL, "device out of range");
    BCU(cudaSetDevice(device), "cudaSetDevice failed");
    hough_batch *b = new (std::nothrow) hough_batch();
    if (!b) return bfail(HOUGH_ENOMEM, "host allocation failed");
    b->device = device;
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, device);
    b->ax = make_axes(geometry, binning);
    b->tiling = default_tiling_for(b->ax);
    b->refine_eps = refine_eps_for(b->ax);
    b->limits = *limits;
    const Axes &ax = b->ax;
    const int64_t E = limits->max_events, H = limits->max_hits, C = limits->max_candidates, Mm = limits->max_members;
    const int nkeys = n_keys(ax);
    Workspace &w = b->w;
    w.max_cand = (int)C;
    w.max_members = (int)Mm;
    w.n_hits_total = -1;           // read on the device
    w.hit_capacity = H;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(b->alloc(&b->hit_start, E + 1));
    A(b->alloc(&b->inputs_dev, 1));
    A(b->alloc(&b->in_r, H)); A(b->alloc(&b->in_phi, H)); A(b->alloc(&b->in_z, H)); A(b->alloc(&b->in_layer, H));
    A(b->alloc(&w.key, H)); A(b->alloc(&w.rank, H)); A(b->alloc(&w.hot_tmp, H));
    A(b->alloc(&w.hot, H)); A(b->alloc(&w.cold, H)); A(b->alloc(&w.fsort, H)); A(b->alloc(&w.zsort, H));
    A(b->alloc(&w.counts, E * nkeys)); A(b->alloc(&w.offs, E * (nkeys + 1)));
    A(b->alloc(&w.prof, (size_t)(E * prof_event_entries(ax))));
    A(b->alloc(&w.radii, 1)); A(b->alloc(&w.info, HOUGH_MAX_LAYERS)); A(b->alloc(&w.memo, 1));
    A(b->alloc(&w.tab, (size_t)ax.n_layers * ax.n_qpt)); A(b->alloc(&w.arc, (size_t)ax.n_layers * ax.n_qpt));
    A(b->alloc(&w.zco, (size_t)ax.n_layers * ax.n_qpt));
    A(b->alloc(&w.kq32, ax.n_qpt));
    A(b->alloc(&w.M, (size_t)E * ax.n_qpt * ax.n_phi));
    A(b->alloc(&w.band_cands, (size_t)E * band_list_entries(ax)));
    A(b->alloc(&w.band_counts, (size_t)E * n_bands(ax, 1))); A(b->alloc(&w.band_offs, (size_t)E * n_bands(ax, 1)));
    A(b->alloc(&w.cands, E * C));
    A(b->alloc(&w.cand_base, E + 1)); A(b->alloc(&w.counters, 1));
    A(b->alloc(&w.stats, E));
    A(b->alloc(&b->packed, E * C));
    if (e != cudaSuccess) {
        delete b;
        return bfail(e == cudaErrorMemoryAllocation ? HOUGH_ENOMEM : HOUGH_ECUDA, "hough_batch_create allocation failed");
    }
    w.hit_start = b->hit_start;
    w.inputs = b->inputs_dev;
    w.band_rows = b->tiling.band_rows;
    w.band_cap = band_capacity(ax, b->tiling.band_rows);
    w.fused = b->tiling.vote_mode == HOUGH_VOTE_FUSED;
    std::vector<float> kq(ax.n_qpt);
    for (int i = 0; i < ax.n_qpt; ++i) kq[i] = (float)(ax.qpt_min + (i % ax.q_rows + 0.5) * ax.dk);
    A(cudaMemcpy(w.kq32, kq.data(), sizeof(float) * ax.n_qpt, cudaMemcpyHostToDevice));
    A(cudaMemset(w.memo, 0, sizeof(TableMemo)));
    A(cudaMemset(b->inputs_dev, 0, sizeof(HitInputs)));   // as inputs_on_device says
    A(cudaMemset(w.stats, 0, sizeof(DevStats) * E));
    A(cudaMemset(w.cand_base, 0, sizeof(int32_t) * (E + 1)));
    A(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
    A(cudaDeviceSynchronize());
    if (e != cudaSuccess) {
        delete b;
        return bfail(HOUGH_ECUDA, "hough_batch_create initialisation failed");
    }
    *out = b;
    return HOUGH_OK;
}

void hough_batch_destroy(hough_batch *b) { delete b; }

int hough_batch_set_tiling(hough_batch *b, const hough_tiling *t)
{
    if (!b) return bfail(HOUGH_EINVAL, "batch is required");
    int rc = check_tiling_for(b->ax, b->device, t);
    if (rc) return rc;
    b->tiling = resolve_tiling(b->ax, t);
    b->w.band_rows = t->band_rows;
    b->w.band_cap = band_capacity(b->ax, t->band_rows);
    b->w.fused = b->tiling.vote_mode == HOUGH_VOTE_FUSED;
    // captured graphs hold the old configuration
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
    return HOUGH_OK;
}

}  // extern "C"

// Checks of a run's arguments, the copies of its inputs and hit offsets (enqueued on `stream`).
static int batch_prepare(hough_batch *b, const float *r, const float *phi, const float *z, const uint8_t *layer,
                         const int64_t *hit_start, int32_t n_events, int where, cudaStream_t stream, bool check_hits)
{
    if (!b || !hit_start) return bfail(HOUGH_EINVAL, "batch and hit_start are required");
    if (n_events < 1 || n_events > b->limits.max_events) return bfail(HOUGH_ECAPACITY, "n_events outside 1..max_events");
    if (where != HOUGH_HOST && where != HOUGH_DEVICE) return bfail(HOUGH_EINVAL, "where must be HOUGH_HOST or HOUGH_DEVICE");
    if (hit_start[0] != 0) return bfail(HOUGH_EINVAL, "hit_start[0] must be 0");
    for (int e = 0; e < n_events; ++e)
        if (hit_start[e + 1] < hit_start[e]) return bfail(HOUGH_EINVAL, "hit_start must not decrease");
    const int64_t n = hit_start[n_events];
    if (n > b->limits.max_hits) return bfail(HOUGH_ECAPACITY, "the batch has more hits than max_hits");
    if (n > 0 && (!r || !phi || !z || !layer)) return bfail(HOUGH_EINVAL, "hit arrays are required");
    BCU(cudaSetDevice(b->device), "cudaSetDevice failed");
    cudaStream_t s = stream;
    if (where == HOUGH_HOST) {
        if (check_hits) {
            int rc = check_host_hits_for(b->ax, r, phi, z, layer, n);
            if (rc) return rc;
        }
        if (n > 0) {
            BCU(cudaMemcpyAsync(b->in_r, r, sizeof(float) * n, cudaMemcpyHostToDevice, s), "copy r failed");
            BCU(cudaMemcpyAsync(b->in_phi, phi, sizeof(float) * n, cudaMemcpyHostToDevice, s), "copy phi failed");
            BCU(cudaMemcpyAsync(b->in_z, z, sizeof(float) * n, cudaMemcpyHostToDevice, s), "copy z failed");
            BCU(cudaMemcpyAsync(b->in_layer, layer, n, cudaMemcpyHostToDevice, s), "copy layer failed");
        }
        b->inputs_host = HitInputs{b->in_r, b->in_phi, b->in_z, b->in_layer};
    } else {
        b->inputs_host = HitInputs{r, phi, z, layer};
    }
    // the next replay reads these through device memory; the record changes only when the caller
    // switches buffers (copies from pageable host memory are staged before the call returns)
    if (std::memcmp(&b->inputs_host, &b->inputs_on_device, sizeof(HitInputs)) != 0) {
        BCU(cudaMemcpyAsync(b->inputs_dev, &b->inputs_host, sizeof(HitInputs), cudaMemcpyHostToDevice, s),
            "copy inputs failed");
        b->inputs_on_device = b->inputs_host;
    }
    BCU(cudaMemcpyAsync(b->hit_start, hit_start, sizeof(int64_t) * (n_events + 1), cudaMemcpyHostToDevice, s),
        "copy hit_start failed");
    b->w.n_events = n_events;
    return HOUGH_OK;
}

int hough::batch_run(hough_batch *b, const float *r, const float *phi, const float *z, const uint8_t *layer,
                     const int64_t *hit_start, int32_t n_events, int where, cudaStream_t stream, bool check_hits)
{
    int rc = batch_prepare(b, r, phi, z, layer, hit_start, n_events, where, stream, check_hits);
    if (rc) return rc;
    cudaStream_t s = stream;
    auto it = b->graphs.find(n_events);
    if (it == b->graphs.end()) {
        // capture on the library's own stream, ordered after the copies above
        cudaEvent_t ready;
        BCU(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming), "event failed");
        BCU(cudaEventRecord(ready, s), "event record failed");
        BCU(cudaStreamWaitEvent(b->capture_stream, ready, 0), "stream wait failed");
        BCU(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeRelaxed), "capture begin failed");
        cudaError_t ce = b->enqueue(b->capture_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t ee = cudaStreamEndCapture(b->capture_stream, &graph);
        cudaEventDestroy(ready);
        if (ce != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return bfail(HOUGH_ECUDA, "capturing the batch launch sequence failed");
        }
        cudaGraphExec_t exec = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return bfail(HOUGH_ECUDA, "instantiating the batch graph failed");
        it = b->graphs.emplace(n_events, exec).first;
    }
    BCU(cudaGraphLaunch(it->second, s), "graph launch failed");
    note_launches(kStageLaunches + kVoteLaunches + peak_launches(n_events) + kStage2Launches);
    b->n_events = n_events;
    b->ran = true;
    return HOUGH_OK;
}

// Enqueue the concatenation of the last run's candidates into the batch's device buffer and the
// copy of the per-event offsets (int32, n_events + 1) to `offsets_host`; no synchronisation.
int hough::batch_enqueue_offsets(hough_batch *b, int32_t *offsets_host, cudaStream_t s)
{
    BCU(launch_pack_candidates(b->ax, b->w, b->packed, s), "pack kernel failed");
    note_launches(1);
    BCU(cudaMemcpyAsync(offsets_host, b->w.cand_base, sizeof(int32_t) * (b->n_events + 1), cudaMemcpyDeviceToHost, s),
        "copy offsets failed");
    return HOUGH_OK;
}

int hough::batch_enqueue_offsets_mapped(hough_batch *b, int32_t *offsets_host, hough_candidate *mapped, int64_t cap,
                                        cudaStream_t s)
{
    BCU(launch_pack_candidates(b->ax, b->w, mapped, s, cap, b->packed), "pack kernel failed");   // the rest stays on the device
    note_launches(1);
    BCU(cudaMemcpyAsync(offsets_host, b->w.cand_base, sizeof(int32_t) * (b->n_events + 1), cudaMemcpyDeviceToHost, s),
        "copy offsets failed");
    return HOUGH_OK;
}

// Enqueue the copy of the first n events' counters to `stats_host`; no synchronisation.
int hough::batch_enqueue_stats(hough_batch *b, DevStats *stats_host, int n, cudaStream_t s)
{
    BCU(cudaMemcpyAsync(stats_host, b->w.stats, sizeof(DevStats) * n, cudaMemcpyDeviceToHost, s), "copy stats failed");
    return HOUGH_OK;
}

size_t hough::batch_device_bytes(const hough_batch *b) { return b->device_bytes; }

// Enqueue the copy of packed candidates [first, n) to dst_host[0, n - first); no synchronisation.
int hough::batch_enqueue_candidates(hough_batch *b, hough_candidate *dst_host, int64_t n, cudaStream_t s,
                                    int64_t first)
{
    if (n > first)
        BCU(cudaMemcpyAsync(dst_host, b->packed + first, sizeof(hough_candidate) * (n - first),
                            cudaMemcpyDeviceToHost, s),
            "copy candidates failed");
    return HOUGH_OK;
}

extern "C" {

// The launch sequence of hough_batch_run enqueued kernel by kernel (not the captured graph), with a
// CUDA event on `stream` after each step, so that each step's device time can be read.
int hough_batch_profile(hough_batch *b, const float *r, const float *phi, const float *z, const uint8_t *layer,
                        const int64_t *hit_start, int32_t n_events, int where, void *stream, hough_timing *out)
{
    if (!out) return bfail(HOUGH_EINVAL, "out is required");
    int rc = batch_prepare(b, r, phi, z, layer, hit_start, n_events, where, static_cast<cudaStream_t>(stream), true);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t ev[7] = {};
    for (auto &e : ev) BCU(cudaEventCreate(&e), "event failed");
    auto done = [&](int code) {
        for (auto &e : ev) cudaEventDestroy(e);
        return code;
    };
    const Axes &ax = b->ax;
    const Workspace &w = b->w;
    const Tiling &t = b->tiling;
    cudaError_t e = cudaEventRecord(ev[0], s);
    if (!e) e = launch_stage(ax, w, s);
    if (!e) e = cudaEventRecord(ev[1], s);
    if (!e && t.vote_mode != HOUGH_VOTE_SCATTER) e = launch_gather(ax, w, t, s);
    if (!e) e = cudaEventRecord(ev[2], s);
    if (!e) e = launch_scatter(ax, w, t, b->refine_eps, t.vote_mode != HOUGH_VOTE_SCATTER, s);
    if (!e) e = cudaEventRecord(ev[3], s);
    if (!e) e = launch_band_peaks(ax, w, t, s);
    if (!e) e = cudaEventRecord(ev[4], s);
    if (!e) e = launch_compact(ax, w, s);
    if (!e) e = cudaEventRecord(ev[5], s);
    if (!e) e = launch_stage2(ax, w, b->sms, b->refine_eps, s);
    if (!e) e = cudaEventRecord(ev[6], s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return done(bfail(HOUGH_ECUDA, "profiled batch run failed"));
    note_launches(kStageLaunches + kVoteLaunches + peak_launches(n_events) + kStage2Launches);
    b->n_events = n_events;
    b->ran = true;
    float ms[6];
    for (int k = 0; k < 6; ++k)
        if (cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]) != cudaSuccess) return done(bfail(HOUGH_ECUDA, "event time failed"));
    std::memset(out, 0, sizeof(*out));
    out->stage_ms = ms[0];
    out->gather_ms = ms[1];
    out->scatter_ms = ms[2];
    out->vote_ms = ms[1] + ms[2];
    out->band_peaks_ms = ms[3];
    out->compact_ms = ms[4];
    out->peaks_ms = ms[3] + ms[4];
    out->stage2_ms = out->member_ms = ms[5];
    return done(HOUGH_OK);
}

int hough_batch_run(hough_batch *b, const float *r, const float *phi, const float *z, const uint8_t *layer,
                    const int64_t *hit_start, int32_t n_events, int where, void *stream)
{
    return batch_run(b, r, phi, z, layer, hit_start, n_events, where, static_cast<cudaStream_t>(stream), true);
}

int hough_batch_candidates(hough_batch *b, hough_candidate *out, int64_t cap, int64_t *offsets, int where, void *stream)
{
    if (!b || !offsets || cap < 0 || (cap > 0 && !out)) return bfail(HOUGH_EINVAL, "bad arguments");
    if (where != HOUGH_HOST && where != HOUGH_DEVICE) return bfail(HOUGH_EINVAL, "bad where");
    if (!b->ran) return bfail(HOUGH_ENOTREADY, "hough_batch_run has not run");
    BCU(cudaSetDevice(b->device), "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int E = b->n_events;
    std::vector<int32_t> base(E + 1);
    BCU(cudaMemcpyAsync(base.data(), b->w.cand_base, sizeof(int32_t) * (E + 1), cudaMemcpyDeviceToHost, s),
        "copy offsets failed");
    BCU(cudaStreamSynchronize(s), "synchronise failed");
    for (int e = 0; e <= E; ++e) offsets[e] = base[e];
    const int64_t total = base[E];
    const int64_t ncopy = std::min(total, cap);
    if (ncopy > 0) {
        hough_candidate *dst = where == HOUGH_DEVICE && ncopy == total ? out : b->packed;
        Workspace w = b->w;
        w.n_events = E;
        BCU(launch_pack_candidates(b->ax, w, dst, s), "pack kernel failed");
        note_launches(1);
        if (dst != out)
            BCU(cudaMemcpyAsync(out, b->packed, sizeof(hough_candidate) * ncopy,
                                where == HOUGH_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s),
                "copy candidates failed");
        BCU(cudaStreamSynchronize(s), "synchronise failed");
    }
    if (total > cap) return bfail(HOUGH_ETRUNC, "more candidates than the capacity");
    return HOUGH_OK;
}

int hough_batch_stats(hough_batch *b, int32_t event, hough_stats *out, void *stream)
{
    if (!b || !out) return bfail(HOUGH_EINVAL, "bad arguments");
    if (!b->ran) return bfail(HOUGH_ENOTREADY, "hough_batch_run has not run");
    if (event < 0 || event >= b->n_events) return bfail(HOUGH_EINVAL, "event out of range");
    BCU(cudaSetDevice(b->device), "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevStats d;
    LayerInfo info[HOUGH_MAX_LAYERS];
    BCU(cudaMemcpyAsync(&d, b->w.stats + event, sizeof(DevStats), cudaMemcpyDeviceToHost, s), "copy stats failed");
    BCU(cudaMemcpyAsync(info, b->w.info, sizeof(info), cudaMemcpyDeviceToHost, s), "copy layer info failed");
    BCU(cudaStreamSynchronize(s), "synchronise failed");
    fill_stats(d, info, b->ax.n_layers, out);
    if (d.device_error) return bfail(HOUGH_EDEVICE, "device-side check failed");
    return HOUGH_OK;
}

int hough_batch_accumulator(hough_batch *b, int32_t event, uint16_t *out, int where, void *stream)
{
    if (!b || !out) return bfail(HOUGH_EINVAL, "bad arguments");
    if (!b->ran) return bfail(HOUGH_ENOTREADY, "hough_batch_run has not run");
    if (event < 0 || event >= b->n_events) return bfail(HOUGH_EINVAL, "event out of range");
    if (where != HOUGH_HOST && where != HOUGH_DEVICE) return bfail(HOUGH_EINVAL, "bad where");
    if (b->w.fused) return bfail(HOUGH_ENOTREADY, "the fused vote and peak search does not keep the accumulator");
    BCU(cudaSetDevice(b->device), "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t cells = (size_t)b->ax.n_qpt * b->ax.n_phi;
    BCU(cudaMemcpyAsync(out, b->w.M + cells * event, sizeof(uint16_t) * cells,
                        where == HOUGH_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s),
        "copy accumulator failed");
    BCU(cudaStreamSynchronize(s), "synchronise failed");
    return HOUGH_OK;
}

}  // extern "C"
