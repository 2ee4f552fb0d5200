// C ABI of the hough library (declared in include/hough.h): argument checks, the context and its
// device buffers, and the order in which the kernels of the path are enqueued.
#include <algorithm>
#include <cstddef>
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "hough_internal.cuh"

using namespace hough;

namespace {

thread_local char g_err[512] = "";
std::atomic<uint64_t> g_launches{0};

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? HOUGH_ENOMEM : HOUGH_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CU(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

}  // namespace

int hough::set_last_error(int code, const char *msg) { return fail(code, "%s", msg); }



void hough::note_launches(uint64_t n) { g_launches += n; }

struct hough_ctx {
    int device = 0;
    int sms = 0;
    hough_geometry geometry{};
    hough_binning binning{};
    hough_limits limits{};
    Axes ax{};
    Tiling tiling{};
    float refine_eps = 0.f;
    // device buffers
    std::vector<void *> allocations;
    Workspace w{};
    int64_t *hit_start = nullptr;        // device, 2 entries, zero
    float *in_r = nullptr, *in_phi = nullptr, *in_z = nullptr;
    uint8_t *in_layer = nullptr;
    int32_t *mem_idx = nullptr;
    DevStats *stats_host = nullptr;      // pinned
    hough_candidate *cands_mapped = nullptr;       // pinned, mapped: hough_process's result staging
    hough_candidate *cands_mapped_dev = nullptr;   // its device address
    DevStats *stats_mapped = nullptr;              // pinned, mapped: hough_process's counters
    DevStats *stats_mapped_dev = nullptr;
    int64_t n_hits = 0;
    int stage = 0;                       // 0 nothing, 1 voted, 2 peaks, 3 stage 2
    // counters and radius ranges alternate between two buffers (Workspace::recycle); `clean`: the
    // last event's kernels left the rest of the state as the next event starts from
    DevStats *stats_buf[2] = {nullptr, nullptr};
    LayerRadii *radii_buf[2] = {nullptr, nullptr};
    int parity = 0;
    bool clean = true;
    // the peak search left the candidate list uncompacted (stage 2 reads the band lists itself);
    // a call that reads the list or the counters before stage 2 compacts it first
    bool list_pending = false;
    bool timing = false;
    // 0 before staging, 1 after staging, 2 after the gather, 3 after the vote, 4 after the band
    // peaks, 5 after the candidate scan, 6 after stage 2
    cudaEvent_t ev[12] = {};   // 0..7 step boundaries, 8..11 inside the staging
    int timed = 0;                       // bit k: ev[k] recorded for the current event
    bool cleared = false, compacted = false;   // the clearing / compaction kernel ran for this event

    ~hough_ctx()
    {
        cudaSetDevice(device);
        cudaDeviceSynchronize();
        for (void *p : allocations) cudaFree(p);
        if (stats_host) cudaFreeHost(stats_host);
        if (cands_mapped) cudaFreeHost(cands_mapped);
        if (stats_mapped) cudaFreeHost(stats_mapped);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }

    template <typename T>
    cudaError_t alloc(T **p, size_t count)
    {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess) allocations.push_back(q);
        *p = static_cast<T *>(q);
        return e;
    }
};

namespace {

int check_binning(const hough_geometry *g, const hough_binning *b)
{
    if (!g || !b) return fail(HOUGH_EINVAL, "geometry and binning are required");
    if (g->n_layers < 1 || g->n_layers > HOUGH_MAX_LAYERS) return fail(HOUGH_EINVAL, "n_layers must be 1..16");
    if (g->reserved != 0) return fail(HOUGH_EINVAL, "reserved fields must be 0");
    if (b->accumulator != HOUGH_ACC_LAYERS && b->accumulator != HOUGH_ACC_COUNTS)
        return fail(HOUGH_EINVAL, "accumulator must be HOUGH_ACC_LAYERS or HOUGH_ACC_COUNTS");
    if (!(g->b_tesla > 0.0) || !std::isfinite(g->b_tesla)) return fail(HOUGH_EINVAL, "b_tesla must be > 0");
    if (b->n_qpt < 1 || b->n_qpt > 65535) return fail(HOUGH_EINVAL, "n_qpt must be 1..65535");
    if (b->n_phi < 64 || b->n_phi > 32768 || b->n_phi % 64) return fail(HOUGH_EINVAL, "n_phi must be a multiple of 64 in 64..32768");
    if (b->accumulator == HOUGH_ACC_LAYERS && (b->threshold < 1 || b->threshold > 16))
        return fail(HOUGH_EINVAL, "threshold must be 1..16 layers");
    if (b->accumulator == HOUGH_ACC_COUNTS && (b->threshold < 1 || b->threshold > 65535))
        return fail(HOUGH_EINVAL, "threshold must be 1..65535 votes");
    if (b->n_cot < 1 || b->n_cot > 256 || b->n_z0 < 1 || b->n_z0 > 256 || b->n_cot * b->n_z0 > 16384)
        return fail(HOUGH_EINVAL, "n_cot and n_z0 must be 1..256 with n_cot * n_z0 <= 16384");
    if (!(b->qpt_min < b->qpt_max) || !(b->cot_min < b->cot_max) || !(b->z0_min_cm < b->z0_max_cm))
        return fail(HOUGH_EINVAL, "axis minimum must be below its maximum");
    if (!std::isfinite(b->qpt_min) || !std::isfinite(b->qpt_max) || !std::isfinite(b->cot_min) ||
        !std::isfinite(b->cot_max) || !std::isfinite(b->z0_min_cm) || !std::isfinite(b->z0_max_cm))
        return fail(HOUGH_EINVAL, "axis bounds must be finite");
    if (b->reserved != 0) return fail(HOUGH_EINVAL, "reserved fields must be 0");
    if (b->n_d0 < 0 || (int64_t)b->n_d0 * b->n_qpt > 65535)
        return fail(HOUGH_EINVAL, "n_d0 must be >= 0 with n_d0 * n_qpt <= 65535");
    if (b->n_d0 > 0 && (!(b->d0_min_cm < b->d0_max_cm) || !std::isfinite(b->d0_min_cm) || !std::isfinite(b->d0_max_cm)))
        return fail(HOUGH_EINVAL, "the d0 axis needs finite d0_min_cm < d0_max_cm");
    // the 3 x 3 x 3 peak search stages at least nine rows in shared memory (227 KB on this GPU family)
    if (b->n_d0 > 0 && (size_t)9 * b->n_phi * (b->accumulator == HOUGH_ACC_COUNTS ? 2 : 1) + 1024 > 232448)
        return fail(HOUGH_EINVAL, "n_phi too large for a d0 axis: nine rows of it must fit in shared memory");
    return HOUGH_OK;
}

Axes make_axes_impl(const hough_geometry *g, const hough_binning *b)
{
    Axes ax;
    ax.n_layers = g->n_layers;
    ax.q_rows = b->n_qpt;
    ax.n_d0 = b->n_d0 > 0 ? b->n_d0 : 0;
    ax.n_qpt = b->n_qpt * (ax.n_d0 ? ax.n_d0 : 1);   // rows of the stacked grid
    ax.d0_min = ax.n_d0 ? b->d0_min_cm : 0.0;
    ax.dd = ax.n_d0 ? (b->d0_max_cm - b->d0_min_cm) / b->n_d0 : 0.0;
    ax.n_phi = b->n_phi;
    ax.threshold = b->threshold;
    ax.counts = b->accumulator == HOUGH_ACC_COUNTS ? 1 : 0;
    ax.n_cot = b->n_cot;
    ax.n_z0 = b->n_z0;
    ax.b = g->b_tesla;
    ax.qpt_min = b->qpt_min;
    ax.qpt_max = b->qpt_max;
    ax.dk = (b->qpt_max - b->qpt_min) / b->n_qpt;
    ax.cot_min = b->cot_min;
    ax.cot_max = b->cot_max;
    ax.dt = (b->cot_max - b->cot_min) / b->n_cot;
    ax.z0_min = b->z0_min_cm;
    ax.z0_max = b->z0_max_cm;
    ax.zscale = (double)b->n_z0 / (b->z0_max_cm - b->z0_min_cm);
    ax.zs_hi = (float)ax.zscale;
    ax.zs_lo = (float)(ax.zscale - (double)ax.zs_hi);
    ax.zmin_hi = (float)ax.z0_min;
    ax.zmin_lo = (float)(ax.z0_min - (double)ax.zmin_hi);
    ax.pi_hi = (float)kPi;
    ax.pi_lo = (float)(kPi - (double)ax.pi_hi);
    const double upr = (double)b->n_phi / kTwoPi;
    ax.u_hi = (float)upr;
    ax.u_lo = (float)(upr - (double)ax.u_hi);
    return ax;
}

int default_gather_cols(const Axes &ax)
{
    int cols = std::min(ax.n_phi, 512);
    cols -= cols % 64;
    while (ax.n_phi % cols) cols -= 64;
    return cols;
}

// A public tiling with its gather defaults (zero fields) filled in.
Tiling resolve_tiling_impl(const Axes &ax, const hough_tiling *t)
{
    Tiling r{t->tile_qpt, t->tile_phi, t->threads, t->vote_mode, t->band_rows,
             t->gather_rows, t->gather_cols, t->gather_threads};
    if (!r.gather_rows) r.gather_rows = 4;
    if (!r.gather_cols) r.gather_cols = default_gather_cols(ax);
    if (!r.gather_threads) r.gather_threads = 256;
    return r;
}

int check_tiling_impl(const Axes &ax, int device, const hough_tiling *t)
{
    if (!t) return fail(HOUGH_EINVAL, "tiling is required");
    if (t->tile_qpt < 1 || t->tile_qpt > 256) return fail(HOUGH_EINVAL, "tile_qpt must be 1..256");
    if (t->tile_phi < 64 || t->tile_phi % 64 || ax.n_phi % t->tile_phi)
        return fail(HOUGH_EINVAL, "tile_phi must be a multiple of 64 dividing n_phi");
    if (t->threads != 128 && t->threads != 256 && t->threads != 512 && t->threads != 1024)
        return fail(HOUGH_EINVAL, "threads must be 128, 256, 512 or 1024");
    if (t->vote_mode != HOUGH_VOTE_GATHER && t->vote_mode != HOUGH_VOTE_SCATTER && t->vote_mode != HOUGH_VOTE_FUSED)
        return fail(HOUGH_EINVAL, "vote_mode must be HOUGH_VOTE_GATHER, HOUGH_VOTE_SCATTER or HOUGH_VOTE_FUSED");
    if (t->vote_mode == HOUGH_VOTE_FUSED && (ax.counts || ax.n_d0))
        return fail(HOUGH_EINVAL, "HOUGH_VOTE_FUSED needs the layer accumulator and no d0 axis");
    if (t->band_rows < 1 || t->band_rows > 16) return fail(HOUGH_EINVAL, "band_rows must be 1..16");
    if (t->gather_rows < 0 || t->gather_rows > 32) return fail(HOUGH_EINVAL, "gather_rows must be 0..32");
    if (t->gather_cols && (t->gather_cols < 64 || t->gather_cols % 64 || ax.n_phi % t->gather_cols))
        return fail(HOUGH_EINVAL, "gather_cols must be 0 or a multiple of 64 dividing n_phi");
    if (t->gather_threads && t->gather_threads != 256 && t->gather_threads != 512 && t->gather_threads != 1024)
        return fail(HOUGH_EINVAL, "gather_threads must be 0, 256, 512 or 1024");
    const Tiling tt = resolve_tiling_impl(ax, t);
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (vote_smem_bytes(ax, tt) + 1024 > (size_t)max_smem)
        return fail(HOUGH_EINVAL, "tile needs %zu bytes of shared memory, the device allows %d",
                    vote_smem_bytes(ax, tt), max_smem);
    if (band_smem_bytes(ax, t->band_rows) + 1024 > (size_t)max_smem)
        return fail(HOUGH_EINVAL, "band of %d rows needs %zu bytes of shared memory, the device allows %d",
                    t->band_rows, band_smem_bytes(ax, t->band_rows), max_smem);
    if (ax.counts && t->vote_mode == HOUGH_VOTE_GATHER) {
        if (gather_count_smem_bytes(ax, tt) + 1024 > (size_t)max_smem)
            return fail(HOUGH_EINVAL, "count gather tile needs %zu bytes of shared memory, the device allows %d",
                        gather_count_smem_bytes(ax, tt), max_smem);
    }
    if (gather_smem_bytes(ax, tt) + 1024 > (size_t)max_smem)
        return fail(HOUGH_EINVAL, "gather tile needs %zu bytes of shared memory, the device allows %d",
                    gather_smem_bytes(ax, tt), max_smem);
    // the fused kernel's band of masks, plus its row tables (5 KB) in static shared memory
    if (t->vote_mode == HOUGH_VOTE_FUSED && fused_smem_bytes(ax, t->band_rows) + 6144 + 1024 > (size_t)max_smem)
        return fail(HOUGH_EINVAL, "fused band of %d rows needs %zu bytes of shared memory, the device allows %d",
                    t->band_rows, fused_smem_bytes(ax, t->band_rows), max_smem);
    return HOUGH_OK;
}

Tiling default_tiling_impl(const Axes &ax)
{
    Tiling t;
    t.tile_phi = std::min(ax.n_phi, 256);
    while (ax.n_phi % t.tile_phi) t.tile_phi -= 64;
    t.tile_qpt = std::min(ax.n_qpt, 32);   // the scatter kernel's lanes take 32 rows
    t.threads = 256;                       // the autotuner tries 512 and 1024 for the scatter vote (a
                                           // per-vote detector runs it 2x faster at 1024; an empty
                                           // launch over a batch's tiles costs 3x more at 1024)
    t.vote_mode = HOUGH_VOTE_GATHER;
    t.band_rows = 1;
    // with a d0 axis a band stages its rows in three slices: taller bands stage each row fewer times
    if (ax.n_d0)
        for (int r : {4, 2})
            if (band_smem_bytes(ax, r) + 1024 <= 232448) {
                t.band_rows = r;
                break;
            }
    t.gather_rows = 4;
    t.gather_cols = default_gather_cols(ax);
    t.gather_threads = 256;
    return t;
}

// Largest band-list storage over every allowed band height.
size_t band_list_entries_impl(const Axes &ax)
{
    size_t best = 0;
    for (int r = 1; r <= 16; ++r)
        best = std::max(best, (size_t)n_bands(ax, r) * (size_t)band_capacity(ax, r));
    return best;
}

// Hits are checked a block at a time without branches (the compiler vectorises the pass); only a
// block with a bad hit is scanned again hit by hit, to name the first one.
int check_host_hits_impl(const Axes &ax, const float *r, const float *phi, const float *z,
                         const uint8_t *layer, int64_t n)
{
    constexpr int64_t kBlock = 4096;
    const unsigned L = (unsigned)ax.n_layers;
    int64_t first_bad_block = -1;
    for (int64_t b0 = 0; b0 < n && first_bad_block < 0; b0 += kBlock) {
        const int64_t b1 = std::min(n, b0 + kBlock);
        unsigned bad = 0;
        for (int64_t h = b0; h < b1; ++h) {
            const float rr = r[h], pp = phi[h], zz = z[h];
            bad |= (unsigned)(layer[h] >= L) | (unsigned)!(rr > 0.f) | (unsigned)!(rr <= FLT_MAX) |
                   (unsigned)!(std::fabs(pp) <= 1000.f) | (unsigned)!(std::fabs(zz) <= FLT_MAX);
        }
        if (bad) first_bad_block = b0;
    }
    if (first_bad_block < 0) return HOUGH_OK;
    for (int64_t h = first_bad_block; h < n; ++h) {
        if (layer[h] >= ax.n_layers) return fail(HOUGH_EINVAL, "hit %lld: layer %d >= n_layers", (long long)h, layer[h]);
        if (!(r[h] > 0.f) || !std::isfinite(r[h])) return fail(HOUGH_EINVAL, "hit %lld: r must be finite and > 0", (long long)h);
        if (!(std::fabs(phi[h]) <= 1000.f)) return fail(HOUGH_EINVAL, "hit %lld: phi must be finite, |phi| <= 1000", (long long)h);
        if (!std::isfinite(z[h])) return fail(HOUGH_EINVAL, "hit %lld: z must be finite", (long long)h);
    }
    return HOUGH_OK;
}

// The device address of pinned host memory (cudaHostAlloc, cudaHostRegister) under unified
// addressing; false for other memory.
bool device_view(const void *p, const void **dp)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // not a pointer the runtime knows: plain host memory
        return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    *dp = a.devicePointer;
    return true;
}

// host_check: check host hits on the host before anything runs (else the staging kernel applies
// the same predicates on the device and drops a bad hit, reporting it in device_error).
int enqueue_vote(hough_ctx *c, const float *r, const float *phi, const float *z, const uint8_t *layer,
                 int64_t n, int where, cudaStream_t s, bool host_check = true)
{
    if (n < 0) return fail(HOUGH_EINVAL, "n_hits must be >= 0");
    if (n > c->limits.max_hits) return fail(HOUGH_ECAPACITY, "n_hits %lld exceeds max_hits %lld", (long long)n, (long long)c->limits.max_hits);
    if (where != HOUGH_HOST && where != HOUGH_DEVICE) return fail(HOUGH_EINVAL, "where must be HOUGH_HOST or HOUGH_DEVICE");
    if (n > 0 && (!r || !phi || !z || !layer)) return fail(HOUGH_EINVAL, "hit arrays are required");
    if (where == HOUGH_HOST) {
        // pinned hits are read in place by the staging kernels, over the host link; other host
        // memory is copied into the context's own input buffers, the copies running while the
        // host checks the hits (a bad hit returns before anything reads them)
        const void *dv[4] = {nullptr, nullptr, nullptr, nullptr};
        const bool in_place = n > 0 && device_view(r, &dv[0]) && device_view(phi, &dv[1]) &&
                              device_view(z, &dv[2]) && device_view(layer, &dv[3]);
        if (n > 0 && !in_place) {
            CU(cudaMemcpyAsync(c->in_r, r, sizeof(float) * n, cudaMemcpyHostToDevice, s), "copy r");
            CU(cudaMemcpyAsync(c->in_phi, phi, sizeof(float) * n, cudaMemcpyHostToDevice, s), "copy phi");
            CU(cudaMemcpyAsync(c->in_z, z, sizeof(float) * n, cudaMemcpyHostToDevice, s), "copy z");
            CU(cudaMemcpyAsync(c->in_layer, layer, n, cudaMemcpyHostToDevice, s), "copy layer");
        }
        if (host_check) {
            int rc = check_host_hits_impl(c->ax, r, phi, z, layer, n);
            if (rc) return rc;
        }
        if (in_place) {
            c->w.r = static_cast<const float *>(dv[0]);
            c->w.phi = static_cast<const float *>(dv[1]);
            c->w.z = static_cast<const float *>(dv[2]);
            c->w.layer = static_cast<const uint8_t *>(dv[3]);
        } else {
            c->w.r = c->in_r; c->w.phi = c->in_phi; c->w.z = c->in_z; c->w.layer = c->in_layer;
        }
    } else {
        c->w.r = r; c->w.phi = phi; c->w.z = z; c->w.layer = layer;
    }
    // one event: its hits start at 0 (hit_start holds {0, 0} from creation; the kernels read
    // only the start of an event and take the total by value)
    c->w.n_hits_total = n;
    c->n_hits = n;
    c->timed = 0;
    c->w.band_rows = c->tiling.band_rows;
    c->w.band_cap = band_capacity(c->ax, c->tiling.band_rows);
    c->w.fused = c->tiling.vote_mode == HOUGH_VOTE_FUSED;
    if (c->timing) { CU(cudaEventRecord(c->ev[0], s), "event"); c->timed |= 1 | (0xF << 8); }
    // this event's counters and radius ranges; the other buffer of each is zeroed for the next one
    c->w.stats = c->stats_buf[c->parity];
    c->w.radii = c->radii_buf[c->parity];
    c->w.stats_next = c->stats_buf[c->parity ^ 1];
    c->w.radii_next = c->radii_buf[c->parity ^ 1];
    const bool clear = !c->clean;   // the last event did not run its peak search: clear the state
    CU(launch_stage(c->ax, c->w, s, c->timing ? c->ev + 8 : nullptr, clear), "stage kernels");
    c->cleared = clear;
    c->compacted = false;
    c->parity ^= 1;
    c->clean = false;
    c->list_pending = false;
    if (c->timing) { CU(cudaEventRecord(c->ev[1], s), "event"); c->timed |= 2; }
    if (c->tiling.vote_mode != HOUGH_VOTE_SCATTER) CU(launch_gather(c->ax, c->w, c->tiling, s), "gather kernel");
    if (c->timing) { CU(cudaEventRecord(c->ev[2], s), "event"); c->timed |= 4; }
    CU(launch_scatter(c->ax, c->w, c->tiling, c->refine_eps, c->tiling.vote_mode != HOUGH_VOTE_SCATTER, s), "vote kernel");
    if (c->timing) { CU(cudaEventRecord(c->ev[3], s), "event"); c->timed |= 8; }
    g_launches += kStageLaunches - (clear ? 0 : 1) + (c->tiling.vote_mode == HOUGH_VOTE_SCATTER ? 1 : kVoteLaunches);
    c->stage = 1;
    return HOUGH_OK;
}

// The compaction a peak search left to stage 2, run now for a caller that reads the list first.
int settle_list(hough_ctx *c, cudaStream_t s)
{
    if (!c->list_pending) return HOUGH_OK;
    CU(launch_compact(c->ax, c->w, s), "candidate scan kernel");
    g_launches += peak_launches(1) - 1;
    c->list_pending = false;
    return HOUGH_OK;
}

// The member pool's reservations exceed max_members exactly when some candidate's list was cut:
// reported with the device's bits (the kernels count the reservations, the host compares).
void note_member_cut(hough_ctx *c)
{
    if (c->stats_host->pool_used > (unsigned)c->w.max_members) c->stats_host->device_error |= HOUGH_DEVERR_MEMBERS;
}

int read_stats(hough_ctx *c, cudaStream_t s)
{
    int rc = settle_list(c, s);
    if (rc) return rc;
    CU(cudaMemcpyAsync(c->stats_host, c->w.stats, sizeof(DevStats), cudaMemcpyDeviceToHost, s), "copy stats");
    CU(cudaStreamSynchronize(s), "synchronise");
    note_member_cut(c);
    return HOUGH_OK;
}

}  // namespace

Axes hough::make_axes(const hough_geometry *g, const hough_binning *b) { return make_axes_impl(g, b); }
int hough::check_geometry_binning(const hough_geometry *g, const hough_binning *b) { return check_binning(g, b); }
int hough::check_tiling_for(const Axes &ax, int device, const hough_tiling *t) { return check_tiling_impl(ax, device, t); }
Tiling hough::resolve_tiling(const Axes &ax, const hough_tiling *t) { return resolve_tiling_impl(ax, t); }
void hough::public_tiling(const Tiling &t, hough_tiling *out)
{
    *out = hough_tiling{t.tile_qpt, t.tile_phi, t.threads, t.vote_mode, t.band_rows,
                        t.gather_rows, t.gather_cols, t.gather_threads};
}
Tiling hough::default_tiling_for(const Axes &ax) { return default_tiling_impl(ax); }
size_t hough::band_list_entries(const Axes &ax) { return band_list_entries_impl(ax); }
int hough::check_host_hits_for(const Axes &ax, const float *r, const float *phi, const float *z, const uint8_t *layer,
                               int64_t n)
{
    return check_host_hits_impl(ax, r, phi, z, layer, n);
}

void hough::fill_stats(const DevStats &d, const LayerInfo *info, int n_layers, hough_stats *out)
{
    std::memset(out, 0, sizeof(*out));
    for (int l = 0; l < HOUGH_MAX_LAYERS; ++l) {
        out->votes_by_layer[l] = d.votes_by_layer[l];
        out->votes += d.votes_by_layer[l];
        if (l < n_layers && info[l].present && info[l].uniform) out->uniform_layers |= 1u << l;
        else if (l < n_layers) out->general_votes += d.votes_by_layer[l];
    }
    out->refined_votes = d.refined_votes;
    out->stage2_votes = d.stage2_votes;
    out->n_hits = (int64_t)d.n_hits;
    out->n_candidates = d.n_candidates;
    out->n_members = d.n_members;
    out->device_error = d.device_error;
}

extern "C" {

const char *hough_last_error(void) { return g_err; }

const char *hough_version(void) { return "0.1.0"; }

int hough_create(const hough_geometry *geometry, const hough_binning *binning, const hough_limits *limits,
                 int device, hough_ctx **out)
{
    if (!out) return fail(HOUGH_EINVAL, "out is required");
    *out = nullptr;
    int rc = check_binning(geometry, binning);
    if (rc) return rc;
    if (!limits || limits->max_hits < 1 || limits->max_hits > (1LL << 30) || limits->max_candidates < 1 ||
        limits->max_members < 1)
        return fail(HOUGH_EINVAL, "limits: max_hits in 1..2^30, max_candidates >= 1, max_members >= 1");
    int ndev = 0;
    CU(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(HOUGH_EINVAL, "device %d out of range (%d devices)", device, ndev);
    CU(cudaSetDevice(device), "cudaSetDevice");
    hough_ctx *c = new (std::nothrow) hough_ctx();
    if (!c) return fail(HOUGH_ENOMEM, "host allocation");
    c->device = device;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    c->geometry = *geometry;
    c->binning = *binning;
    c->limits = *limits;
    c->ax = make_axes_impl(geometry, binning);
    c->tiling = default_tiling_impl(c->ax);
    c->refine_eps = refine_eps_for(c->ax);
    const Axes &ax = c->ax;
    const int64_t n = limits->max_hits;
    const int nkeys = n_keys(ax);
    Workspace &w = c->w;
    w.n_events = 1;
    w.max_cand = limits->max_candidates;
    w.max_members = limits->max_members;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(c->alloc(&c->hit_start, 2));
    A(c->alloc(&c->in_r, n)); A(c->alloc(&c->in_phi, n)); A(c->alloc(&c->in_z, n)); A(c->alloc(&c->in_layer, n));
    A(c->alloc(&w.key, n)); A(c->alloc(&w.rank, n)); A(c->alloc(&w.hot_tmp, n));
    A(c->alloc(&w.counts, nkeys)); A(c->alloc(&w.offs, nkeys + 1)); A(c->alloc(&w.prof, (size_t)prof_event_entries(ax)));
    A(c->alloc(&w.hot, n)); A(c->alloc(&w.cold, n)); A(c->alloc(&w.fsort, n)); A(c->alloc(&w.zsort, n));
    A(c->alloc(&c->radii_buf[0], 1)); A(c->alloc(&c->radii_buf[1], 1));
    A(c->alloc(&w.info, HOUGH_MAX_LAYERS)); A(c->alloc(&w.memo, 1));
    A(c->alloc(&w.tab, (size_t)ax.n_layers * ax.n_qpt)); A(c->alloc(&w.arc, (size_t)ax.n_layers * ax.n_qpt));
    A(c->alloc(&w.zco, (size_t)ax.n_layers * ax.n_qpt));
    A(c->alloc(&w.kq32, ax.n_qpt));
    A(c->alloc(&w.M, (size_t)ax.n_qpt * ax.n_phi));
    A(c->alloc(&w.cands, w.max_cand));
    A(c->alloc(&w.band_cands, band_list_entries_impl(ax)));
    A(c->alloc(&w.band_counts, n_bands(ax, 1))); A(c->alloc(&w.band_offs, n_bands(ax, 1)));
    A(c->alloc(&w.mem_start, w.max_cand)); A(c->alloc(&w.mem_count, w.max_cand));
    A(c->alloc(&w.cand_base, 2)); A(c->alloc(&w.counters, 1));
    A(c->alloc(&w.mem_pool, w.max_members)); A(c->alloc(&c->mem_idx, w.max_members));
    A(c->alloc(&c->stats_buf[0], 1)); A(c->alloc(&c->stats_buf[1], 1));
    A(cudaMallocHost(&c->stats_host, sizeof(DevStats)));
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "hough_create allocation");
    }
    w.hit_start = c->hit_start;
    w.hit_capacity = n;
    w.inputs = nullptr;
    w.band_rows = c->tiling.band_rows;
    w.band_cap = band_capacity(ax, c->tiling.band_rows);
    w.fused = 0;
    w.keep_members = 1;   // hough_get_members reads the member lists
    w.recycle = 1;
    w.compact_in_peaks = 1;
    w.stats = c->stats_buf[0];
    w.radii = c->radii_buf[0];
    // FP32 q/pT bin centres: the FP64 centre rounded once
    std::vector<float> kq(ax.n_qpt);
    for (int i = 0; i < ax.n_qpt; ++i) kq[i] = (float)(ax.qpt_min + (i % ax.q_rows + 0.5) * ax.dk);
    A(cudaMemcpy(w.kq32, kq.data(), sizeof(float) * ax.n_qpt, cudaMemcpyHostToDevice));
    A(cudaMemset(c->hit_start, 0, 2 * sizeof(int64_t)));
    A(cudaMemset(w.memo, 0, sizeof(TableMemo)));
    // the state every event starts from (Workspace::recycle keeps it so from then on)
    for (int q = 0; q < 2; ++q) {
        A(cudaMemset(c->stats_buf[q], 0, sizeof(DevStats)));
        char *rb = reinterpret_cast<char *>(c->radii_buf[q]);
        A(cudaMemset(rb + offsetof(LayerRadii, rmin), 0xFF, sizeof(LayerRadii::rmin)));
        A(cudaMemset(rb + offsetof(LayerRadii, rmax), 0, sizeof(LayerRadii::rmax)));
    }
    A(cudaMemset(w.counts, 0, sizeof(int32_t) * nkeys));
    A(cudaMemset(w.prof, 0, sizeof(uint2) * (size_t)prof_event_entries(ax)));
    A(cudaMemset(w.counters, 0, sizeof(BatchCounters)));
    A(cudaDeviceSynchronize());
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "hough_create initialisation");
    }
    *out = c;
    return HOUGH_OK;
}

void hough_destroy(hough_ctx *ctx) { delete ctx; }

int hough_vote(hough_ctx *c, const float *r, const float *phi, const float *z, const uint8_t *layer,
               int64_t n_hits, int where, void *stream)
{
    if (!c) return fail(HOUGH_EINVAL, "ctx is required");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    return enqueue_vote(c, r, phi, z, layer, n_hits, where, (cudaStream_t)stream);
}

int hough_peaks(hough_ctx *c, void *stream)
{
    if (!c) return fail(HOUGH_EINVAL, "ctx is required");
    if (c->stage < 1) return fail(HOUGH_ENOTREADY, "hough_vote has not run");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    // The candidate list: stage 2 reads the band lists itself when their offsets fit its shared
    // memory (the list is compacted later only for a caller that reads it first); else the peak
    // kernel's last CTA compacts it, except after the fused vote (whose peak kernel may not run).
    // Either way the peak kernel zeroes the bucket profile for the next event.
    const bool fused = c->tiling.vote_mode == HOUGH_VOTE_FUSED;
    const bool deferred = !fused && stage2_reads_bands(c->ax, c->tiling.band_rows);
    c->w.compact_in_peaks = fused || deferred ? 0 : 1;
    CU(launch_band_peaks(c->ax, c->w, c->tiling, (cudaStream_t)stream), "peak kernel");
    c->compacted = fused;   // a separate compaction kernel (the peak kernel's own last CTA is timed with it)
    if (c->timing) { CU(cudaEventRecord(c->ev[4], (cudaStream_t)stream), "event"); c->timed |= 16; }
    if (fused) CU(launch_compact(c->ax, c->w, (cudaStream_t)stream), "candidate scan kernel");
    if (c->timing) { CU(cudaEventRecord(c->ev[5], (cudaStream_t)stream), "event"); c->timed |= 32; }
    g_launches += fused ? peak_launches(1) : 1;
    c->list_pending = deferred;
    c->clean = true;
    c->stage = 2;
    return HOUGH_OK;
}

int hough_stage2(hough_ctx *c, void *stream)
{
    if (!c) return fail(HOUGH_EINVAL, "ctx is required");
    if (c->stage < 2) return fail(HOUGH_ENOTREADY, "hough_peaks has not run");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    c->w.cands_from_bands = c->list_pending ? 1 : 0;   // the confirmation compacts as it goes
    CU(launch_stage2(c->ax, c->w, c->sms, c->refine_eps, (cudaStream_t)stream, c->timing ? c->ev[7] : nullptr),
       "stage-2 kernels");
    c->w.cands_from_bands = 0;
    c->list_pending = false;
    if (c->timing) { CU(cudaEventRecord(c->ev[6], (cudaStream_t)stream), "event"); c->timed |= 64 | 128; }
    g_launches += kStage2Launches;
    c->stage = 3;
    return HOUGH_OK;
}

int hough_get_candidates(hough_ctx *c, hough_candidate *out, int32_t cap, int32_t *n_out, int where, void *stream)
{
    if (!c || !n_out || cap < 0 || (cap > 0 && !out)) return fail(HOUGH_EINVAL, "bad arguments");
    if (where != HOUGH_HOST && where != HOUGH_DEVICE) return fail(HOUGH_EINVAL, "bad where");
    if (c->stage < 2) return fail(HOUGH_ENOTREADY, "hough_peaks has not run");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = read_stats(c, s);
    if (rc) return rc;
    const int64_t found = c->stats_host->n_candidates;
    const int64_t kept = std::min<int64_t>(found, c->w.max_cand);
    const int64_t ncopy = std::min<int64_t>(kept, cap);
    *n_out = (int32_t)std::min<int64_t>(found, INT32_MAX);
    if (ncopy > 0) {
        CU(cudaMemcpyAsync(out, c->w.cands, sizeof(hough_candidate) * ncopy,
                           where == HOUGH_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s),
           "copy candidates");
        CU(cudaStreamSynchronize(s), "synchronise");
    }
    if (found > cap) return fail(HOUGH_ETRUNC, "%lld candidates, capacity %d", (long long)found, cap);
    if (found > kept) return fail(HOUGH_ETRUNC, "%lld candidates, max_candidates %d", (long long)found, c->w.max_cand);
    return HOUGH_OK;
}

int hough_get_accumulator(hough_ctx *c, uint16_t *out, int where, void *stream)
{
    if (!c || !out) return fail(HOUGH_EINVAL, "bad arguments");
    if (where != HOUGH_HOST && where != HOUGH_DEVICE) return fail(HOUGH_EINVAL, "bad where");
    if (c->stage < 1) return fail(HOUGH_ENOTREADY, "hough_vote has not run");
    if (c->w.fused) return fail(HOUGH_ENOTREADY, "the fused vote and peak search does not keep the accumulator");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaMemcpyAsync(out, c->w.M, sizeof(uint16_t) * (size_t)c->ax.n_qpt * c->ax.n_phi,
                       where == HOUGH_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s),
       "copy accumulator");
    CU(cudaStreamSynchronize(s), "synchronise");
    return HOUGH_OK;
}

int hough_get_members(hough_ctx *c, int64_t *offsets, int32_t *hits, int64_t hit_cap, int where, void *stream)
{
    if (!c || !offsets || hit_cap < 0 || (hit_cap > 0 && !hits)) return fail(HOUGH_EINVAL, "bad arguments");
    if (where != HOUGH_HOST) return fail(HOUGH_EINVAL, "member lists are returned to host memory only");
    if (c->stage < 3) return fail(HOUGH_ENOTREADY, "hough_stage2 has not run");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = read_stats(c, s);
    if (rc) return rc;
    const int64_t ncand = std::min<int64_t>(c->stats_host->n_candidates, c->w.max_cand);
    const int64_t pooled = std::min<int64_t>(c->stats_host->pool_used, c->w.max_members);
    std::vector<int32_t> start(ncand), count(ncand), pool(pooled);
    if (ncand > 0) {
        CU(cudaMemcpyAsync(start.data(), c->w.mem_start, sizeof(int32_t) * ncand, cudaMemcpyDeviceToHost, s), "copy member starts");
        CU(cudaMemcpyAsync(count.data(), c->w.mem_count, sizeof(int32_t) * ncand, cudaMemcpyDeviceToHost, s), "copy member counts");
    }
    CU(launch_member_index(c->w, c->mem_idx, pooled, s), "member index kernel");
    if (pooled > 0) CU(cudaMemcpyAsync(pool.data(), c->mem_idx, sizeof(int32_t) * pooled, cudaMemcpyDeviceToHost, s), "copy members");
    CU(cudaStreamSynchronize(s), "synchronise");
    // lists in candidate order, each sorted by hit index
    offsets[0] = 0;
    bool cut = c->stats_host->pool_used > (unsigned)c->w.max_members;
    for (int64_t q = 0; q < ncand; ++q) {
        const int64_t a = offsets[q];
        int64_t n = count[q];
        if (a + n > hit_cap) { n = std::max<int64_t>(0, hit_cap - a); cut = true; }
        if (n > 0) {
            std::copy(pool.begin() + start[q], pool.begin() + start[q] + n, hits + a);
            std::sort(hits + a, hits + a + n);
        }
        offsets[q + 1] = a + n;
    }
    if (cut) return fail(HOUGH_ETRUNC, "member lists were cut (max_members %d, capacity %lld)", c->w.max_members, (long long)hit_cap);
    return HOUGH_OK;
}

int hough_get_stats(hough_ctx *c, hough_stats *out, void *stream)
{
    if (!c || !out) return fail(HOUGH_EINVAL, "bad arguments");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = read_stats(c, s);
    if (rc) return rc;
    LayerInfo info[HOUGH_MAX_LAYERS];
    CU(cudaMemcpy(info, c->w.info, sizeof(info), cudaMemcpyDeviceToHost), "copy layer info");
    const DevStats &d = *c->stats_host;
    fill_stats(d, info, c->ax.n_layers, out);
    if (d.device_error) return fail(HOUGH_EDEVICE, "device-side check failed: bits 0x%x", d.device_error);
    return HOUGH_OK;
}

// With host memory the path has one round trip: the hits' per-hit checks run in the staging kernel
// (the predicates of the host check; a rejected hit makes the call fail with HOUGH_EINVAL once it
// has synchronised), and the candidates are packed into mapped pinned memory beside the counters'
// copy, so one synchronisation delivers both.
int hough_process(hough_ctx *c, const float *r, const float *phi, const float *z, const uint8_t *layer,
                  int64_t n_hits, hough_candidate *out, int32_t cap, int32_t *n_out, int where, void *stream)
{
    if (where != HOUGH_HOST) {
        int rc = hough_vote(c, r, phi, z, layer, n_hits, where, stream);
        if (rc) return rc;
        if ((rc = hough_peaks(c, stream))) return rc;
        if ((rc = hough_stage2(c, stream))) return rc;
        return hough_get_candidates(c, out, cap, n_out, where, stream);
    }
    if (!c || !n_out || cap < 0 || (cap > 0 && !out)) return fail(HOUGH_EINVAL, "bad arguments");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->cands_mapped) {   // the first call allocates the staging, once
        void *h = nullptr, *d = nullptr;
        CU(cudaHostAlloc(&h, sizeof(hough_candidate) * std::max(c->w.max_cand, 1), cudaHostAllocMapped),
           "cudaHostAlloc of the result staging");
        c->cands_mapped = static_cast<hough_candidate *>(h);
        CU(cudaHostGetDevicePointer(&d, h, 0), "cudaHostGetDevicePointer");
        c->cands_mapped_dev = static_cast<hough_candidate *>(d);
        CU(cudaHostAlloc(&h, sizeof(DevStats), cudaHostAllocMapped), "cudaHostAlloc of the counters");
        c->stats_mapped = static_cast<DevStats *>(h);
        CU(cudaHostGetDevicePointer(&d, h, 0), "cudaHostGetDevicePointer");
        c->stats_mapped_dev = static_cast<DevStats *>(d);
    }
    int rc = enqueue_vote(c, r, phi, z, layer, n_hits, HOUGH_HOST, s, false);
    if (rc) return rc;
    if ((rc = hough_peaks(c, stream))) return rc;
    if ((rc = hough_stage2(c, stream))) return rc;
    // one kernel writes both the candidates and the counters into mapped memory
    CU(launch_pack_candidates(c->ax, c->w, c->cands_mapped_dev, s, std::min<long long>(cap, c->w.max_cand), nullptr,
                              c->stats_mapped_dev, 152),
       "pack kernel");
    g_launches += 1;
    CU(cudaStreamSynchronize(s), "synchronise");
    *c->stats_host = *c->stats_mapped;   // hough_get_stats and friends read the last event's copy
    note_member_cut(c);
    const DevStats &d = *c->stats_host;
    if (d.device_error & (HOUGH_DEVERR_LAYER | HOUGH_DEVERR_RADIUS))
        return fail(HOUGH_EINVAL, "a hit had layer >= n_layers, r <= 0, |phi| > 1000 or a non-finite coordinate");
    const int64_t found = d.n_candidates;
    const int64_t kept = std::min<int64_t>(found, c->w.max_cand);
    const int64_t ncopy = std::min<int64_t>(kept, cap);
    *n_out = (int32_t)std::min<int64_t>(found, INT32_MAX);
    if (ncopy > 0) std::memcpy(out, c->cands_mapped, sizeof(hough_candidate) * ncopy);
    if (found > cap) return fail(HOUGH_ETRUNC, "%lld candidates, capacity %d", (long long)found, cap);
    if (found > kept) return fail(HOUGH_ETRUNC, "%lld candidates, max_candidates %d", (long long)found, c->w.max_cand);
    return HOUGH_OK;
}

int hough_set_tiling(hough_ctx *c, const hough_tiling *t)
{
    if (!c) return fail(HOUGH_EINVAL, "ctx is required");
    int rc = check_tiling_impl(c->ax, c->device, t);
    if (rc) return rc;
    c->tiling = resolve_tiling(c->ax, t);
    return HOUGH_OK;
}

int hough_set_copy_wait(hough_ctx *c, int first_bound)
{
    if (!c) return fail(HOUGH_EINVAL, "ctx is required");
    c->w.copy_wait = first_bound < 0 ? -1 : 0;
    return HOUGH_OK;
}

int hough_enable_timing(hough_ctx *c, int on)
{
    if (!c) return fail(HOUGH_EINVAL, "ctx is required");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    if (on && !c->ev[0])
        for (cudaEvent_t &e : c->ev) CU(cudaEventCreate(&e), "cudaEventCreate");
    c->timing = on != 0;
    c->timed = 0;
    return HOUGH_OK;
}

int hough_get_timing(hough_ctx *c, hough_timing *out)
{
    if (!c || !out) return fail(HOUGH_EINVAL, "bad arguments");
    if ((c->timed & 15) != 15) return fail(HOUGH_ENOTREADY, "no timed event");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    auto span = [&](int a, int b, float *ms) -> int {
        *ms = 0.f;
        if (((c->timed >> a) & 1) && ((c->timed >> b) & 1)) {
            CU(cudaEventSynchronize(c->ev[b]), "event synchronise");
            CU(cudaEventElapsedTime(ms, c->ev[a], c->ev[b]), "event elapsed");
        }
        return HOUGH_OK;
    };
    int rc;
    if ((rc = span(0, 1, &out->stage_ms)) || (rc = span(1, 3, &out->vote_ms)) || (rc = span(1, 2, &out->gather_ms)) ||
        (rc = span(2, 3, &out->scatter_ms)) || (rc = span(3, 5, &out->peaks_ms)) ||
        (rc = span(3, 4, &out->band_peaks_ms)) || (rc = span(4, 5, &out->compact_ms)) ||
        (rc = span(5, 6, &out->stage2_ms)) || (rc = span(5, 7, &out->member_ms)) || (rc = span(7, 6, &out->large_ms)) ||
        (rc = span(0, 8, &out->clear_ms)) || (rc = span(8, 9, &out->count_ms)) || (rc = span(9, 10, &out->table_ms)) ||
        (rc = span(10, 11, &out->scan_ms)) || (rc = span(11, 1, &out->sort_ms)))
        return rc;
    // a kernel that did not run for this event has no time of its own (its span is only the gap
    // between two event records)
    if (!c->cleared) out->clear_ms = 0.f;
    if (!c->compacted) out->compact_ms = 0.f;
    return HOUGH_OK;
}

uint64_t hough_kernel_launches(void) { return g_launches.load(); }

int hough_microbench_smem_or(int device, int pattern, double ms, double *atomics_per_s)
{
    if (!atomics_per_s || (pattern != 0 && pattern != 1) || !(ms > 0.0) || ms > 10000.0)
        return fail(HOUGH_EINVAL, "bad arguments");
    uint64_t n = 0;
    cudaError_t e = run_smem_or_bench(device, pattern, ms, atomics_per_s, &n);
    g_launches += n;
    if (e) return cuda_fail(e, "shared-atomic microbenchmark");
    return HOUGH_OK;
}

int hough_get_tiling(const hough_ctx *c, hough_tiling *t)
{
    if (!c || !t) return fail(HOUGH_EINVAL, "bad arguments");
    public_tiling(c->tiling, t);
    return HOUGH_OK;
}

}  // extern "C"
