// hough_vote_static: the stage-1 vote of one event without any allocation.
//
// Some callers cannot allocate device memory once they are running.  A trigger farm's event loop
// is the typical case: cudaMalloc and cudaFree can synchronise the whole device and take an
// unbounded time, so real-time code reserves all its memory at start-up and forbids allocation
// afterwards.  Frameworks that hand all device memory to their own pool are in the same position.
// Such callers cannot create a hough_ctx (hough_create allocates every buffer it needs).  This entry
// point runs the same staging and vote kernels as hough_vote, but keeps their scratch in one
// fixed, file-scope device array; the caller passes only its inputs and the output accumulator.
// The array is reserved on a device when the library's device code is loaded there: with the CUDA
// runtime's lazy loading (its default) that is the first call on that device, which therefore
// belongs to the caller's start-up, outside its real-time loop and before any stream capture.
//
// Limits of the fixed array (8 MiB per GPU that loads the library, held until the process exits):
// at most kStaticMaxHits hits, n_qpt <= kStaticMaxQpt, n_phi <= kStaticMaxPhi, 16 layers.
#include <mutex>

#include "hough_internal.cuh"

namespace hough {

namespace {

constexpr int64_t kStaticMaxHits = 1 << 17;   // 131,072 hits
constexpr int kStaticMaxQpt = 1024;
constexpr int kStaticMaxPhi = 4096;
constexpr int kStaticMaxKeys = HOUGH_MAX_LAYERS * kStaticMaxPhi;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte offsets of each scratch buffer inside the array.
constexpr size_t kOffHitStart = 0;
constexpr size_t kOffStats = align256(kOffHitStart + 2 * sizeof(int64_t));
constexpr size_t kOffRadii = align256(kOffStats + sizeof(DevStats));
constexpr size_t kOffInfo = align256(kOffRadii + sizeof(LayerRadii));
constexpr size_t kOffMemo = align256(kOffInfo + HOUGH_MAX_LAYERS * sizeof(LayerInfo));
constexpr size_t kOffKq = align256(kOffMemo + sizeof(TableMemo));
constexpr size_t kOffTab = align256(kOffKq + kStaticMaxQpt * sizeof(float));
constexpr size_t kOffArc = align256(kOffTab + (size_t)HOUGH_MAX_LAYERS * kStaticMaxQpt * sizeof(TabEntry));
constexpr size_t kOffCounts = align256(kOffArc + (size_t)HOUGH_MAX_LAYERS * kStaticMaxQpt * sizeof(double));
constexpr size_t kOffOffs = align256(kOffCounts + (size_t)kStaticMaxKeys * sizeof(int32_t));
constexpr size_t kOffKey = align256(kOffOffs + (size_t)(kStaticMaxKeys + 1) * sizeof(int32_t));
constexpr size_t kOffRank = align256(kOffKey + (size_t)kStaticMaxHits * sizeof(int32_t));
constexpr size_t kOffHotTmp = align256(kOffRank + (size_t)kStaticMaxHits * sizeof(int32_t));
constexpr size_t kOffHot = align256(kOffHotTmp + (size_t)kStaticMaxHits * sizeof(HotHit));
constexpr size_t kOffCold = align256(kOffHot + (size_t)kStaticMaxHits * sizeof(HotHit));
constexpr size_t kStaticBytes = align256(kOffCold + (size_t)kStaticMaxHits * sizeof(ColdHit));
static_assert(kStaticBytes <= (size_t)8 << 20, "the fixed scratch must stay within 8 MiB");

// The scratch itself.  In host code this name is only a stand-in for the symbol; kernels get the
// device address looked up below.
static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

std::mutex g_setup_mutex;

// Device address of g_scratch on the current device.  It is looked up on every call (a table
// lookup in the runtime, no allocation) rather than cached: after cudaDeviceReset, or once the
// primary context has been released and created again, the module is loaded anew and the array
// may sit elsewhere.
cudaError_t scratch_address(unsigned char **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char *>(p);
    return cudaSuccess;
}

// FP32 q/pT bin centres (the FP64 centre rounded once), computed on the device because a host
// copy would need a staging buffer.
__global__ void static_kq_kernel(Axes ax, float *kq32)
{
    // rounded like the host's centres of a context: the product, then the sum, each rounded once
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ax.n_qpt) kq32[i] = (float)__dadd_rn(ax.qpt_min, __dmul_rn((double)(i % ax.q_rows) + 0.5, ax.dk));
}

}  // namespace

}  // namespace hough

using namespace hough;

extern "C" int hough_vote_static(const hough_geometry *g, const hough_binning *b, const float *r, const float *phi,
                                 const float *z, const uint8_t *layer, int64_t n_hits, uint16_t *accumulator,
                                 uint32_t *device_error, void *stream)
{
    auto fail = [](int code, const char *msg) { return set_last_error(code, msg); };
    if (!g || !b || !accumulator) return fail(HOUGH_EINVAL, "geometry, binning and accumulator are required");
    // the vote kernel writes the accumulator in 16-byte vectors
    if (reinterpret_cast<uintptr_t>(accumulator) & 15u)
        return fail(HOUGH_EINVAL, "hough_vote_static: the accumulator must be 16-byte aligned");
    if (g->n_layers < 1 || g->n_layers > HOUGH_MAX_LAYERS || !(g->b_tesla > 0.0))
        return fail(HOUGH_EINVAL, "n_layers must be 1..16 and b_tesla > 0");
    if (b->n_qpt < 1 || b->n_phi < 64 || b->n_phi % 64 || b->threshold < 1 || !(b->qpt_min < b->qpt_max))
        return fail(HOUGH_EINVAL, "invalid binning");
    if (b->accumulator != HOUGH_ACC_LAYERS && b->accumulator != HOUGH_ACC_COUNTS)
        return fail(HOUGH_EINVAL, "accumulator must be HOUGH_ACC_LAYERS or HOUGH_ACC_COUNTS");
    if (b->n_d0 < 0 || b->reserved != 0 || (b->n_d0 > 0 && !(b->d0_min_cm < b->d0_max_cm)))
        return fail(HOUGH_EINVAL, "invalid d0 axis");
    if ((int64_t)b->n_qpt * (b->n_d0 > 0 ? b->n_d0 : 1) > kStaticMaxQpt || b->n_phi > kStaticMaxPhi)
        return fail(HOUGH_ECAPACITY, "hough_vote_static: rows must be <= 1024 and n_phi <= 4096");
    if (n_hits < 0) return fail(HOUGH_EINVAL, "n_hits must be >= 0");
    if (n_hits > kStaticMaxHits) return fail(HOUGH_ECAPACITY, "hough_vote_static: at most 131072 hits");
    if (n_hits > 0 && (!r || !phi || !z || !layer)) return fail(HOUGH_EINVAL, "hit arrays are required");

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0)
        return fail(HOUGH_ECUDA, "no usable current device");
    unsigned char *base = nullptr;
    if (scratch_address(&base) != cudaSuccess)
        return fail(HOUGH_ECUDA, "cudaGetSymbolAddress of the fixed scratch failed");

    const Axes ax = make_axes(g, b);   // host arithmetic only: nothing is allocated

    Workspace w{};
    w.n_events = 1;
    w.n_hits_total = n_hits;
    w.hit_start = reinterpret_cast<int64_t *>(base + kOffHitStart);
    w.r = r;
    w.phi = phi;
    w.z = z;
    w.layer = layer;
    w.stats = reinterpret_cast<DevStats *>(base + kOffStats);
    w.radii = reinterpret_cast<LayerRadii *>(base + kOffRadii);
    w.info = reinterpret_cast<LayerInfo *>(base + kOffInfo);
    w.memo = reinterpret_cast<TableMemo *>(base + kOffMemo);
    w.kq32 = reinterpret_cast<float *>(base + kOffKq);
    w.tab = reinterpret_cast<TabEntry *>(base + kOffTab);
    w.arc = reinterpret_cast<double *>(base + kOffArc);
    w.counts = reinterpret_cast<int32_t *>(base + kOffCounts);
    w.offs = reinterpret_cast<int32_t *>(base + kOffOffs);
    w.key = reinterpret_cast<int32_t *>(base + kOffKey);
    w.rank = reinterpret_cast<int32_t *>(base + kOffRank);
    w.hot_tmp = reinterpret_cast<HotHit *>(base + kOffHotTmp);
    w.hot = reinterpret_cast<HotHit *>(base + kOffHot);
    w.cold = reinterpret_cast<ColdHit *>(base + kOffCold);
    w.M = accumulator;

    Tiling t;
    t.tile_phi = b->n_phi < 256 ? b->n_phi : 256;
    while (b->n_phi % t.tile_phi) t.tile_phi -= 64;
    t.tile_qpt = b->n_qpt < 32 ? b->n_qpt : 32;
    t.threads = 256;
    t.vote_mode = HOUGH_VOTE_SCATTER;   // the shared-atomic vote kernel alone: no bucket profile needed
    t.band_rows = 4;
    t.gather_rows = 4;
    t.gather_cols = t.tile_phi;
    t.gather_threads = 512;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The array keeps the previous call's contents: reset what the kernels expect to start at zero.
    // The arcsine-table memo is cleared too, since the previous call may have used other axes.
    if (cudaMemsetAsync(base + kOffHitStart, 0, 2 * sizeof(int64_t), s) != cudaSuccess ||
        cudaMemsetAsync(base + kOffMemo, 0, sizeof(TableMemo), s) != cudaSuccess)
        return fail(HOUGH_ECUDA, "clearing the fixed scratch failed");
    static_kq_kernel<<<(ax.n_qpt + 127) / 128, 128, 0, s>>>(ax, w.kq32);
    if (cudaGetLastError() != cudaSuccess) return fail(HOUGH_ECUDA, "q/pT centre kernel failed to launch");
    if (launch_stage(ax, w, s) != cudaSuccess) return fail(HOUGH_ECUDA, "staging kernels failed to launch");
    if (launch_vote(ax, w, t, refine_eps_for(ax), s) != cudaSuccess) return fail(HOUGH_ECUDA, "vote kernel failed to launch");
    note_launches(1 + kStageLaunches + kVoteLaunches);
    if (device_error &&
        cudaMemcpyAsync(device_error, &w.stats->device_error, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(HOUGH_ECUDA, "copying the device error word failed");
    return HOUGH_OK;
}
