// Internal declarations shared by the CUDA translation units of the hough library.
//
// Device layout of a batch of events that share one set of axes (L layers, Nq x Nphi grid).
// Hits of event e occupy [hit_start[e], hit_start[e+1]) of the concatenated hit arrays; every
// other per-event array has a fixed stride:
//   key[n], rank[n]           counting-sort key (layer * Nphi + J) and the hit's rank in its bucket
//   hot_tmp[n]                the hit's 16-byte staged record, input order
//   counts[L*Nphi]            bucket sizes; offs[L*Nphi + 1] their exclusive prefix sum (event-local)
//   prof[16*(Nphi+16)] (8 B)  per (layer, bucket J): .x = max over the bucket of bits(f) + 1,
//                             .y = max over bucket J+1 of ~bits(f) (0 when the bucket is empty);
//                             entries Nphi..Nphi+15 of each layer repeat entries 0..15
//                             (so a window of consecutive buckets never wraps), 16 layers always
//   hot[n], cold[n] (16 B)    staged hits sorted by (layer, J); cold holds r, phi, z, input index
//   tab[L*Nq] (8 B)           per (layer, q/pT row): Nphi asin(x) / (2 pi) = I + g, for layers whose
//                             hits share one radius; arc[L*Nq] the arc length s (FP64)
//   M[Nq*Nphi] (uint16)       stage-1 accumulator, row-major layer masks
//   band_cands[n_bands*band_cap] (8 B)  peak candidates of each row band: cell index, mask
//   cands[max_cand] (32 B)    hough_candidate records in raster order
//   mem_pool[max_members]     member hits (staged positions); mem_start/mem_count per candidate
//                             (contexts only: a batch keeps no member lists)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hough.h"

namespace hough {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.283185307179586;       // 2 * kPi, exactly the double product
constexpr double kInvTwoPi = 0.15915494309189535;  // 1 / (2 pi) rounded to double

// Axes of the two grids, by value into every kernel.
struct Axes {
    int n_layers, n_qpt, n_phi, threshold, n_cot, n_z0;   // n_qpt: rows of the grid, every d0 slice's
    int counts;                   // 1: cells hold saturating vote counts; 0: layer masks
    int q_rows;                   // q/pT bins: row r holds q/pT bin r % q_rows of d0 slice r / q_rows
    int n_d0;                     // d0 bins (0: prompt tracks, one slice at d0 = 0)
    double d0_min, dd;            // d0 axis: first edge and bin width (cm)
    double b, qpt_min, qpt_max, dk;
    double cot_min, cot_max, dt, z0_min, z0_max;
    double zscale;                // n_z0 / (z0_max - z0_min): z0 bins per cm
    float zs_hi, zs_lo;           // zscale as an unevaluated sum of two floats
    float zmin_hi, zmin_lo;       // z0_min likewise
    float pi_hi, pi_lo;           // pi as two floats
    float u_hi, u_lo;             // n_phi / (2 pi) as two floats: bins per radian
};

// Staged hit, the record the vote and membership kernels stream (16 bytes, one vector load).
struct __align__(16) HotHit {
    float f;          // fractional part of the hit's own bin coordinate u_h = Nphi (phi + pi) / (2 pi)
    float c;          // FP32 sagitta coefficient 0.15 B r / 100 (per-vote path)
    uint32_t jl;      // J = floor(u_h) mod Nphi in bits 0..15, layer in bits 16..19
    uint32_t rows;    // first voting row in bits 0..15, last in bits 16..31 (first > last: none)
};

// The same hit's coordinates and its index in the caller's arrays.
struct __align__(16) ColdHit {
    float r, phi, z;
    int32_t idx;
};

// Nphi * asin(x) / (2 pi) = I + g with I integer and g in [0, 1).
struct __align__(8) TabEntry {
    int32_t I;
    float g;
};

// Device counters of one event.
struct DevStats {
    unsigned long long votes_by_layer[HOUGH_MAX_LAYERS];
    unsigned long long refined_votes;
    unsigned long long stage2_votes;
    unsigned long long n_hits;
    unsigned int n_candidates;
    unsigned int n_members;
    unsigned int device_error;
    unsigned int pool_used;     // member-pool entries handed out
    unsigned int pad;
};

// Per-layer radius range: min and max of the hit radii as float bits (radii are > 0).
struct LayerRadii {
    unsigned int rmin[HOUGH_MAX_LAYERS];
    unsigned int rmax[HOUGH_MAX_LAYERS];
};

// Per-layer facts of the current batch, written by the layer-info kernel.
struct LayerInfo {
    int32_t present;    // the layer has hits
    int32_t uniform;    // all its hits share one radius (or it has none): the table path applies
    int32_t lo, hi;     // rows of that radius that may vote (lo > hi: none); a row votes when its
                        // table entry is not kNoVote
    uint32_t r_bits;    // the radius (float bits)
    int32_t nvote;      // rows that vote
    int32_t pad[2];
};

// Table entry of a (layer, row) on which the layer's radius casts no vote.
constexpr int32_t kNoVote = -(1 << 30);

// Memo of the per-(layer, row) table: the radius each layer's rows were computed for.
struct TableMemo {
    uint32_t r_bits[HOUGH_MAX_LAYERS];
    int32_t valid[HOUGH_MAX_LAYERS];
    int32_t dirty[HOUGH_MAX_LAYERS];
    int32_t lo[HOUGH_MAX_LAYERS], hi[HOUGH_MAX_LAYERS];   // voting rows of r_bits
    int32_t nvote[HOUGH_MAX_LAYERS];
};

// Device-resident hit pointers, for launch sequences captured once and replayed on new inputs.
struct HitInputs {
    const float *r, *phi, *z;
    const uint8_t *layer;
};

// Counters of a whole batch.
struct BatchCounters {
    unsigned int total_cands;      // candidates kept over all events
    unsigned int pad1;
    unsigned int peaks_done;       // CTAs of the peak search finished (compaction in the last one)
    unsigned int pad;
};

// Device buffers of a batch of events that share one set of axes.
struct Workspace {
    int n_events;
    int64_t n_hits_total;         // < 0: read hit_start[n_events] on the device
    int64_t hit_capacity;         // grid sizing when the total is read on the device
    const int64_t *hit_start;     // device, n_events + 1
    const float *r, *phi, *z;
    const uint8_t *layer;
    const HitInputs *inputs;      // when set, the hit pointers are read from here on the device
    int32_t *key, *rank;          // per hit
    HotHit *hot_tmp;              // per hit, input order
    int32_t *counts;              // n_events * nkeys
    int32_t *offs;                // n_events * (nkeys + 1)
    uint2 *prof;                  // n_events * prof_event_entries
    HotHit *hot;                  // per hit, sorted within each event's range
    float *fsort;                 // per hit, sorted: the hot record's f alone (count gather, membership)
    float *zsort;                 // per hit, sorted: z alone (membership; may be null when no stage 2 runs)
    ColdHit *cold;
    LayerRadii *radii;            // batch-wide
    LayerInfo *info;              // HOUGH_MAX_LAYERS
    TableMemo *memo;
    TabEntry *tab;                // n_layers * n_qpt
    double *arc;                  // n_layers * n_qpt
    float4 *zco;                  // n_layers * n_qpt stage-2 terms {S hi, S lo, B hi, B lo} (may be null)
    float *kq32;                  // n_qpt: FP32 q/pT bin centres
    uint16_t *M;                  // n_events * n_qpt * n_phi
    uint2 *band_cands;            // n_events * n_bands * band_cap
    int32_t *band_counts;         // n_events * n_bands
    int32_t *band_offs;           // n_events * n_bands
    hough_candidate *cands;       // n_events * max_cand
    int32_t *mem_pool;            // max_members: event-local staged positions (contexts only)
    int32_t *mem_start;           // max_cand (contexts only)
    int32_t *mem_count;           // max_cand: entries written to the pool (contexts only)
    int32_t *cand_base;           // n_events + 1: first flattened candidate index of each event
    BatchCounters *counters;
    DevStats *stats;              // n_events
    int max_cand, max_members;
    int band_rows, band_cap;
    int fused;                    // vote_mode HOUGH_VOTE_FUSED: the vote kernel searched the bands
    int keep_members;             // 1: confirmation writes member lists to mem_pool (contexts); 0: none (batches)
    int copy_wait;                // < 0: the first bound on a bulk-copy wait expires at once (a test of the error path)
    int compact_in_peaks;         // one event: the peak kernel's last CTA compacts the candidate list
    int cands_from_bands;         // one event: the confirmation reads its candidates from the band lists
    // A context's state is left clean for its next event by the kernels that last use it, so that no
    // clearing kernel opens the next event: the hit sort zeroes the bucket counts, the peak search
    // the bucket profile, and the counting kernel the counters and radius ranges of the next event,
    // which alternate between two buffers (the host may read this event's counters meanwhile).
    int recycle;
    DevStats *stats_next;         // recycle: the next event's counters, zeroed by the counting kernel
    LayerRadii *radii_next;       // recycle: the next event's radius ranges, reset likewise
};

// Vote-kernel configuration.
struct Tiling {
    int tile_qpt, tile_phi, threads;
    int vote_mode;                // HOUGH_VOTE_GATHER, HOUGH_VOTE_SCATTER or HOUGH_VOTE_FUSED
    int band_rows;                // rows per band of the peak search
    int gather_rows, gather_cols, gather_threads;   // tile of the gather kernel (0: its default)
};

constexpr int kPeakThreads = 256;

// Refinement of the per-vote FP32 path: votes whose FP32 bin coordinate lies within the refine
// window of an edge, or whose |x| exceeds kRefineXLim, are recomputed in FP64.
constexpr float kRefineXLim = 0.99f;

__host__ __device__ inline int n_keys(const Axes &ax) { return ax.n_layers * ax.n_phi; }
// Bucket-profile stride per layer and per event (16 layers, each padded by 16 repeated buckets).
constexpr int kProfPad = 16;
__host__ __device__ inline int prof_stride(const Axes &ax) { return ax.n_phi + kProfPad; }
__host__ __device__ inline int64_t prof_event_entries(const Axes &ax) { return (int64_t)HOUGH_MAX_LAYERS * prof_stride(ax); }
// Bands of band_rows rows; with a d0 axis a band never crosses a slice (each slice is cut alone).
__host__ __device__ inline int n_bands(const Axes &ax, int band_rows)
{
    if (ax.n_d0) return ax.n_d0 * ((ax.q_rows + band_rows - 1) / band_rows);
    return (ax.n_qpt + band_rows - 1) / band_rows;
}
// Candidates are never 8-neighbours, so a band holds at most one per 2 x 2 block.
__host__ __device__ inline int band_capacity(const Axes &ax, int band_rows)
{
    return ((band_rows + 1) / 2) * ((ax.n_phi + 1) / 2);
}

// Refine window (in bins) of the per-vote FP32 path.  Its error is bounded by the asinf error,
// the FP32 rounding of x = c k propagated through asin up to |x| = kRefineXLim, and the rounding
// of the bin coordinate; the sum grows with Nphi / (2 pi).
inline float refine_eps_for(const Axes &ax) { return (float)(ax.n_phi * 5e-7 + 1e-4); }

// Kernel launchers (each enqueues on `stream` and returns the launch status).
// `after`, when given, receives an event after each of the first four staging kernels (clear, count,
// layer table, scan); the caller times the last one.
// clear: open with the clearing kernel (else the state must have been left clean, Workspace::recycle).
cudaError_t launch_stage(const Axes &ax, const Workspace &w, cudaStream_t stream, cudaEvent_t *after = nullptr,
                         bool clear = true);
cudaError_t launch_vote(const Axes &ax, const Workspace &w, const Tiling &t, float refine_eps,
                        cudaStream_t stream);
cudaError_t launch_peaks(const Axes &ax, const Workspace &w, const Tiling &t, cudaStream_t stream);
// The pieces of launch_vote and launch_peaks, for callers that time them separately.
cudaError_t launch_gather(const Axes &ax, const Workspace &w, const Tiling &t, cudaStream_t stream);
cudaError_t launch_scatter(const Axes &ax, const Workspace &w, const Tiling &t, float refine_eps, bool general_only,
                           cudaStream_t stream);
cudaError_t launch_band_peaks(const Axes &ax, const Workspace &w, const Tiling &t, cudaStream_t stream);
cudaError_t launch_compact(const Axes &ax, const Workspace &w, cudaStream_t stream);
// All events' candidates concatenated: the first `limit` into `out` (device-accessible), the rest
// into `rest` at the same indices when it is given, else dropped; the first event's counters to
// `stats_out` (device-accessible) when it is given.
cudaError_t launch_pack_candidates(const Axes &ax, const Workspace &w, hough_candidate *out, cudaStream_t stream,
                                   long long limit = 1LL << 62, hough_candidate *rest = nullptr,
                                   DevStats *stats_out = nullptr, int blocks = 1216);
cudaError_t launch_stage2(const Axes &ax, const Workspace &w, int sms, float refine_eps, cudaStream_t stream,
                          cudaEvent_t between = nullptr);
cudaError_t launch_member_index(const Workspace &w, int32_t *idx_out, int64_t total, cudaStream_t stream);
cudaError_t run_smem_or_bench(int device, int pattern, double ms, double *atomics_per_s, uint64_t *launches);

size_t vote_smem_bytes(const Axes &ax, const Tiling &t);
// Shared memory of the peak search over bands of band_rows rows.
__host__ __device__ inline size_t band_smem_bytes(const Axes &ax, int band_rows)
{
    // with a d0 axis the band's rows and their halo in three slices
    const size_t rows = (size_t)(band_rows + 2) * (ax.n_d0 ? 3 : 1);
    // layer masks: the layer counts as bytes, then the band's own rows' masks (the candidates' masks,
    // read from there instead of from device memory)
    const size_t masks = (!ax.n_d0 && !ax.counts) ? (size_t)band_rows * ax.n_phi * 2 : 0;
    return rows * ax.n_phi * (ax.counts ? 2 : 1) + masks;
}
size_t stage2_smem_bytes(const Axes &ax);
// Whether the confirmation of one event may read its candidates straight from the band lists.
bool stage2_reads_bands(const Axes &ax, int band_rows);

// Host helpers shared by the single-event and the batch entry points (hough_api.cu).
Axes make_axes(const hough_geometry *g, const hough_binning *b);
int check_geometry_binning(const hough_geometry *g, const hough_binning *b);
int check_tiling_for(const Axes &ax, int device, const hough_tiling *t);
Tiling default_tiling_for(const Axes &ax);
Tiling resolve_tiling(const Axes &ax, const hough_tiling *t);   // gather defaults filled in
void public_tiling(const Tiling &t, hough_tiling *out);
size_t gather_smem_bytes(const Axes &ax, const Tiling &t);
// Dynamic shared memory of the fused vote and peak kernel: the band's masks and its two halo rows.
size_t fused_smem_bytes(const Axes &ax, int band_rows);
// Shared memory of the count accumulator's gather kernel.
size_t gather_count_smem_bytes(const Axes &ax, const Tiling &t);
size_t band_list_entries(const Axes &ax);
int check_host_hits_for(const Axes &ax, const float *r, const float *phi, const float *z, const uint8_t *layer,
                        int64_t n);
void fill_stats(const DevStats &d, const LayerInfo *info, int n_layers, hough_stats *out);

// Batch internals used by the server: a run with or without the host-side hit checks, and the
// asynchronous result copies (offsets first, then exactly the candidates they announce).
int batch_run(hough_batch *b, const float *r, const float *phi, const float *z, const uint8_t *layer,
              const int64_t *hit_start, int32_t n_events, int where, cudaStream_t stream, bool check_hits);
int batch_enqueue_offsets(hough_batch *b, int32_t *offsets_host, cudaStream_t s);
// The same, with the candidates packed straight into `mapped` (a device pointer of mapped pinned
// host memory), at most `cap` of them; the rest stay in the batch's device buffer.
int batch_enqueue_offsets_mapped(hough_batch *b, int32_t *offsets_host, hough_candidate *mapped, int64_t cap,
                                 cudaStream_t s);
int batch_enqueue_candidates(hough_batch *b, hough_candidate *dst_host, int64_t n, cudaStream_t s, int64_t first = 0);
int batch_enqueue_stats(hough_batch *b, DevStats *stats_host, int n, cudaStream_t s);
size_t batch_device_bytes(const hough_batch *b);

// Record a failure for hough_last_error (returns code), and count launches for hough_kernel_launches.
int set_last_error(int code, const char *msg);
void note_launches(uint64_t n);

// Kernels launched by each enqueue function (for hough_kernel_launches).
constexpr int kStageLaunches = 4;
constexpr int kVoteLaunches = 2;
// peak search, compaction, and for batches of several events the candidate-base scan
inline int peak_launches(int n_events) { return n_events == 1 ? 2 : 3; }
constexpr int kStage2Launches = 1;

// Exact FP64 helpers used by the staging, table and refinement code.  They evaluate the
// definitions in the order of the method's formulas with explicitly rounded operations,
// so no multiply-add is fused.
// Programmatic dependent launch: every kernel of the path is launched with programmatic stream
// serialisation (launch_chained), so the next kernel's grid is set up while this one runs; each
// kernel first waits for its predecessor's completion and memory (griddepcontrol.wait) and only
// then lets its own dependent launch.  A kernel launched without the attribute passes the wait at
// once.  Every kernel launched through launch_chained must begin with pdl_enter().
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                                  Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Bulk asynchronous copies (TMA, untiled form) from global to shared memory, completing on an
// mbarrier.  Both addresses must be 16-byte aligned and the size a multiple of 16 bytes.
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Wait for phase `phase` of the mbarrier for at most `max_cycles` SM cycles; false when the bound
// ran out (the caller reports it and must not use the copied data).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned phase, long long max_cycles)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase))
        if (clock64() - t0 > max_cycles) return false;
    return true;
}

// Error-free transformations of FP32 arithmetic (Knuth's two-sum, and the product with its
// rounding error from one fused multiply-add): a + b = s + e and a b = p + e exactly.
__device__ __forceinline__ float2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}

__device__ __forceinline__ float2 two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return make_float2(p, fmaf(a, b, -p));
}

// q/pT bin centre of row r (its q/pT bin r % q_rows with a d0 axis).
__device__ __forceinline__ double qpt_centre(const Axes &ax, int r)
{
    const int i = ax.n_d0 ? r % ax.q_rows : r;
    return __dadd_rn(ax.qpt_min, __dmul_rn((double)i + 0.5, ax.dk));
}

// d0 bin centre of row r (0 without a d0 axis).
__device__ __forceinline__ double d0_centre(const Axes &ax, int r)
{
    if (!ax.n_d0) return 0.0;
    return __dadd_rn(ax.d0_min, __dmul_rn((double)(r / ax.q_rows) + 0.5, ax.dd));
}

// sin(phi - phi0) of a hit at radius r on the track of sagitta argument x and impact parameter d0:
// (rho r^2 + 2 d0 + rho d0^2) / (2 r (1 + rho d0)) with rho = 2 x / r, in FP64 in that order; x
// itself at d0 = 0.  Returns false when 1 + rho d0 <= 0 (no such track).
__device__ __forceinline__ bool track_sin(double r, double x, double d0, double *y)
{
    if (d0 == 0.0) {
        *y = x;
        return true;
    }
    const double rho = __ddiv_rn(__dmul_rn(2.0, x), r);
    const double den = __dmul_rn(__dmul_rn(2.0, r), __dadd_rn(1.0, __dmul_rn(rho, d0)));
    if (!(den > 0.0)) return false;
    const double num = __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(rho, r), r), __dmul_rn(2.0, d0)),
                                 __dmul_rn(__dmul_rn(rho, d0), d0));
    *y = __ddiv_rn(num, den);
    return true;
}

// Transverse arc length from the closest approach to that hit: r asin(|x|) / |x| at d0 = 0, else
// 2 asin(|rho| chord / 2) / |rho| with chord^2 = r^2 + d0^2 - 2 r d0 y.
__device__ __forceinline__ double track_arc(double r, double x, double d0, double y)
{
    const double ax = fabs(x);
    if (d0 == 0.0) return ax > 0.0 ? __ddiv_rn(__dmul_rn(r, asin(ax)), ax) : r;
    const double c2 = __dsub_rn(__dadd_rn(__dmul_rn(r, r), __dmul_rn(d0, d0)), __dmul_rn(__dmul_rn(__dmul_rn(2.0, r), d0), y));
    const double chord = __dsqrt_rn(c2);
    const double arho = __ddiv_rn(__dmul_rn(2.0, ax), r);
    return arho > 0.0 ? __ddiv_rn(__dmul_rn(2.0, asin(__ddiv_rn(__dmul_rn(arho, chord), 2.0))), arho) : chord;
}

__device__ __forceinline__ double sagitta_coef(const Axes &ax, double r_cm)
{
    return __dmul_rn(__dmul_rn(0.15, ax.b), __ddiv_rn(r_cm, 100.0));
}

// Hit total and hit arrays of the batch (from the device when the launch sequence is replayed).
__device__ __forceinline__ int64_t hit_total(const Workspace &w)
{
    return w.n_hits_total >= 0 ? w.n_hits_total : w.hit_start[w.n_events];
}

__device__ __forceinline__ HitInputs hit_inputs(const Workspace &w)
{
    if (w.inputs) return *w.inputs;
    HitInputs in;
    in.r = w.r;
    in.phi = w.phi;
    in.z = w.z;
    in.layer = w.layer;
    return in;
}

// Last index e in [0, n) with base[e] <= f (base non-decreasing, base[0] = 0).
template <typename T>
__device__ __forceinline__ int upper_index(const T *base, int n, long long f)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((long long)__ldg(&base[mid]) <= f) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Event index of hit h: the last e with hit_start[e] <= h.
__device__ __forceinline__ int event_of(const int64_t *hit_start, int n_events, int64_t h)
{
    int lo = 0, hi = n_events - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&hit_start[mid]) <= h) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Voting rows of a hit with FP64 sagitta coefficient c > 0: rows i with |c k_i| <= 1, decided
// with the exact predicate.  Returns lo > hi when there is none.
__device__ __forceinline__ void row_range(const Axes &ax, double c, int *lo_out, int *hi_out)
{
    const int n = ax.n_qpt;
    auto valid = [&](int i) { return fabs(__dmul_rn(c, qpt_centre(ax, i))) <= 1.0; };
    double klim = 1.0 / c;
    double flo = ceil((-klim - ax.qpt_min) / ax.dk - 0.5);
    double fhi = floor((klim - ax.qpt_min) / ax.dk - 0.5);
    int lo = (int)fmin(fmax(flo, 0.0), (double)(n - 1));
    int hi = (int)fmin(fmax(fhi, 0.0), (double)(n - 1));
    // the estimates sit within a row of the true edges; settle them with the exact predicate
    while (lo > 0 && valid(lo - 1)) --lo;
    while (lo < n && !valid(lo)) ++lo;
    if (lo >= n) { *lo_out = 1; *hi_out = 0; return; }
    if (hi < lo) hi = lo;
    while (hi + 1 < n && valid(hi + 1)) ++hi;
    while (hi > lo && !valid(hi)) --hi;
    *lo_out = lo;
    *hi_out = hi;
}

// phi0 bin of one vote, evaluated like the definition: floor(Nphi (phi - asin(x) + pi) / (2 pi)) mod Nphi.
__device__ __forceinline__ int exact_bin(const Axes &ax, double phi, double x)
{
    double phi0 = __dsub_rn(phi, asin(x));
    double u = __ddiv_rn(__dmul_rn((double)ax.n_phi, __dadd_rn(phi0, kPi)), kTwoPi);
    long long j = (long long)floor(u) % ax.n_phi;
    return (int)(j < 0 ? j + ax.n_phi : j);
}

// The vote of a hit (r, phi) on row `row` by the definition, in FP64: false when the row's track
// cannot pass the hit's radius (1 + rho d0 <= 0 or |sin(phi - phi0)| > 1), else its phi0 bin in *j.
__device__ __forceinline__ bool exact_vote(const Axes &ax, double r, double phi, int row, int *j)
{
    const double x = __dmul_rn(sagitta_coef(ax, r), qpt_centre(ax, row));
    double y = 2.0;
    if (!track_sin(r, x, d0_centre(ax, row), &y) || !(fabs(y) <= 1.0)) return false;
    *j = exact_bin(ax, phi, y);
    return true;
}

__device__ __forceinline__ int wrap_col(int j, int n)
{
    j += j < 0 ? n : 0;
    return j >= n ? j - n : j;
}

// Peak test of the cells of rows 1..nrows of a band held as cell values in shared memory
// (`pc`, (nrows + 2) rows of Nphi values of type V -- layer counts as bytes, or 16-bit vote
// counts -- row 0 and row nrows + 1 the halo), in raster order.
// A cell with value p is a candidate when p >= threshold, the neighbours at (-1,-1), (-1,0),
// (-1,+1), (0,-1) are below p and the other four are not above it; phi0 wraps.  Each thread tests
// 8 consecutive cells per pass, so thread order is raster order and one block-wide scan of the
// per-thread counts places every candidate.  Candidates go to `out` (cell index i * Nphi + j,
// mask read from M) in raster order; returns their number.  Called by all TPB threads.
// D3 (a grid with a d0 axis): the band's 3 x 3 x 3 blocks are held as three slices of nrows + 2
// rows each -- slice m - 1, the band's own, slice m + 1 -- the band's rows in the middle one; the
// nine neighbours of slice m - 1 precede a cell in raster order (strictly lower), the nine of
// slice m + 1 follow it (not higher).
// MASKS: the staged values are the cells' layer masks themselves (compared by their layer counts,
// and written out from shared memory, M unused).  SMASK: M points to the band's own rows' masks in
// shared memory (nrows rows of Nphi), not to the accumulator.
template <int TPB, typename V, bool D3 = false, bool MASKS = false, bool SMASK = false>
__device__ __forceinline__ int band_peak_search(const V *pc, int nrows, int i0, int nphi, int threshold,
                                                const uint16_t *M, uint2 *out, int cap)
{
    auto val = [](V x) -> int { return MASKS ? __popc((unsigned)x) : (int)x; };
    __shared__ int s_warp[TPB / 32];
    __shared__ int s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int eighth = nphi >> 3;
    const int items = nrows * eighth;
    int running = 0;
    for (int base = 0; base < items; base += TPB) {
        const int it = base + threadIdx.x;
        unsigned pk = 0u;
        int rr = 0, j0 = 0;
        if (it < items) {
            rr = it / eighth;
            j0 = (it - rr * eighth) * 8;
            const int S = nrows + 2;   // rows of one staged slice (D3)
            const V *row = pc + (D3 ? S + rr + 1 : rr + 1) * nphi;
            const V *up = row - nphi, *dn = row + nphi;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int j = j0 + c;
                const int p = val(row[j]);
                if (p >= threshold) {
                    const int jm = wrap_col(j - 1, nphi), jp = wrap_col(j + 1, nphi);
                    bool peak = val(up[jm]) < p && val(up[j]) < p && val(up[jp]) < p && val(row[jm]) < p &&
                                val(row[jp]) <= p && val(dn[jm]) <= p && val(dn[j]) <= p && val(dn[jp]) <= p;
                    if (D3) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            const V *a = pc + (rr + q) * nphi, *b = pc + (2 * S + rr + q) * nphi;
                            peak = peak && a[jm] < p && a[j] < p && a[jp] < p && b[jm] <= p && b[j] <= p &&
                                   b[jp] <= p;
                        }
                    }
                    pk |= (unsigned)peak << c;
                }
            }
        }
        const int cnt = __popc(pk);
        // skip the block-wide scan when no thread of the block found a candidate
        if (!__syncthreads_or(cnt)) continue;
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int v = lane < TPB / 32 ? s_warp[lane] : 0;
            int wi = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(0xFFFFFFFFu, wi, d);
                if (lane >= d) wi += t;
            }
            if (lane < TPB / 32) s_warp[lane] = wi - v;
            if (lane == 31) s_total = wi;
        }
        __syncthreads();
        int idx = running + s_warp[warp] + incl - cnt;
        while (pk) {
            const int c = __ffs(pk) - 1;
            pk &= pk - 1u;
            const unsigned cellg = (unsigned)(i0 + rr) * (unsigned)nphi + (unsigned)(j0 + c);
            if (idx < cap)
                out[idx] = make_uint2(cellg, MASKS   ? (unsigned)pc[(rr + 1) * nphi + j0 + c]
                                             : SMASK ? (unsigned)M[rr * nphi + j0 + c]
                                                     : (unsigned)M[cellg]);
            ++idx;
        }
        running += s_total;
        __syncthreads();
    }
    return running;
}

}  // namespace hough
