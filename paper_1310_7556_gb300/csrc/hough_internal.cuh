// Internal declarations shared by the CUDA translation units of the hough library.
//
// Data layout in device memory for one event (n hits, L layers, Nq x Nphi grid):
//   key[n], rank[n]          counting-sort key (layer * Nphi + J) and the hit's rank in its bucket
//   counts[L*Nphi]           bucket sizes; offs[L*Nphi + 1] their exclusive prefix sum
//   hot[n]   (16 B)          staged hit, sorted by (layer, J): fraction f, FP32 c, J | layer, row range
//   cold[n]  (16 B)          the same hit's r, phi, z and input index, same order
//   tab[L*Nq] (8 B)          per (layer, q/pT row): Nphi * asin(x) / (2 pi) = I + g  (uniform-radius layers)
//   arc[L*Nq] (8 B)          per (layer, q/pT row): arc length s in FP64         (uniform-radius layers)
//   M[Nq*Nphi] (uint16)      stage-1 accumulator, row-major layer masks
//   cands[max_cand] (32 B)   hough_candidate records in raster order
//   mem_pos[max_members]     member hits (staged positions), grouped per candidate
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hough.h"

namespace hough {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.283185307179586;   // 2 * kPi, exactly the double product
constexpr double kInvTwoPi = 0.15915494309189535;  // 1 / (2 pi) rounded to double

// Axes of the two grids, by value into every kernel.
struct Axes {
    int n_layers, n_qpt, n_phi, threshold, n_cot, n_z0;
    double b, qpt_min, qpt_max, dk;
    double cot_min, cot_max, dt, z0_min, z0_max;
};

// Staged hit, the record the vote kernel streams (16 bytes, one vector load).
struct __align__(16) HotHit {
    float f;          // fractional part of the hit's phi0 bin coordinate u_h = Nphi (phi + pi) / (2 pi)
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
    unsigned int pad;
};

// Per-layer radius range: min and max of the hit radii as float bits (radii are > 0).
struct LayerRadii {
    unsigned int rmin[HOUGH_MAX_LAYERS];
    unsigned int rmax[HOUGH_MAX_LAYERS];
};

// Per-layer facts of the current batch, written by the layer-info kernel.
struct LayerInfo {
    int32_t uniform;    // all hits of the layer share one radius: the table path applies
    int32_t lo, hi;     // voting rows of that radius (lo > hi: none)
    uint32_t r_bits;    // the radius (float bits)
};

// Memo of the per-(layer, row) table: the radius each layer's rows were computed for.
struct TableMemo {
    uint32_t r_bits[HOUGH_MAX_LAYERS];
    int32_t valid[HOUGH_MAX_LAYERS];
    int32_t dirty[HOUGH_MAX_LAYERS];
};

// Device buffers of a batch of events that share one set of axes.  Hits of event e occupy
// [hit_start[e], hit_start[e+1]) of the concatenated arrays; every other per-event array
// has a fixed stride.
struct Workspace {
    int n_events;
    int64_t n_hits_total;
    const int64_t *hit_start;     // device, n_events + 1
    const float *r, *phi, *z;
    const uint8_t *layer;
    int32_t *key, *rank;          // per hit
    HotHit *hot_tmp;              // per hit, input order
    int32_t *counts;              // n_events * nkeys
    int32_t *offs;                // n_events * (nkeys + 1), event-local
    HotHit *hot;                  // per hit, staged order within each event's range
    ColdHit *cold;
    LayerRadii *radii;            // batch-wide
    LayerInfo *info;              // HOUGH_MAX_LAYERS
    TableMemo *memo;
    TabEntry *tab;                // n_layers * n_qpt
    double *arc;                  // n_layers * n_qpt
    float *kq32;                  // n_qpt: FP32 q/pT bin centres
    uint16_t *M;                  // n_events * n_qpt * n_phi
    hough_candidate *cands;       // n_events * max_cand
    int32_t *band_counts;         // n_events * n_bands
    int32_t *band_offs;           // n_events * n_bands
    int32_t *mem_counts;          // n_events * max_cand
    int64_t *mem_offs;            // n_events * (max_cand + 1)
    int32_t *mem_pos;             // n_events * max_members: event-local staged positions
    DevStats *stats;              // n_events
    int max_cand, max_members;
};

struct Tiling {
    int tile_qpt, tile_phi, threads;
};

// Row band of the peak kernels.
constexpr int kPeakRows = 4;
constexpr int kPeakThreads = 256;

// Refinement of the per-vote FP32 path: votes whose FP32 bin coordinate lies within
// the refine window of an edge, or whose |x| exceeds kRefineXLim, are recomputed in FP64.
constexpr float kRefineXLim = 0.99f;
// Stage-2 FP32 window: a (member, cot) vote within this distance of a z0 edge is recomputed in FP64.
constexpr float kStage2Eps = 2e-4f;

// Kernel launchers (each enqueues on `stream` and returns the launch status).
cudaError_t launch_stage(const Axes &ax, const Workspace &w, cudaStream_t stream);
cudaError_t launch_vote(const Axes &ax, const Workspace &w, const Tiling &t, float refine_eps,
                        cudaStream_t stream);
cudaError_t launch_peaks(const Axes &ax, const Workspace &w, cudaStream_t stream);
cudaError_t launch_stage2(const Axes &ax, const Workspace &w, int sms, cudaStream_t stream);

cudaError_t launch_member_index(const Workspace &w, int32_t *idx_out, int64_t total, cudaStream_t stream);

cudaError_t run_smem_or_bench(int device, int pattern, double ms, double *atomics_per_s, uint64_t *launches);

// Record a failure for hough_last_error (returns code), and count launches for hough_kernel_launches.
int set_last_error(int code, const char *msg);
void note_launches(uint64_t n);

// Kernels launched by each enqueue function (for hough_kernel_launches).
constexpr int kStageLaunches = 5;
constexpr int kVoteLaunches = 1;
constexpr int kPeakLaunches = 3;
constexpr int kStage2Launches = 4;

size_t vote_smem_bytes(const Axes &ax, const Tiling &t);
size_t stage2_smem_bytes(const Axes &ax);

// Refine window (in bins) of the per-vote FP32 path.  Its error is bounded by the asinf error,
// the FP32 rounding of x = c k propagated through asin up to |x| = kRefineXLim, and the rounding
// of the bin coordinate; the sum grows with Nphi / (2 pi).
inline float refine_eps_for(const Axes &ax) { return (float)(ax.n_phi * 5e-7 + 1e-4); }
__host__ __device__ inline int n_bands(const Axes &ax) { return (ax.n_qpt + kPeakRows - 1) / kPeakRows; }
__host__ __device__ inline int n_keys(const Axes &ax) { return ax.n_layers * ax.n_phi; }

// Exact FP64 helpers used by the staging, table and refinement code.  They evaluate the
// definitions in the order of the method's formulas with explicitly rounded operations,
// so no multiply-add is fused.
__device__ __forceinline__ double qpt_centre(const Axes &ax, int i)
{
    return __dadd_rn(ax.qpt_min, __dmul_rn((double)i + 0.5, ax.dk));
}

__device__ __forceinline__ double sagitta_coef(const Axes &ax, double r_cm)
{
    return __dmul_rn(__dmul_rn(0.15, ax.b), __ddiv_rn(r_cm, 100.0));
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

}  // namespace hough
