// Hit staging (the first step of the path): validation, the phi0 bin of each hit's own
// azimuth, a counting sort of the hits by (layer, phi bin) and the per-(layer, q/pT row)
// arcsine table.
//
// Sorting by (layer, phi bin) is what lets the vote kernel read only the hits that can
// vote into its accumulator tile: a hit's votes on row i sit Nphi * asin(x_i) / (2 pi) bins
// from its own azimuth bin, so the hits of a tile form a few contiguous key ranges.
//
// The arcsine of the sagitta argument x = 0.15 B (r/100) k_i depends only on the hit's
// radius and the row, not on its azimuth (the paper's GPU optimisation of cutting the
// trigonometric work, Sec. 6.1).  When every hit of a layer shares one radius the table
// holds that value per (layer, row) in FP64, and a vote reduces to an integer subtraction
// and one FP32 comparison.  The staging also records, per (layer, phi bucket), the largest
// and smallest fraction f of the hits in it: with the table they decide every cell of the
// accumulator directly (see vote_kernel.cu).
#include <algorithm>
#include <cstdint>

#include "hough_internal.cuh"

namespace hough {

namespace {

constexpr int kStageThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kClearThreads = 256;

// The per-call state the staging starts from, cleared by one kernel instead of one memset each:
// up to kClearSegs ranges of 32-bit words, each set to a value (16-byte stores where aligned).
constexpr int kClearSegs = 6;
struct ClearList {
    uint32_t *p[kClearSegs];
    long long words[kClearSegs];
    uint32_t value[kClearSegs];
    int n;
};

__global__ void __launch_bounds__(kClearThreads) clear_kernel(ClearList cl)
{
    pdl_enter();
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int q = 0; q < cl.n; ++q) {
        uint32_t *p = cl.p[q];
        const long long n = cl.words[q];
        const uint32_t v = cl.value[q];
        const bool vec = ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) && (n % 4 == 0);
        if (vec) {
            uint4 *p4 = reinterpret_cast<uint4 *>(p);
            const uint4 v4 = make_uint4(v, v, v, v);
            for (long long k = t0; k < n / 4; k += stride) p4[k] = v4;
        } else {
            for (long long k = t0; k < n; k += stride) p[k] = v;
        }
    }
}

__global__ void __launch_bounds__(kStageThreads) stage_count_kernel(Axes ax, Workspace w)
{
    pdl_enter();
    __shared__ unsigned int s_rmin[HOUGH_MAX_LAYERS], s_rmax[HOUGH_MAX_LAYERS];
    if (threadIdx.x < HOUGH_MAX_LAYERS) {
        s_rmin[threadIdx.x] = 0xFFFFFFFFu;
        s_rmax[threadIdx.x] = 0u;
    }
    if (w.recycle && blockIdx.x == 0) {
        // the next event's counters and radius ranges (the other buffer of each pair)
        uint32_t *sn = reinterpret_cast<uint32_t *>(w.stats_next);
        for (int q = threadIdx.x; q < (int)(sizeof(DevStats) / 4); q += blockDim.x) sn[q] = 0u;
        if (threadIdx.x < HOUGH_MAX_LAYERS) {
            w.radii_next->rmin[threadIdx.x] = 0xFFFFFFFFu;
            w.radii_next->rmax[threadIdx.x] = 0u;
        }
    }
    __syncthreads();
    const int nkeys = n_keys(ax);
    // FP32 sagitta coefficient of the per-vote path; its rounding is covered by the refine window
    const float cscale = (float)(0.15 * ax.b / 100.0);
    const int64_t total = hit_total(w);
    const HitInputs in = hit_inputs(w);
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < total;
         h += (int64_t)gridDim.x * blockDim.x) {
        const int e = event_of(w.hit_start, w.n_events, h);
        const float rr = __ldg(&in.r[h]);
        const float ph = __ldg(&in.phi[h]);
        const float zz = __ldg(&in.z[h]);
        const int l = __ldg(&in.layer[h]);
        unsigned bad = 0;
        if (l >= ax.n_layers) bad |= HOUGH_DEVERR_LAYER;
        if (!(rr > 0.f) || !isfinite(rr) || !(fabsf(ph) <= 1000.f) || !isfinite(zz))
            bad |= HOUGH_DEVERR_RADIUS;
        if (bad) {
            atomicOr(&w.stats[e].device_error, bad);
            w.key[h] = -1;
            continue;
        }
        // bin coordinate of the hit's own azimuth: u_h = Nphi (phi + pi) / (2 pi) = J + f, in
        // two-float arithmetic (about 2^-44 relative: 1e-10 bins at Nphi = 2048), since the
        // fraction must resolve far below the 1e-4-bin window in which votes may differ
        float2 sp = two_sum(ph, ax.pi_hi);
        sp.y = __fadd_rn(sp.y, ax.pi_lo);
        float2 u = two_prod(sp.x, ax.u_hi);
        u.y = u.y + (sp.x * ax.u_lo + sp.y * ax.u_hi);
        float fl = floorf(u.x);
        float f = __fadd_rn(__fsub_rn(u.x, fl), u.y);   // u.x - fl is exact
        if (f < 0.f) {
            f = __fadd_rn(f, 1.f);
            fl -= 1.f;
        }
        if (f >= 1.f) {   // also the fraction that rounded up to 1: carry into J
            f = __fsub_rn(f, 1.f);
            fl += 1.f;
        }
        int J = (int)fl % ax.n_phi;
        if (J < 0) J += ax.n_phi;
        const int k = l * ax.n_phi + J;
        w.key[h] = k;
        w.rank[h] = atomicAdd(&w.counts[(int64_t)e * nkeys + k], 1);
        // bucket extrema of f as ordered bit patterns (f >= 0): .x of bucket J keeps the maximum
        // (offset by one so an empty bucket, 0, is below every hit), .y of bucket J-1 keeps the
        // maximum of the complement, i.e. the minimum of bucket J
        if (w.prof) {
            uint2 *prof = w.prof + (int64_t)e * prof_event_entries(ax) + (int64_t)l * prof_stride(ax);
            const int Jm = J == 0 ? ax.n_phi - 1 : J - 1;
            atomicMax(&prof[J].x, __float_as_uint(f) + 1u);
            atomicMax(&prof[Jm].y, ~__float_as_uint(f));
            if (J < kProfPad) atomicMax(&prof[J + ax.n_phi].x, __float_as_uint(f) + 1u);   // the repeated copy
            if (Jm < kProfPad) atomicMax(&prof[Jm + ax.n_phi].y, ~__float_as_uint(f));
        }
        HotHit hh;
        hh.f = f;
        hh.c = __fmul_rn(cscale, rr);
        hh.jl = (uint32_t)J | ((uint32_t)l << 16);
        hh.rows = 0;
        w.hot_tmp[h] = hh;
        // radii are mostly equal within a layer: only a hit outside the range seen so far updates it
        const unsigned rb = __float_as_uint(rr);
        if (rb < *(volatile unsigned *)&s_rmin[l]) atomicMin(&s_rmin[l], rb);
        if (rb > *(volatile unsigned *)&s_rmax[l]) atomicMax(&s_rmax[l], rb);
    }
    __syncthreads();
    if (threadIdx.x < HOUGH_MAX_LAYERS && s_rmax[threadIdx.x] != 0u) {
        atomicMin(&w.radii->rmin[threadIdx.x], s_rmin[threadIdx.x]);
        atomicMax(&w.radii->rmax[threadIdx.x], s_rmax[threadIdx.x]);
    }
}

// One CTA per layer: whether all the layer's hits share one radius, that radius's voting rows and
// whether the memoised table rows must be recomputed; then, for a uniform layer whose radius
// changed, per row: T = Nphi asin(y) / (2 pi) split into I + g, y = sin(phi - phi0) of the row's
// track (y = x for prompt tracks, the d0 relation on a grid with a d0 axis), the arc length from
// the closest approach for stage 2, and the stage-2 terms derived from it.  Rows on which the
// radius casts no vote get the entry kNoVote.
__device__ __forceinline__ void layer_table(const Axes &ax, const Workspace &w, const int l)
{
    __shared__ LayerInfo s_li;
    __shared__ int s_dirty;
    if (threadIdx.x == 0) {
        LayerInfo li;
        const unsigned rmin = w.radii->rmin[l], rmax = w.radii->rmax[l];
        li.present = (l < ax.n_layers) && rmax != 0u;
        li.uniform = !li.present || rmin == rmax;   // a layer without hits is trivially uniform
        li.lo = 1;
        li.hi = 0;
        li.r_bits = rmin;
        li.nvote = 0;
        li.pad[0] = li.pad[1] = 0;
        const int dirty = li.present && li.uniform && !(w.memo->valid[l] && w.memo->r_bits[l] == rmin);
        if (li.present && li.uniform) {
            if (dirty) {
                if (ax.n_d0) {   // every slice has its own rows; the table marks those that vote
                    li.lo = 0;
                    li.hi = ax.n_qpt - 1;
                } else {
                    row_range(ax, sagitta_coef(ax, (double)__uint_as_float(rmin)), &li.lo, &li.hi);
                }
                w.memo->r_bits[l] = rmin;
                w.memo->lo[l] = li.lo;
                w.memo->hi[l] = li.hi;
                w.memo->valid[l] = 1;
            } else {
                li.lo = w.memo->lo[l];   // the same radius as before: its rows are memoised
                li.hi = w.memo->hi[l];
                li.nvote = w.memo->nvote[l];
            }
        }
        w.info[l] = li;
        w.memo->dirty[l] = dirty;
        s_li = li;
        s_dirty = dirty;
    }
    __syncthreads();
    if (!s_dirty) return;
    __shared__ int s_nvote;
    if (threadIdx.x == 0) s_nvote = 0;
    __syncthreads();
    const LayerInfo li = s_li;
    const double r = (double)__uint_as_float(li.r_bits);
    const double t0 = __dadd_rn(ax.cot_min, __dmul_rn(0.5, ax.dt));
    int nvote = 0;
    for (int i = threadIdx.x; i < ax.n_qpt; i += blockDim.x) {
        const int q = l * ax.n_qpt + i;
        TabEntry te;
        te.I = kNoVote;
        te.g = 0.f;
        double s = 0.0;
        if (i >= li.lo && i <= li.hi) {
            const double x = __dmul_rn(sagitta_coef(ax, r), qpt_centre(ax, i));
            const double d0 = d0_centre(ax, i);
            double y = 2.0;
            if (track_sin(r, x, d0, &y) && fabs(y) <= 1.0) {
                const double T = __dmul_rn(__dmul_rn((double)ax.n_phi, asin(y)), kInvTwoPi);
                const double fI = floor(T);
                te.I = (int32_t)fI;
                te.g = (float)(T - fI);
                if (te.g >= 1.0f) {
                    te.I += 1;
                    te.g = 0.f;
                }
                s = track_arc(r, x, d0, y);
                ++nvote;
            }
        }
        w.tab[q] = te;
        w.arc[q] = s;
        if (w.zco) {
            // stage-2 terms of the layer's members on this row: the z0 coordinate of cot row m is
            // zscale (z - z0_min) - S - m B with S = zscale s t_0 and B = zscale s dt
            const double S = __dmul_rn(ax.zscale, __dmul_rn(s, t0));
            const double B = __dmul_rn(ax.zscale, __dmul_rn(s, ax.dt));
            const float sh = (float)S, bh = (float)B;
            w.zco[q] = make_float4(sh, (float)(S - (double)sh), bh, (float)(B - (double)bh));
        }
    }
    if (nvote) atomicAdd(&s_nvote, nvote);
    __syncthreads();
    if (threadIdx.x == 0) {
        w.info[l].nvote = s_nvote;
        w.memo->nvote[l] = s_nvote;
    }
}

// One CTA per event: exclusive scan of the bucket sizes, kScanRound counts per round.  The counts
// are loaded and the offsets stored coalesced through a shared tile; in between each thread scans
// kScanPerThread consecutive entries in registers and the CTA scans the threads' totals (one
// shuffle scan per warp, one over the warps).  The tile has one padding word per 32, which keeps
// the per-thread reads of consecutive words free of bank conflicts.
constexpr int kScanPerThread = 8;
constexpr int kScanRound = kScanThreads * kScanPerThread;

__device__ __forceinline__ int scan_pad(int k) { return k + (k >> 5); }

// Exclusive scan of counts[k0, k1) into offs[k0, k1), starting from `carry`; returns the running
// total after k1.  Every thread of the CTA takes part.
__device__ __forceinline__ int scan_range(const int32_t *counts, int32_t *offs, const int k0, const int k1, int carry)
{
    __shared__ int s_tile[kScanRound + kScanRound / 32];
    __shared__ int s_warp[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = k0; base < k1; base += kScanRound) {
        const int n = min(kScanRound, k1 - base);
#pragma unroll
        for (int r = 0; r < kScanPerThread; ++r) {
            const int k = r * kScanThreads + threadIdx.x;
            s_tile[scan_pad(k)] = k < n ? counts[base + k] : 0;
        }
        __syncthreads();
        const int k0 = threadIdx.x * kScanPerThread;
        int v[kScanPerThread];
        int sum = 0;
#pragma unroll
        for (int q = 0; q < kScanPerThread; ++q) {
            v[q] = s_tile[scan_pad(k0 + q)];
            sum += v[q];
        }
        int incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int x = s_warp[lane];
            int wi = x;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(0xFFFFFFFFu, wi, d);
                if (lane >= d) wi += t;
            }
            s_warp[lane] = wi;   // inclusive over warps
        }
        __syncthreads();
        int run = carry + (warp > 0 ? s_warp[warp - 1] : 0) + incl - sum;
#pragma unroll
        for (int q = 0; q < kScanPerThread; ++q) {
            s_tile[scan_pad(k0 + q)] = run;
            run += v[q];
        }
        carry += s_warp[kScanThreads / 32 - 1];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kScanPerThread; ++r) {
            const int k = r * kScanThreads + threadIdx.x;
            if (k < n) offs[base + k] = s_tile[scan_pad(k)];
        }
        __syncthreads();
    }
    return carry;
}

// One CTA per event: the scan of all its keys.
__device__ __forceinline__ void scan_keys(const Axes &ax, const Workspace &w, const int e)
{
    const int nkeys = n_keys(ax);
    const int total = scan_range(w.counts + (int64_t)e * nkeys, w.offs + (int64_t)e * (nkeys + 1), 0, nkeys, 0);
    if (threadIdx.x == 0) {
        w.offs[(int64_t)e * (nkeys + 1) + nkeys] = total;
        w.stats[e].n_hits = (unsigned long long)total;
    }
}

// One CTA per (event, layer) for events with few CTAs to spread over: the CTA first sums the
// event's counts of the layers before its own (its offset), then scans its layer's buckets, so the
// layers of an event are scanned side by side instead of one after another.  Integer sums: the
// same offsets as scan_keys.
__device__ __forceinline__ void scan_layer(const Axes &ax, const Workspace &w, const int e, const int l)
{
    __shared__ int s_part[kScanThreads / 32];
    const int nkeys = n_keys(ax), nphi = ax.n_phi;
    const int32_t *counts = w.counts + (int64_t)e * nkeys;
    int32_t *offs = w.offs + (int64_t)e * (nkeys + 1);
    int part = 0;
    for (int k = threadIdx.x; k < l * nphi; k += kScanThreads) part += counts[k];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, d);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    int base = 0;
#pragma unroll
    for (int q = 0; q < kScanThreads / 32; ++q) base += s_part[q];
    const int total = scan_range(counts, offs, l * nphi, (l + 1) * nphi, base);
    if (threadIdx.x == 0 && l == ax.n_layers - 1) {
        offs[nkeys] = total;
        w.stats[e].n_hits = (unsigned long long)total;
    }
}

// The layer tables and the bucket scans in one launch, as they do not depend on each other: the
// first `scans` blocks scan the events' bucket counts (one block per event, or with `by_layer` one
// per (event, layer)), the next HOUGH_MAX_LAYERS blocks compute one layer's table each.
__global__ void __launch_bounds__(kScanThreads) table_scan_kernel(Axes ax, Workspace w, int by_layer)
{
    pdl_enter();
    const int scans = by_layer ? w.n_events * ax.n_layers : w.n_events;
    const int b = blockIdx.x;
    if (b >= scans) layer_table(ax, w, b - scans);
    else if (by_layer) scan_layer(ax, w, b / ax.n_layers, b % ax.n_layers);
    else scan_keys(ax, w, b);
}

// Scatter every valid hit to its sorted position, completing its hot record with its voting rows.
__global__ void __launch_bounds__(kStageThreads) scatter_kernel(Axes ax, Workspace w)
{
    pdl_enter();
    const int nkeys = n_keys(ax);
    // the votes of layers of one radius: the layer's hits times its voting rows, per event
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)w.n_events * ax.n_layers;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t / ax.n_layers), l = (int)(t - (int64_t)e * ax.n_layers);
        const LayerInfo li = w.info[l];
        if (li.present && li.uniform && li.nvote > 0) {
            const int32_t *offs = w.offs + (int64_t)e * (nkeys + 1);
            const long long n_l = offs[(l + 1) * ax.n_phi] - offs[l * ax.n_phi];
            if (n_l) atomicAdd(&w.stats[e].votes_by_layer[l], (unsigned long long)(n_l * li.nvote));
        }
    }
    if (w.recycle) {
        // the bucket counts are read for the last time by the scan, which this kernel follows
        uint4 *c4 = reinterpret_cast<uint4 *>(w.counts);
        const int64_t n4 = (int64_t)w.n_events * nkeys / 4;
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x)
            c4[q] = make_uint4(0u, 0u, 0u, 0u);
        for (int64_t q = n4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)w.n_events * nkeys;
             q += (int64_t)gridDim.x * blockDim.x)
            w.counts[q] = 0;
    }
    const int64_t total = hit_total(w);
    const HitInputs in = hit_inputs(w);
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < total;
         h += (int64_t)gridDim.x * blockDim.x) {
        const int k = w.key[h];
        if (k < 0) continue;
        const int e = event_of(w.hit_start, w.n_events, h);
        const int64_t start = w.hit_start[e];
        const int64_t pos = start + w.offs[(int64_t)e * (nkeys + 1) + k] + w.rank[h];
        HotHit hh = w.hot_tmp[h];
        if (w.fsort) w.fsort[pos] = hh.f;
        const int l = (hh.jl >> 16) & 0xF;
        const LayerInfo li = w.info[l];
        int lo = li.lo, hi = li.hi;
        const float rr = in.r[h];
        if (!li.uniform && ax.n_d0) {
            // every row may hold a vote; the vote kernels decide each in FP64
            lo = 0;
            hi = ax.n_qpt - 1;
            const double c = sagitta_coef(ax, (double)rr);
            unsigned long long nv = 0;
            for (int row = 0; row < ax.n_qpt; ++row) {
                double y = 2.0;
                if (track_sin((double)rr, __dmul_rn(c, qpt_centre(ax, row)), d0_centre(ax, row), &y) && fabs(y) <= 1.0)
                    ++nv;
            }
            if (nv) atomicAdd(&w.stats[e].votes_by_layer[l], nv);
        } else if (!li.uniform) {
            row_range(ax, sagitta_coef(ax, (double)rr), &lo, &hi);
            if (hi >= lo)
                atomicAdd(&w.stats[e].votes_by_layer[l], (unsigned long long)(hi - lo + 1));
        }
        if (hi < lo) { lo = 1; hi = 0; }
        hh.rows = (uint32_t)lo | ((uint32_t)hi << 16);
        w.hot[pos] = hh;
        ColdHit ch;
        ch.r = rr;
        ch.phi = in.phi[h];
        ch.z = in.z[h];
        ch.idx = (int32_t)(h - start);
        w.cold[pos] = ch;
        if (w.zsort) w.zsort[pos] = ch.z;
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65535LL * 16) g = 65535LL * 16;
    return (int)g;
}

}  // namespace

cudaError_t launch_stage(const Axes &ax, const Workspace &w, cudaStream_t stream, cudaEvent_t *after, bool clear)
{
    const int nkeys = n_keys(ax);
    ClearList cl{};
    auto add = [&](void *p, size_t bytes, uint32_t value) {
        cl.p[cl.n] = static_cast<uint32_t *>(p);
        cl.words[cl.n] = (long long)(bytes / 4);
        cl.value[cl.n] = value;
        ++cl.n;
    };
    add(w.counts, sizeof(int32_t) * (size_t)w.n_events * nkeys, 0u);
    if (w.prof) add(w.prof, sizeof(uint2) * (size_t)w.n_events * prof_event_entries(ax), 0u);
    add(w.stats, sizeof(DevStats) * (size_t)w.n_events, 0u);
    if (w.counters) add(w.counters, sizeof(BatchCounters), 0u);
    add(w.radii->rmin, sizeof(w.radii->rmin), 0xFFFFFFFFu);
    add(w.radii->rmax, sizeof(w.radii->rmax), 0u);
    long long vec_words = 0;
    for (int q = 0; q < cl.n; ++q) vec_words += cl.words[q] / 4 + 1;
    const int clear_grid = (int)std::min<long long>(2048, (vec_words + kClearThreads - 1) / kClearThreads);
    cudaError_t err;
    auto mark = [&](int k) { return after ? cudaEventRecord(after[k], stream) : cudaSuccess; };
    if (clear && (err = launch_chained(clear_kernel, dim3(std::max(1, clear_grid)), dim3(kClearThreads), 0, stream, cl)))
        return err;
    if ((err = mark(0))) return err;
    const int g = grid_for(w.n_hits_total >= 0 ? w.n_hits_total : w.hit_capacity, kStageThreads);
    if ((err = launch_chained(stage_count_kernel, dim3(g), dim3(kStageThreads), 0, stream, ax, w))) return err;
    if ((err = mark(1))) return err;
    // a few events leave most SMs idle under one scan block each: then a block per (event, layer)
    const int by_layer = w.n_events <= 16 ? 1 : 0;
    const int scans = by_layer ? w.n_events * ax.n_layers : w.n_events;
    if ((err = launch_chained(table_scan_kernel, dim3(scans + HOUGH_MAX_LAYERS), dim3(kScanThreads), 0, stream, ax, w,
                              by_layer)))
        return err;
    if ((err = mark(2))) return err;   // table_ms covers both; scan_ms stays empty
    if ((err = mark(3))) return err;
    return launch_chained(scatter_kernel, dim3(g), dim3(kStageThreads), 0, stream, ax, w);
}

}  // namespace hough
