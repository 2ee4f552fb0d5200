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

// The state a counting CTA starts from: its radius ranges, and (with recycling, block 0) the next
// event's counters and radius ranges.  The caller synchronises the CTA afterwards.
__device__ __forceinline__ void count_prologue(const Workspace &w, unsigned *s_rmin, unsigned *s_rmax)
{
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
}

// Hit h of event e: validation, its key (layer, azimuth bucket) and rank within the bucket, the
// bucket's extrema of f, its hot record in input order, and the CTA's radius range of its layer.
__device__ __forceinline__ void count_hit(const Axes &ax, const Workspace &w, const HitInputs &in, float cscale,
                                          int nkeys, int64_t h, int e, unsigned *s_rmin, unsigned *s_rmax)
{
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
        return;
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

// The CTA's radius ranges into the event's (after a CTA barrier).
__device__ __forceinline__ void count_epilogue(const Workspace &w, const unsigned *s_rmin, const unsigned *s_rmax)
{
    if (threadIdx.x < HOUGH_MAX_LAYERS && s_rmax[threadIdx.x] != 0u) {
        atomicMin(&w.radii->rmin[threadIdx.x], s_rmin[threadIdx.x]);
        atomicMax(&w.radii->rmax[threadIdx.x], s_rmax[threadIdx.x]);
    }
}

__global__ void __launch_bounds__(kStageThreads) stage_count_kernel(Axes ax, Workspace w)
{
    pdl_enter();
    __shared__ unsigned int s_rmin[HOUGH_MAX_LAYERS], s_rmax[HOUGH_MAX_LAYERS];
    count_prologue(w, s_rmin, s_rmax);
    __syncthreads();
    const int nkeys = n_keys(ax);
    // FP32 sagitta coefficient of the per-vote path; its rounding is covered by the refine window
    const float cscale = (float)(0.15 * ax.b / 100.0);
    const int64_t total = hit_total(w);
    const HitInputs in = hit_inputs(w);
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < total; h += (int64_t)gridDim.x * blockDim.x)
        count_hit(ax, w, in, cscale, nkeys, h, event_of(w.hit_start, w.n_events, h), s_rmin, s_rmax);
    __syncthreads();
    count_epilogue(w, s_rmin, s_rmax);
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
        // every load of the decision at once (one round trip, not a chain of them)
        const unsigned rmin = w.radii->rmin[l], rmax = w.radii->rmax[l];
        const int m_valid = w.memo->valid[l], m_lo = w.memo->lo[l], m_hi = w.memo->hi[l], m_nvote = w.memo->nvote[l];
        const unsigned m_r = w.memo->r_bits[l];
        li.present = (l < ax.n_layers) && rmax != 0u;
        li.uniform = !li.present || rmin == rmax;   // a layer without hits is trivially uniform
        li.lo = 1;
        li.hi = 0;
        li.r_bits = rmin;
        li.nvote = 0;
        li.pad[0] = li.pad[1] = 0;
        const int dirty = li.present && li.uniform && !(m_valid && m_r == rmin);
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
                li.lo = m_lo;   // the same radius as before: its rows are memoised
                li.hi = m_hi;
                li.nvote = m_nvote;
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
        int cv[kScanPerThread];   // every load in flight before the first store
#pragma unroll
        for (int r = 0; r < kScanPerThread; ++r) {
            const int k = r * kScanThreads + threadIdx.x;
            cv[r] = k < n ? counts[base + k] : 0;
        }
#pragma unroll
        for (int r = 0; r < kScanPerThread; ++r) s_tile[scan_pad(r * kScanThreads + threadIdx.x)] = cv[r];
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
    // the counts of the layers before: 16-byte loads, eight in flight per thread (one round trip
    // for most grids, where a sum of dependent loads would take one per element)
    int part = 0;
    const int4 *c4 = reinterpret_cast<const int4 *>(counts);   // n_phi is a multiple of 64
    const int n4 = l * nphi / 4;
    for (int base = 0; base < n4; base += 8 * kScanThreads) {
        int4 v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int q = base + r * kScanThreads + threadIdx.x;
            v[r] = q < n4 ? c4[q] : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) part += (v[r].x + v[r].y) + (v[r].z + v[r].w);
    }
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

// The votes of layers of one radius, per event: the layer's hits times its voting rows (thread t of
// `nthreads` takes (event, layer) pairs t, t + nthreads, ...).  offs_of(e) is the event's offsets.
template <typename Offs>
__device__ __forceinline__ void count_table_votes(const Axes &ax, const Workspace &w, int64_t t0, int64_t nthreads,
                                                  Offs offs_of)
{
    for (int64_t t = t0; t < (int64_t)w.n_events * ax.n_layers; t += nthreads) {
        const int e = (int)(t / ax.n_layers), l = (int)(t - (int64_t)e * ax.n_layers);
        const LayerInfo li = w.info[l];
        if (li.present && li.uniform && li.nvote > 0) {
            const long long n_l = offs_of(e, (l + 1) * ax.n_phi) - offs_of(e, l * ax.n_phi);
            if (n_l) atomicAdd(&w.stats[e].votes_by_layer[l], (unsigned long long)(n_l * li.nvote));
        }
    }
}

// The bucket counts zeroed for the next event (recycling), by thread t0 of nthreads: the scan has
// read them for the last time.
__device__ __forceinline__ void recycle_counts(const Axes &ax, const Workspace &w, int64_t t0, int64_t nthreads)
{
    const int64_t n = (int64_t)w.n_events * n_keys(ax);
    uint4 *c4 = reinterpret_cast<uint4 *>(w.counts);
    for (int64_t q = t0; q < n / 4; q += nthreads) c4[q] = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t q = n / 4 * 4 + t0; q < n; q += nthreads) w.counts[q] = 0;
}

// Valid hit h (input index; event start `start`) to its sorted position pos: its f, hot record hh
// completed with its voting rows, cold record (r, phi, z) and z.
__device__ __forceinline__ void sort_hit(const Axes &ax, const Workspace &w, int64_t h, int e, int64_t start,
                                         int64_t pos, HotHit hh, float rr, float ph, float zz)
{
    if (w.fsort) w.fsort[pos] = hh.f;
    const int l = (hh.jl >> 16) & 0xF;
    const LayerInfo li = w.info[l];
    int lo = li.lo, hi = li.hi;
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
    ch.phi = ph;
    ch.z = zz;
    ch.idx = (int32_t)(h - start);
    w.cold[pos] = ch;
    if (w.zsort) w.zsort[pos] = ch.z;
}

// Scatter every valid hit to its sorted position, completing its hot record with its voting rows.
__global__ void __launch_bounds__(kStageThreads) hit_sort_kernel(Axes ax, Workspace w)
{
    const int nkeys = n_keys(ax);
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    const int64_t total = hit_total(w);
    const HitInputs in = hit_inputs(w);
    // The thread's first hit's own inputs -- its key, rank and record from the counting kernel,
    // which finished before this grid could launch, and its coordinates -- are requested before
    // waiting on the table and scan kernel, whose bucket offsets and layer records come after.
    int k = -1, rank = 0;
    HotHit hh{};
    float rr = 0.f, ph = 0.f, zz = 0.f;
    if (t0 < total) {
        k = w.key[t0];
        rank = w.rank[t0];
        hh = w.hot_tmp[t0];
        rr = in.r[t0];
        ph = in.phi[t0];
        zz = in.z[t0];
    }
    pdl_enter();
    // this thread's first (event, layer) pair of the one-radius vote counts: its inputs requested
    // now, counted after the hits, so the loads overlap the hits' own
    const int64_t npairs = (int64_t)w.n_events * ax.n_layers;
    LayerInfo tli{};
    int tn = 0, te = 0, tl = 0;
    if (t0 < npairs) {
        te = (int)(t0 / ax.n_layers);
        tl = (int)(t0 - (int64_t)te * ax.n_layers);
        tli = w.info[tl];
        const int32_t *o = w.offs + (int64_t)te * (nkeys + 1);
        tn = o[(tl + 1) * ax.n_phi] - o[tl * ax.n_phi];
    }
    for (int64_t h = t0; h < total; h += nt) {
        // every load that does not depend on another first, then the bucket offset and layer
        // record that do
        if (h != t0) {
            k = w.key[h];
            rank = w.rank[h];
            hh = w.hot_tmp[h];
            rr = in.r[h];
            ph = in.phi[h];
            zz = in.z[h];
        }
        const int e = event_of(w.hit_start, w.n_events, h);
        const int64_t start = w.hit_start[e];
        if (k >= 0) sort_hit(ax, w, h, e, start, start + w.offs[(int64_t)e * (nkeys + 1) + k] + rank, hh, rr, ph, zz);
    }
    if (t0 < npairs && tli.present && tli.uniform && tli.nvote > 0 && tn)
        atomicAdd(&w.stats[te].votes_by_layer[tl], (unsigned long long)tn * (unsigned long long)tli.nvote);
    count_table_votes(ax, w, t0 + nt, nt, [&](int e, int k) { return w.offs[(int64_t)e * (nkeys + 1) + k]; });
    if (w.recycle) recycle_counts(ax, w, t0, nt);
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
    return launch_chained(hit_sort_kernel, dim3(g), dim3(kStageThreads), 0, stream, ax, w);
}

}  // namespace hough
