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
#include "hough_internal.cuh"

namespace hough {

namespace {

constexpr int kStageThreads = 256;
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kStageThreads) stage_count_kernel(Axes ax, Workspace w)
{
    __shared__ unsigned int s_rmin[HOUGH_MAX_LAYERS], s_rmax[HOUGH_MAX_LAYERS];
    if (threadIdx.x < HOUGH_MAX_LAYERS) {
        s_rmin[threadIdx.x] = 0xFFFFFFFFu;
        s_rmax[threadIdx.x] = 0u;
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
        // bin coordinate of the hit's own azimuth: u_h = Nphi (phi + pi) / (2 pi) = J + f
        const double uh = __dmul_rn(__dmul_rn((double)ax.n_phi, __dadd_rn((double)ph, kPi)), kInvTwoPi);
        const double fl = floor(uh);
        long long J = (long long)fl % ax.n_phi;
        if (J < 0) J += ax.n_phi;
        float f = (float)(uh - fl);
        if (f >= 1.0f) {   // the fraction rounded up to 1: carry into J
            f = 0.0f;
            J = (J + 1 == ax.n_phi) ? 0 : J + 1;
        }
        const int k = l * ax.n_phi + (int)J;
        w.key[h] = k;
        w.rank[h] = atomicAdd(&w.counts[(int64_t)e * nkeys + k], 1);
        // bucket extrema of f as ordered bit patterns (f >= 0): .x of bucket J keeps the maximum
        // (offset by one so an empty bucket, 0, is below every hit), .y of bucket J-1 keeps the
        // maximum of the complement, i.e. the minimum of bucket J
        if (w.prof) {
            uint2 *prof = w.prof + (int64_t)e * prof_event_entries(ax) + (int64_t)l * prof_stride(ax);
            const int Jm = J == 0 ? ax.n_phi - 1 : (int)J - 1;
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
        atomicMin(&s_rmin[l], __float_as_uint(rr));
        atomicMax(&s_rmax[l], __float_as_uint(rr));
    }
    __syncthreads();
    if (threadIdx.x < HOUGH_MAX_LAYERS && s_rmax[threadIdx.x] != 0u) {
        atomicMin(&w.radii->rmin[threadIdx.x], s_rmin[threadIdx.x]);
        atomicMax(&w.radii->rmax[threadIdx.x], s_rmax[threadIdx.x]);
    }
}

// One warp: per layer, whether all its hits share one radius, that radius's voting rows,
// and whether the memoised table rows must be recomputed.
__global__ void layer_info_kernel(Axes ax, Workspace w)
{
    const int l = threadIdx.x;
    if (l >= HOUGH_MAX_LAYERS) return;
    LayerInfo li;
    const unsigned rmin = w.radii->rmin[l], rmax = w.radii->rmax[l];
    li.present = (l < ax.n_layers) && rmax != 0u;
    li.uniform = !li.present || rmin == rmax;   // a layer without hits is trivially uniform
    li.lo = 1;
    li.hi = 0;
    li.r_bits = rmin;
    li.pad[0] = li.pad[1] = li.pad[2] = 0;
    const int dirty = li.present && li.uniform && !(w.memo->valid[l] && w.memo->r_bits[l] == rmin);
    if (li.present && li.uniform) {
        if (dirty) {
            row_range(ax, sagitta_coef(ax, (double)__uint_as_float(rmin)), &li.lo, &li.hi);
            w.memo->r_bits[l] = rmin;
            w.memo->lo[l] = li.lo;
            w.memo->hi[l] = li.hi;
            w.memo->valid[l] = 1;
        } else {
            li.lo = w.memo->lo[l];   // the same radius as before: its rows are memoised
            li.hi = w.memo->hi[l];
        }
    }
    w.info[l] = li;
    w.memo->dirty[l] = dirty;
}

// Per (layer, row) of a uniform layer whose radius changed: T = Nphi asin(x) / (2 pi) split into
// I + g, and the arc length s = r asin(|x|) / |x| for stage 2.
__global__ void table_kernel(Axes ax, Workspace w)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= ax.n_layers * ax.n_qpt) return;
    const int l = q / ax.n_qpt, i = q % ax.n_qpt;
    if (!w.memo->dirty[l]) return;
    const LayerInfo li = w.info[l];
    TabEntry te;
    te.I = 0;
    te.g = 0.f;
    double s = 0.0;
    if (i >= li.lo && i <= li.hi) {
        const double r = (double)__uint_as_float(li.r_bits);
        const double x = __dmul_rn(sagitta_coef(ax, r), qpt_centre(ax, i));
        const double T = __dmul_rn(__dmul_rn((double)ax.n_phi, asin(x)), kInvTwoPi);
        const double fI = floor(T);
        te.I = (int32_t)fI;
        te.g = (float)(T - fI);
        if (te.g >= 1.0f) {
            te.I += 1;
            te.g = 0.f;
        }
        const double axv = fabs(x);
        s = axv > 0.0 ? __ddiv_rn(__dmul_rn(r, asin(axv)), axv) : r;
    }
    w.tab[q] = te;
    w.arc[q] = s;
    if (w.zco) {
        // stage-2 terms of the layer's members on this row: the z0 coordinate of cot row m is
        // zscale (z - z0_min) - S - m B with S = zscale s t_0 and B = zscale s dt
        const double t0 = __dadd_rn(ax.cot_min, __dmul_rn(0.5, ax.dt));
        const double S = __dmul_rn(ax.zscale, __dmul_rn(s, t0));
        const double B = __dmul_rn(ax.zscale, __dmul_rn(s, ax.dt));
        const float sh = (float)S, bh = (float)B;
        w.zco[q] = make_float4(sh, (float)(S - (double)sh), bh, (float)(B - (double)bh));
    }
}

// One CTA per event: exclusive scan of the bucket sizes, in tiles of kScanTile counts staged
// through shared memory with coalesced loads and stores; each warp scans 32 consecutive counts
// per round with shuffles (no bank conflicts).  Then the vote count of uniform layers.
constexpr int kScanRounds = 8;
constexpr int kScanTile = kScanThreads * kScanRounds;

__global__ void __launch_bounds__(kScanThreads) scan_keys_kernel(Axes ax, Workspace w)
{
    __shared__ int s_tile[kScanTile];
    __shared__ int s_warp[kScanThreads / 32];
    __shared__ int s_total;
    const int e = blockIdx.x;
    const int nkeys = n_keys(ax);
    const int32_t *counts = w.counts + (int64_t)e * nkeys;
    int32_t *offs = w.offs + (int64_t)e * (nkeys + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int carry = 0;
    for (int base = 0; base < nkeys; base += kScanTile) {
        const int n = min(kScanTile, nkeys - base);
#pragma unroll
        for (int r = 0; r < kScanRounds; ++r) {
            const int k = r * kScanThreads + threadIdx.x;
            s_tile[k] = k < n ? counts[base + k] : 0;
        }
        __syncthreads();
        // warp w owns entries [w * 32 * kScanRounds, (w + 1) * 32 * kScanRounds)
        int run = 0;
#pragma unroll
        for (int r = 0; r < kScanRounds; ++r) {
            const int k = warp * 32 * kScanRounds + r * 32 + lane;
            const int v = s_tile[k];
            int incl = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
                if (lane >= d) incl += t;
            }
            s_tile[k] = run + incl - v;
            run += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
        if (lane == 0) s_warp[warp] = run;
        __syncthreads();
        if (warp == 0) {
            const int v = s_warp[lane];
            int incl = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
                if (lane >= d) incl += t;
            }
            s_warp[lane] = incl - v;   // exclusive over warps
            if (lane == 31) s_total = incl;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kScanRounds; ++r) {
            const int k = r * kScanThreads + threadIdx.x;
            if (k < n) offs[base + k] = carry + s_warp[k / (32 * kScanRounds)] + s_tile[k];
        }
        carry += s_total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        offs[nkeys] = carry;
        w.stats[e].n_hits = (unsigned long long)carry;
    }
    __syncthreads();
    if (threadIdx.x < ax.n_layers) {
        const int l = threadIdx.x;
        const LayerInfo li = w.info[l];
        if (li.present && li.uniform && li.hi >= li.lo) {
            const long long n_l = offs[(l + 1) * ax.n_phi] - offs[l * ax.n_phi];
            w.stats[e].votes_by_layer[l] += (unsigned long long)(n_l * (li.hi - li.lo + 1));
        }
    }
}

// Scatter every valid hit to its sorted position, completing its hot record with its voting rows.
__global__ void __launch_bounds__(kStageThreads) scatter_kernel(Axes ax, Workspace w)
{
    const int nkeys = n_keys(ax);
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
        const int l = (hh.jl >> 16) & 0xF;
        const LayerInfo li = w.info[l];
        int lo = li.lo, hi = li.hi;
        const float rr = in.r[h];
        if (!li.uniform) {
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

cudaError_t launch_stage(const Axes &ax, const Workspace &w, cudaStream_t stream)
{
    const int nkeys = n_keys(ax);
    cudaError_t err;
    if ((err = cudaMemsetAsync(w.counts, 0, sizeof(int32_t) * (size_t)w.n_events * nkeys, stream))) return err;
    if (w.prof && (err = cudaMemsetAsync(w.prof, 0, sizeof(uint2) * (size_t)w.n_events * prof_event_entries(ax), stream)))
        return err;
    if ((err = cudaMemsetAsync(w.stats, 0, sizeof(DevStats) * (size_t)w.n_events, stream))) return err;
    if (w.counters && (err = cudaMemsetAsync(w.counters, 0, sizeof(BatchCounters), stream))) return err;
    if ((err = cudaMemsetAsync(w.radii->rmin, 0xFF, sizeof(w.radii->rmin), stream))) return err;
    if ((err = cudaMemsetAsync(w.radii->rmax, 0, sizeof(w.radii->rmax), stream))) return err;
    const int g = grid_for(w.n_hits_total >= 0 ? w.n_hits_total : w.hit_capacity, kStageThreads);
    stage_count_kernel<<<g, kStageThreads, 0, stream>>>(ax, w);
    layer_info_kernel<<<1, 32, 0, stream>>>(ax, w);
    const int nt = ax.n_layers * ax.n_qpt;
    table_kernel<<<(nt + 127) / 128, 128, 0, stream>>>(ax, w);
    scan_keys_kernel<<<w.n_events, kScanThreads, 0, stream>>>(ax, w);
    scatter_kernel<<<g, kStageThreads, 0, stream>>>(ax, w);
    return cudaGetLastError();
}

}  // namespace hough
