// Stage-1 vote (Sec. 4, first step; the A[B[i]] += 1 scatter of Sec. 8) with the paper's GPU
// remedy for it: every update goes to an accumulator tile in on-chip shared memory with shared
// atomics (Sec. 6.1), and the tile reaches HBM once, with coalesced 16-byte stores and no
// separate clearing pass.
//
// Work decomposition: one CTA per (event, tile) where a tile is tile_qpt rows of q/pT by
// tile_phi columns of phi0.  The CTA reads only the hits that can vote into its tile -- per
// layer a contiguous range (two when it wraps) of the (layer, phi bin)-sorted hits -- lane by
// lane, and loops over the tile's rows in lockstep, so that at each row the 32 lanes of a warp
// (hits of one layer, sorted by azimuth) vote into neighbouring cells of one row.  A lane whose
// (word, bits) equals its left neighbour's skips its atomic: sorted hits of one layer often
// land in the same cell.
//
// Per-vote arithmetic.  For a layer whose hits share one radius the table gives
// Nphi asin(x_i) / (2 pi) = I + g exactly (FP64, rounded once to FP32 in g), the hit carries its
// own bin coordinate as J + f, and the vote's bin is J - I - (f < g): no transcendental and an
// error below 1e-7 bin.  Other layers take FP32 asinf per vote; a vote whose FP32 bin coordinate
// lies within `refine_eps` of an edge, or whose |x| > kRefineXLim, is recomputed in FP64 from the
// hit's coordinates exactly as the definition reads.
#include "hough_internal.cuh"

namespace hough {

namespace {

struct VoteParams {
    Axes ax;
    Workspace w;
    int R, W, n_spans, tiles_per_event;
    float s32;          // Nphi / (2 pi) in FP32
    float refine_eps;
};

constexpr int kMaxRanges = 2 * HOUGH_MAX_LAYERS;

template <int TPB>
__global__ void __launch_bounds__(TPB) vote_kernel(VoteParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_start[kMaxRanges];
    __shared__ int s_pre[kMaxRanges + 1];
    __shared__ unsigned long long s_refined;
    __shared__ unsigned s_umask;

    const Axes &ax = p.ax;
    const int R = p.R, W = p.W, Wh = W >> 1, L = ax.n_layers, nphi = ax.n_phi;
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem_raw);
    TabEntry *tab = reinterpret_cast<TabEntry *>(tile + R * Wh);
    float *kq = reinterpret_cast<float *>(tab + L * R);

    const int e = blockIdx.x / p.tiles_per_event;
    const int t = blockIdx.x - e * p.tiles_per_event;
    const int slab = t / p.n_spans, span = t - slab * p.n_spans;
    const int i0 = slab * R;
    const int nrows = min(R, ax.n_qpt - i0);
    const int J0 = span * W;
    const int nkeys = L * nphi;
    const int64_t hstart = p.w.hit_start[e];
    const HotHit *hot = p.w.hot + hstart;
    const ColdHit *cold = p.w.cold + hstart;
    const int32_t *offs = p.w.offs + (int64_t)e * (nkeys + 1);

    // layers whose hits share one radius take the table path
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        const unsigned u = __ballot_sync(0xFFFFFFFFu, l < L && p.w.info[l < HOUGH_MAX_LAYERS ? l : 0].uniform);
        if (l == 0) {
            s_umask = u;
            s_refined = 0ull;
        }
    }
    __syncthreads();
    const unsigned umask = s_umask;

    // clear the tile; stage this slab's table rows and FP32 q/pT centres
    uint4 *tile4 = reinterpret_cast<uint4 *>(tile);
    for (int q = threadIdx.x; q < (R * Wh) >> 2; q += TPB) tile4[q] = make_uint4(0u, 0u, 0u, 0u);
    for (int q = threadIdx.x; q < L * R; q += TPB) {
        const int l = q / R, rr = q - l * R;
        TabEntry te;
        te.I = 0;
        te.g = 0.f;
        if (rr < nrows && ((umask >> l) & 1u)) te = p.w.tab[l * ax.n_qpt + i0 + rr];
        tab[q] = te;
    }
    for (int q = threadIdx.x; q < R; q += TPB) kq[q] = q < nrows ? p.w.kq32[i0 + q] : 0.f;

    // per layer, the hits that can vote into this tile: a cyclic range of phi bins J
    if (threadIdx.x < HOUGH_MAX_LAYERS) {
        const int l = threadIdx.x;
        int nr = 0, st[2] = {0, 0}, ln[2] = {0, 0};
        if (l < L) {
            const int lstart = offs[l * nphi], lend = offs[(l + 1) * nphi];
            int ja = 0, jb = -1;   // inclusive J window, possibly beyond [0, nphi)
            bool all = false, none = lend == lstart;
            if (!none && ((umask >> l) & 1u)) {
                const LayerInfo li = p.w.info[l];
                const int a = max(i0, li.lo), b = min(i0 + nrows - 1, li.hi);
                if (a > b) {
                    none = true;
                } else {
                    // vote bin J - I - (f < g) lies in [J0, J0 + W) only for J in [J0 + I_a, J0 + W + I_b]
                    const TabEntry ta = p.w.tab[l * ax.n_qpt + a], tb = p.w.tab[l * ax.n_qpt + b];
                    ja = J0 + ta.I;
                    jb = J0 + W + tb.I;
                }
            } else if (!none) {
                // per-vote layer: bound asin(c k) over the layer's radius range and the slab's rows
                const float c_lo = 0.15f * (float)ax.b / 100.f * __uint_as_float(p.w.radii->rmin[l]);
                const float c_hi = 0.15f * (float)ax.b / 100.f * __uint_as_float(p.w.radii->rmax[l]);
                const float k_a = p.w.kq32[i0], k_b = p.w.kq32[i0 + nrows - 1];
                float amin = 2.f, amax = -2.f;
                const float cs[2] = {c_lo * 0.999f, c_hi * 1.001f};
                const float ks[2] = {k_a, k_b};
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int v = 0; v < 2; ++v) {
                        const float a = asinf(fminf(fmaxf(cs[u] * ks[v], -1.f), 1.f));
                        amin = fminf(amin, a);
                        amax = fmaxf(amax, a);
                    }
                ja = (int)floorf(J0 + p.s32 * amin) - 2;
                jb = (int)floorf(J0 + W + p.s32 * amax) + 2;
            }
            if (!none) {
                if (jb - ja + 1 >= nphi) all = true;
                if (all) {
                    nr = 1;
                    st[0] = lstart;
                    ln[0] = lend - lstart;
                } else {
                    const int a = ((ja % nphi) + nphi) % nphi;
                    const int b = ((jb % nphi) + nphi) % nphi;
                    if (a <= b) {
                        nr = 1;
                        st[0] = offs[l * nphi + a];
                        ln[0] = offs[l * nphi + b + 1] - st[0];
                    } else {
                        nr = 2;
                        st[0] = offs[l * nphi + a];
                        ln[0] = lend - st[0];
                        st[1] = lstart;
                        ln[1] = offs[l * nphi + b + 1] - lstart;
                    }
                }
            }
        }
        s_start[2 * l] = st[0];
        s_start[2 * l + 1] = st[1];
        s_pre[2 * l] = nr >= 1 ? ln[0] : 0;       // lengths for now
        s_pre[2 * l + 1] = nr >= 2 ? ln[1] : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int q = 0; q < kMaxRanges; ++q) {
            const int len = s_pre[q];
            s_pre[q] = acc;
            acc += len;
        }
        s_pre[kMaxRanges] = acc;
    }
    __syncthreads();

    const int total = s_pre[kMaxRanges];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned long long refined = 0;
    for (int base = warp * 32; base < total; base += TPB) {
        const int v = base + lane;
        const bool has = v < total;
        HotHit hh;
        hh.f = 0.f;
        hh.c = 0.f;
        hh.jl = 0u;
        hh.rows = 1u;   // rows [1, 0]: none
        int pos = 0;
        if (has) {
            int q = 0;
            while (q + 1 < kMaxRanges && s_pre[q + 1] <= v) ++q;
            pos = s_start[q] + (v - s_pre[q]);
            hh = hot[pos];
        }
        const int J = (int)(hh.jl & 0xFFFFu);
        const int l = (int)((hh.jl >> 16) & 0xFu);
        const int rlo = (int)(hh.rows & 0xFFFFu), rhi = (int)(hh.rows >> 16);
        const bool uni = (umask >> l) & 1u;
        const uint32_t lbit = 1u << l;
        for (int rr = 0; rr < nrows; ++rr) {
            const int i = i0 + rr;
            const bool act = has && i >= rlo && i <= rhi;
            int j;
            if (uni) {
                const TabEntry te = tab[l * R + rr];
                j = J - te.I - (hh.f < te.g ? 1 : 0);
            } else {
                const float x = fminf(fmaxf(hh.c * kq[rr], -1.f), 1.f);
                const float vq = fmaf(-asinf(x), p.s32, hh.f);
                const float fl = floorf(vq);
                const float d = vq - fl;
                j = J + (int)fl;
                if (act && (d < p.refine_eps || d > 1.f - p.refine_eps || fabsf(x) > kRefineXLim)) {
                    const ColdHit ch = cold[pos];
                    const double x64 = __dmul_rn(sagitta_coef(ax, (double)ch.r), qpt_centre(ax, i));
                    j = exact_bin(ax, (double)ch.phi, x64);
                    ++refined;
                }
            }
            j += j < 0 ? nphi : 0;
            j -= j >= nphi ? nphi : 0;
            const int jt = j - J0;
            const bool in = act && (unsigned)jt < (unsigned)W;
            const int word = rr * Wh + (jt >> 1);
            const uint32_t tag = in ? (((uint32_t)word << 5) | ((uint32_t)l << 1) | (uint32_t)(jt & 1)) : 0xFFFFFFFFu;
            const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, tag, 1);
            if (in && !(lane > 0 && prev == tag)) atomicOr(&tile[word], lbit << ((jt & 1) << 4));
        }
    }
    if (refined) atomicAdd(&s_refined, refined);
    __syncthreads();

    // flush the tile: each row is W/8 16-byte vectors
    uint16_t *M = p.w.M + (int64_t)e * ax.n_qpt * nphi;
    const int v8 = W >> 3;
    for (int q = threadIdx.x; q < nrows * v8; q += TPB) {
        const int rr = q / v8, c8 = q - rr * v8;
        *reinterpret_cast<uint4 *>(M + (int64_t)(i0 + rr) * nphi + J0 + c8 * 8) = tile4[rr * v8 + c8];
    }
    if (threadIdx.x == 0 && s_refined) atomicAdd(&p.w.stats[e].refined_votes, s_refined);
}

template <int TPB>
cudaError_t launch_tpb(const VoteParams &p, size_t smem, int grid, cudaStream_t stream)
{
    cudaError_t err = cudaFuncSetAttribute(vote_kernel<TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err) return err;
    vote_kernel<TPB><<<grid, TPB, smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace

size_t vote_smem_bytes(const Axes &ax, const Tiling &t)
{
    return (size_t)t.tile_qpt * t.tile_phi * 2 + (size_t)ax.n_layers * t.tile_qpt * sizeof(TabEntry) +
           (size_t)t.tile_qpt * sizeof(float);
}

cudaError_t launch_vote(const Axes &ax, const Workspace &w, const Tiling &t, float refine_eps,
                        cudaStream_t stream)
{
    VoteParams p;
    p.ax = ax;
    p.w = w;
    p.R = t.tile_qpt;
    p.W = t.tile_phi;
    p.n_spans = ax.n_phi / t.tile_phi;
    p.tiles_per_event = ((ax.n_qpt + t.tile_qpt - 1) / t.tile_qpt) * p.n_spans;
    p.s32 = (float)(ax.n_phi * kInvTwoPi);
    p.refine_eps = refine_eps;
    const size_t smem = vote_smem_bytes(ax, t);
    const int grid = w.n_events * p.tiles_per_event;
    switch (t.threads) {
    case 128: return launch_tpb<128>(p, smem, grid, stream);
    case 256: return launch_tpb<256>(p, smem, grid, stream);
    case 512: return launch_tpb<512>(p, smem, grid, stream);
    case 1024: return launch_tpb<1024>(p, smem, grid, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hough
