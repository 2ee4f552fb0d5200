// Stage-1 vote (Sec. 4, first step; the A[B[i]] += 1 scatter of Sec. 8), accumulator flush and
// the peak search over row bands (Sec. 4, second step).
//
// Three ways to fill the accumulator, selected per layer on the device:
//
// 1. Gather (layers whose hits share one radius; every configured workload).  On row i every
//    hit of such a layer votes at J - I_i - (f < g_i): its own bin coordinate J + f shifted by the
//    table's Nphi asin(x_i) / (2 pi) = I_i + g_i.  So layer l's bit of cell (i, j) is set exactly
//    when bucket J' = (j + I_i) mod Nphi holds a hit with f >= g_i, or bucket J' + 1 holds one with
//    f < g_i -- a test of the buckets' largest and smallest f, which the staging recorded.  The
//    gather kernel evaluates that test for every (cell, layer) of a tile: no atomics, each
//    accumulator word written once with a coalesced 16-byte store.  Same FP32 comparisons as the
//    per-vote form, so the same accumulator bit for bit.
//
// 2. Scatter (the paper's remedy, Sec. 6.1: shared-memory atomics instead of global ones).  One CTA
//    per (event, tile of tile_qpt rows x tile_phi columns) in shared memory.  The CTA reads only the
//    hits that can vote into its tile -- per layer one or two contiguous ranges of the
//    (layer, phi bin)-sorted hits -- lane by lane, and loops over the tile's rows in lockstep, so a
//    warp's 32 same-layer, azimuth-sorted hits update neighbouring words of one row; a lane whose
//    (word, bit) equals its left neighbour's skips its atomicOr.  With the count accumulator the
//    tile holds a 32-bit counter per cell instead: each run of lanes voting into the same cell
//    adds its length with one atomicAdd from its first lane, and the flush saturates every counter
//    to 16 bits -- the literal A[B[i]] += 1 of Sec. 8.  Table layers vote at
//    J - I - (f < g); other layers take FP32 asinf per vote, and a vote within `refine_eps` of an
//    edge (or with |x| > kRefineXLim) is recomputed in FP64 in the definition's order.  In the
//    default (gather) mode this kernel handles only the layers whose radii differ and ORs its tile
//    into the accumulator (adds it, with counts); in scatter mode it handles every layer and stores
//    its tile.
//
// 3. Count gather (the count accumulator's gather mode): per cell and layer of one radius, the hits
//    of bucket J' with f >= g_i and of bucket J' + 1 with f < g_i, counted from the sorted f values
//    of the tile's window of buckets (gather_count_kernel).
//
// Peaks: candidates of each band of band_rows rows (one row by default) go to a band list in
// raster order; a per-event scan then concatenates the band lists into the raster-ordered list.
// With a d0 axis a band lies in one slice and its cells take the 3 x 3 x 3 rule (peaks3_kernel).
#include <algorithm>
#include <atomic>
#include <climits>

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
constexpr int kRefineQueue = 64;   // a warp's queue of votes decided in FP64 (see scatter_kernel)
constexpr int kCompactThreads = 1024;

// Layers of the batch: bit l of *uniform_out is set when layer l takes the table path; bit l of
// *general_out when it has hits at more than one radius.  Called by warp 0.
__device__ __forceinline__ void layer_masks(const Workspace &w, int L, unsigned *uniform_out, unsigned *general_out)
{
    const int l = threadIdx.x;
    LayerInfo li;
    li.present = 0;
    li.uniform = 1;
    if (l < L) li = w.info[l];
    *uniform_out = __ballot_sync(0xFFFFFFFFu, l < L && li.uniform);
    *general_out = __ballot_sync(0xFFFFFFFFu, l < L && li.present && !li.uniform);
}

// Shared tile of the scatter kernel, column-major: cell (row rr, column jt) of a tile of R rows
// lives in word jt * pitch + rr (CELL 1: a layer mask a word; CELL 2: a 32-bit counter a word) or,
// when that tile does not fit in shared memory, word (jt >> 1) * pitch + rr (CELL 0: two 16-bit layer
// masks a word).  The lanes of a warp vote for 32 consecutive rows, so their 32 atomics fall in 32
// different banks whatever columns the votes land in.
__host__ __device__ inline int tile_row_pitch(int R) { return R <= 32 ? R : (R + 31) & ~31; }
// Margin columns on each side of the tile: a table layer's vote j - J0 lies within its window's
// spread of I beyond the tile's columns, so when that spread fits the margin every vote of the
// layer is cast where it falls -- into the tile or into a margin, which the flush ignores --
// without a test, a clamp or a select (even, so two-mask words keep their pairing).
constexpr int kTileMargin = 64;
__host__ __device__ inline int scatter_tile_words(int R, int W, bool wide)
{
    return (wide ? W + 2 * kTileMargin : (W + 2 * kTileMargin) >> 1) * tile_row_pitch(R);
}
// Byte offset of the per-warp hit buffers in the scatter kernel's dynamic shared memory.
__host__ __device__ inline size_t scatter_hit_offset(int R, int W, int L, bool wide)
{
    return ((size_t)scatter_tile_words(R, W, wide) * 4 + (size_t)L * R * sizeof(TabEntry) + (size_t)R * 4 + 15) &
           ~(size_t)15;
}

// One shared atomic update of cell (rr, jt) of the tile: the layer bit (masks) or one vote (counts).
template <int CELL>
__device__ __forceinline__ void tile_vote(uint32_t *tile, int pitch, int rr, int jt, uint32_t lbit)
{
    if (CELL == 2) atomicAdd(&tile[jt * pitch + rr], 1u);
    else if (CELL == 1) atomicOr(&tile[jt * pitch + rr], lbit);
    else atomicOr(&tile[(jt >> 1) * pitch + rr], lbit << ((jt & 1) << 4));
}

// A vote cast where it falls, at column jt of the lane's row (base: the row's word of column 0 as a
// shared-memory address, s4: the column stride in bytes, 0 for a lane whose votes all go to a
// word of its own).  jt may lie in a margin.
template <int CELL>
__device__ __forceinline__ void tile_vote_at(unsigned base, int s4, int jt, uint32_t lbit)
{
    if (CELL == 2) asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(base + jt * s4) : "memory");
    else if (CELL == 1) asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(base + jt * s4), "r"(lbit) : "memory");
    else asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(base + (jt >> 1) * s4), "r"(lbit << ((jt & 1) << 4)) : "memory");
}

// The votes of hits k0..k1-1 of the warp's buffer (f, byte offset of the column) for one row and
// one layer of one mask a word: the vote of hit k goes to rowbase + offset_k - (f_k < g) s4b.  PRED:
// some lane's row casts nothing (valid false), its atomics predicated off.
template <int CELL, bool PRED>
__device__ __forceinline__ void vote_run(const uint2 *hb2, int k0, int k1, float g, unsigned rowbase, unsigned s4b,
                                         uint32_t lbit, bool valid)
{
    const unsigned vflag = valid ? 1u : 0u;
    auto one = [&](uint2 h) {
        const unsigned a = rowbase + h.y - (__uint_as_float(h.x) < g ? s4b : 0u);
        if (PRED) {
            if (CELL == 2)
                asm volatile("{ .reg .pred p; setp.ne.u32 p, %1, 0; @p red.shared.add.u32 [%0], 1; }" ::"r"(a), "r"(vflag)
                             : "memory");
            else
                asm volatile("{ .reg .pred p; setp.ne.u32 p, %2, 0; @p red.shared.or.b32 [%0], %1; }" ::"r"(a), "r"(lbit),
                             "r"(vflag) : "memory");
        } else {
            if (CELL == 2) asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(a) : "memory");
            else asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(a), "r"(lbit) : "memory");
        }
    };
    int k = k0;
    for (; k + 8 <= k1; k += 8) {
        uint2 h[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) h[u] = hb2[2 * (k + u)];
#pragma unroll
        for (int u = 0; u < 8; ++u) one(h[u]);
    }
    for (; k < k1; ++k) one(hb2[2 * k]);
}

// The same for a vote that may miss the tile (in false): every lane issues its atomic, a missing
// vote adding nothing to a cell of its own row, so that no branch surrounds the atomic.  rowp,
// stride: the lane's row of the tile and the column stride (pitch), or for a lane without a row of
// the tile a word of its own with stride 0.
template <int CELL>
__device__ __forceinline__ void tile_vote_if(uint32_t *rowp, int stride, int jt, int W, bool in, uint32_t lbit)
{
    const int jc = (int)min((unsigned)jt, (unsigned)(W - 1));   // a column of the tile
    if (CELL == 2) atomicAdd(&rowp[jc * stride], in ? 1u : 0u);
    else if (CELL == 1) atomicOr(&rowp[jc * stride], in ? lbit : 0u);
    else atomicOr(&rowp[(jc >> 1) * stride], in ? lbit << ((jc & 1) << 4) : 0u);
}

template <int TPB, bool GENERAL_ONLY, int CELL>
__global__ void __launch_bounds__(TPB) scatter_kernel(VoteParams p)
{
    constexpr bool COUNTS = CELL == 2;
    // After the gather (GENERAL_ONLY) this kernel reads nothing its predecessor writes until its
    // flush ORs its tile into the gathered accumulator: the layer records, tables, bucket offsets
    // and sorted hits come from kernels that finished before the gather could launch.  So it checks
    // for layers of several radii and casts their votes first, and waits for the gather only before
    // the flush (or before returning with nothing to do), which keeps its completion behind the
    // gather's.  Voting every layer, it follows the hit sort and waits at once.
    if (!GENERAL_ONLY) pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_start[kMaxRanges], s_off[kMaxRanges];
    __shared__ int s_pre[kMaxRanges + 1];
    __shared__ unsigned long long s_refined;
    __shared__ unsigned s_umask, s_gmask;
    __shared__ unsigned s_fast;   // table layers whose spread of I fits the tile's margins

    const Axes &ax = p.ax;
    const int R = p.R, W = p.W, L = ax.n_layers, nphi = ax.n_phi;
    const int pitch = tile_row_pitch(R);
    uint32_t *tile_all = reinterpret_cast<uint32_t *>(smem_raw);
    const int tile_words = scatter_tile_words(R, W, CELL != 0);
    uint32_t *tile = tile_all + (CELL != 0 ? kTileMargin : kTileMargin / 2) * pitch;   // column 0
    TabEntry *tab = reinterpret_cast<TabEntry *>(tile_all + tile_words);
    float *kq = reinterpret_cast<float *>(tab + L * R);
    // the warp's 32 staged hits: f (bits), J (shifted into the window for a table layer), c (bits), rows
    uint4 *hitbuf = reinterpret_cast<uint4 *>(smem_raw + scatter_hit_offset(R, W, L, CELL != 0)) + 32 * (threadIdx.x >> 5);
    // the warp's queue of votes to be decided in FP64: (staged position, row | layer << 16)
    uint2 *rq = reinterpret_cast<uint2 *>(smem_raw + scatter_hit_offset(R, W, L, CELL != 0) + (size_t)TPB * sizeof(uint4)) +
                kRefineQueue * (threadIdx.x >> 5);
    // 32 words that the atomics of lanes without a row of the tile go to (adding nothing)
    uint32_t *spare = reinterpret_cast<uint32_t *>(smem_raw + scatter_hit_offset(R, W, L, CELL != 0) +
                                                   (size_t)TPB * sizeof(uint4) + (size_t)(TPB / 32) * kRefineQueue * sizeof(uint2));

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

    if (threadIdx.x < 32) {
        unsigned u, g;
        layer_masks(p.w, L, &u, &g);
        if (threadIdx.x == 0) {
            s_umask = GENERAL_ONLY ? ~g : u;   // layers this kernel treats with the table
            s_gmask = g;
            s_refined = 0ull;
            s_fast = 0u;
        }
    }
    __syncthreads();
    // in gather mode there is nothing to do unless some layer has hits at several radii
    if (GENERAL_ONLY && s_gmask == 0u) {
        pdl_enter();
        return;
    }
    const unsigned umask = s_umask;

    // clear the tile; stage this slab's table rows and FP32 q/pT centres
    uint4 *tile4 = reinterpret_cast<uint4 *>(tile_all);
    for (int q = threadIdx.x; q < tile_words >> 2; q += TPB) tile4[q] = make_uint4(0u, 0u, 0u, 0u);
    for (int q = threadIdx.x; q < L * R; q += TPB) {
        const int l = q / R, rr = q - l * R;
        TabEntry te;
        te.I = kNoVote;
        te.g = 0.f;
        if (!GENERAL_ONLY && rr < nrows && ((umask >> l) & 1u)) te = p.w.tab[l * ax.n_qpt + i0 + rr];
        tab[q] = te;
    }
    for (int q = threadIdx.x; q < R; q += TPB) kq[q] = q < nrows ? p.w.kq32[i0 + q] : 0.f;
    __syncthreads();

    // Per layer, the hits that can vote into this tile: a cyclic window [ja, jb] of phi bins J,
    // as one or two ranges of the sorted hits.  s_off[q] is the shift that takes the J of range q's
    // hits into the window's unwrapped coordinates (J + s_off in [ja, jb]).
    if (threadIdx.x < HOUGH_MAX_LAYERS) {
        const int l = threadIdx.x;
        int nr = 0, st[2] = {0, 0}, ln[2] = {0, 0}, of[2] = {0, 0};
        if (l < L) {
            const int lstart = offs[l * nphi], lend = offs[(l + 1) * nphi];
            int ja = 0, jb = -1;   // inclusive J window, possibly beyond [0, nphi)
            bool none = lend == lstart;
            if (!none && ((umask >> l) & 1u)) {
                if (GENERAL_ONLY) {
                    none = true;   // the gather kernel votes for this layer
                } else {
                    // vote bin J - I - (f < g) lies in [J0, J0 + W) only for J in
                    // [J0 + min I, J0 + W + max I] over the slab's voting rows
                    int imin = INT_MAX, imax = INT_MIN;
                    for (int rr = 0; rr < nrows; ++rr) {
                        const int I = tab[l * R + rr].I;
                        if (I != kNoVote) {
                            imin = min(imin, I);
                            imax = max(imax, I);
                        }
                    }
                    if (imin > imax) {
                        none = true;
                    } else {
                        ja = J0 + imin;
                        jb = J0 + W + imax;
                        // votes of this window fall in [imin - imax - 1, W + imax - imin] of the tile
                        if (imax - imin + 1 <= kTileMargin) atomicOr(&s_fast, 1u << l);
                    }
                }
            } else if (!none && ax.n_d0) {
                ja = 0;   // per-vote layer on a grid with a d0 axis: every hit of the layer
                jb = nphi;
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
                if (jb - ja + 1 >= nphi) {
                    nr = 1;
                    st[0] = lstart;
                    ln[0] = lend - lstart;
                } else {
                    const int a = ((ja % nphi) + nphi) % nphi;
                    const int b = ((jb % nphi) + nphi) % nphi;
                    of[0] = ja - a;
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
                        of[1] = ja - a + nphi;
                    }
                }
            }
        }
        s_start[2 * l] = st[0];
        s_start[2 * l + 1] = st[1];
        s_off[2 * l] = of[0];
        s_off[2 * l + 1] = of[1];
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

    // A warp votes for 32 consecutive rows of the tile, a lane per row, taking the tile's hits 32
    // at a time: the 32 are staged in the warp's buffer and broadcast one by one to all lanes.  For
    // a table layer the lane's vote is j = J - I_row - (f < g_row): with the table entry in
    // registers, a compare, an add and the atomic.  When the tile is at most a quarter of the row,
    // the window of a layer's J is shorter than a row less the tile, so the vote lands in the tile
    // exactly when (J + s_off) - (I + J0) - (f < g) lies in [0, W), with no reduction modulo Nphi.
    const int total = s_pre[kMaxRanges];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = TPB / 32;
    const int NG = (R + 31) >> 5;           // groups of 32 rows
    const int HS = max(1, NW / NG);         // warps sharing a row group's hits
    const bool wrap = W > (nphi >> 2);
    unsigned long long refined = 0;
    // Votes of the per-vote path within the refine window are not decided in the loop below: a
    // warp would run the FP64 arcsine for one lane.  They wait in the warp's queue, and every 32 of
    // them are decided together, a lane each (and cast: the atomics commute).
    int qn = 0;   // queued votes (the same in every lane)
    auto flush_refines = [&]() {
        __syncwarp();
        for (int t = lane; t < qn; t += 32) {
            const uint2 q = rq[t];
            const int row = (int)(q.y & 0xFFFFu);
            const ColdHit ch = cold[q.x];
            const double x64 = __dmul_rn(sagitta_coef(ax, (double)ch.r), qpt_centre(ax, i0 + row));
            const int jt = exact_bin(ax, (double)ch.phi, x64) - J0;
            if ((unsigned)jt < (unsigned)W) tile_vote<CELL>(tile, pitch, row, jt, 1u << (q.y >> 16));
        }
        __syncwarp();
        qn = 0;
    };
    for (int task = warp; task < NG * HS; task += NW) {
        const int rr = (task % NG) * 32 + lane;
        const int hs = task / NG;
        const bool rowok = rr < nrows;
        const int i = i0 + rr;
        const float kqr = rowok ? kq[rr] : 0.f;
        uint32_t *rowp = rowok ? tile + rr : spare + lane;
        const int stride = rowok ? pitch : 0;
        // hit v's staged position, window shift and record (empty past the last hit); the next
        // chunk's record is requested before this chunk votes, so its load overlaps the votes
        auto fetch_hit = [&](int v, int &pos, int &off, HotHit &hh) {
            hh.f = 0.f;
            hh.c = 0.f;
            hh.jl = 16u << 16;   // layer 16: none
            hh.rows = 1u;        // rows [1, 0]: none
            pos = 0;
            off = 0;
            if (v < total) {
                int q = 0;   // the range holding v: the last q with s_pre[q] <= v
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (s_pre[q + step] <= v) q += step;
                pos = s_start[q] + (v - s_pre[q]);
                off = s_off[q];
                hh = hot[pos];
            }
        };
        int pos_n, off_n;
        HotHit hh_n;
        fetch_hit(hs * 32 + lane, pos_n, off_n, hh_n);
        for (int cb = hs * 32; cb < total; cb += HS * 32) {
            const int nvalid = min(32, total - cb);
            const int pos = pos_n, off = off_n;
            const HotHit hh = hh_n;
            if (cb + HS * 32 < total) fetch_hit(cb + HS * 32 + lane, pos_n, off_n, hh_n);
            const int l = (int)((hh.jl >> 16) & 0x1Fu);
            const int J = (int)(hh.jl & 0xFFFFu);
            const bool table_hit = !GENERAL_ONLY && l < 16 && ((umask >> l) & 1u);
            // a table layer whose votes fall within the margins, one mask a word: the byte offset
            // of its column in a row of the tile (the vote then subtracts the row's shift in bytes)
            const bool fast_hit = CELL != 0 && !wrap && table_hit && ((s_fast >> l) & 1u);
            hitbuf[lane] = make_uint4(__float_as_uint(hh.f),
                                      fast_hit ? (uint32_t)((J + off) * 4 * pitch)
                                               : (uint32_t)(wrap || !table_hit ? J : J + off),
                                      __float_as_uint(hh.c), hh.rows);
            __syncwarp();
            // runs of hits of one layer (the ranges are in layer order)
            const int lprev = __shfl_up_sync(0xFFFFFFFFu, l, 1);
            unsigned heads = __ballot_sync(0xFFFFFFFFu, lane < nvalid && (lane == 0 || l != lprev));
            while (heads) {
                const int k0 = __ffs(heads) - 1;
                heads &= heads - 1u;
                const int k1 = heads ? __ffs(heads) - 1 : nvalid;
                const int lr = __shfl_sync(0xFFFFFFFFu, l, k0);
                const uint32_t lbit = 1u << lr;
                if (!GENERAL_ONLY && ((umask >> lr) & 1u)) {
                    const TabEntry te = tab[lr * R + (rowok ? rr : 0)];
                    const bool valid = rowok && te.I != kNoVote;
                    const float g = te.g;
                    if (CELL != 0 && !wrap && ((s_fast >> lr) & 1u)) {
                        // every vote where it falls: the word of column (J + off) - K - (f < g) of the
                        // lane's row, its byte offset from the staged column offset; a lane of an
                        // invalid row (or none) casts nothing
                        const unsigned s4b = 4u * (unsigned)pitch;
                        const unsigned rowbase = smem_u32(tile + rr) - (unsigned)(te.I + J0) * s4b;
                        const uint2 *hb2 = reinterpret_cast<const uint2 *>(hitbuf);   // (f, column bytes) of hit k at 2 k
                        if (__all_sync(0xFFFFFFFFu, valid))
                            vote_run<CELL, false>(hb2, k0, k1, g, rowbase, s4b, lbit, true);
                        else
                            vote_run<CELL, true>(hb2, k0, k1, g, rowbase, s4b, lbit, valid);
                    } else if (!wrap && ((s_fast >> lr) & 1u)) {
                        // the same with two masks a word: the vote's column from its J
                        const unsigned base = valid ? smem_u32(tile + rr) : smem_u32(spare + lane);
                        const int s4 = valid ? 4 * pitch : 0;
                        const int K = te.I + J0;
                        int k = k0;
                        const uint2 *hb2 = reinterpret_cast<const uint2 *>(hitbuf);   // (f, J) of hit k at 2 k
                        for (; k + 8 <= k1; k += 8) {
                            uint2 h[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u) h[u] = hb2[2 * (k + u)];
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                tile_vote_at<CELL>(base, s4, (int)h[u].y - K - (__uint_as_float(h[u].x) < g ? 1 : 0), lbit);
                        }
                        for (; k < k1; ++k) {
                            const uint2 h = hb2[2 * k];
                            tile_vote_at<CELL>(base, s4, (int)h.y - K - (__uint_as_float(h.x) < g ? 1 : 0), lbit);
                        }
                    } else if (!wrap) {
                        const int K = valid ? te.I + J0 : -(1 << 30);   // an invalid row's votes all miss
                        // four hits at a time: their loads issue together, then their atomics
                        int k = k0;
                        const uint2 *hb2 = reinterpret_cast<const uint2 *>(hitbuf);   // (f, J) of hit k at 2 k
                        for (; k + 4 <= k1; k += 4) {
                            uint2 h[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) h[u] = hb2[2 * (k + u)];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int jt = (int)h[u].y - K - (__uint_as_float(h[u].x) < g ? 1 : 0);
                                tile_vote_if<CELL>(rowp, stride, jt, W, (unsigned)jt < (unsigned)W, lbit);
                            }
                        }
                        for (; k < k1; ++k) {
                            const uint2 h = hb2[2 * k];
                            const int jt = (int)h.y - K - (__uint_as_float(h.x) < g ? 1 : 0);
                            tile_vote_if<CELL>(rowp, stride, jt, W, (unsigned)jt < (unsigned)W, lbit);
                        }
                    } else {
                        for (int k = k0; k < k1; ++k) {
                            const uint4 h = hitbuf[k];
                            int j = (int)h.y - te.I - (__uint_as_float(h.x) < g ? 1 : 0);
                            j += j < 0 ? nphi : 0;
                            j -= j >= nphi ? nphi : 0;
                            const int jt = j - J0;
                            tile_vote_if<CELL>(rowp, stride, jt, W, valid && (unsigned)jt < (unsigned)W, lbit);
                        }
                    }
                    continue;
                }
                // a layer whose hits lie at several radii: every vote evaluated per hit
                for (int k = k0; k < k1; ++k) {
                    const uint4 h = hitbuf[k];
                    const float c = __uint_as_float(h.z), fk = __uint_as_float(h.x);
                    const uint32_t rows = h.w;
                    const int Jk = (int)h.y;
                    bool act = rowok && i >= (int)(rows & 0xFFFFu) && i <= (int)(rows >> 16);
                    int j = 0;
                    if (ax.n_d0) {
                        // a grid with a d0 axis: every vote of a per-vote layer in FP64, in the definition's order
                        const int pk = __shfl_sync(0xFFFFFFFFu, pos, k);
                        if (act) {
                            const ColdHit ch = cold[pk];
                            act = exact_vote(ax, (double)ch.r, (double)ch.phi, i, &j);
                        }
                    } else {
                        const float x = fminf(fmaxf(c * kqr, -1.f), 1.f);
                        const float vq = fmaf(-asinf(x), p.s32, fk);
                        const float fl = floorf(vq);
                        const float d = vq - fl;
                        j = Jk + (int)fl;
                        const bool need = act && (d < p.refine_eps || d > 1.f - p.refine_eps || fabsf(x) > kRefineXLim);
                        if (__any_sync(0xFFFFFFFFu, need)) {   // rare: queue them
                            const int pk = __shfl_sync(0xFFFFFFFFu, pos, k);
                            const unsigned rb = __ballot_sync(0xFFFFFFFFu, need);
                            if (need) rq[qn + __popc(rb & ((1u << lane) - 1u))] = make_uint2((uint32_t)pk, (uint32_t)rr | ((uint32_t)lr << 16));
                            qn += __popc(rb);
                            if (lane == 0) refined += __popc(rb);
                            act = act && !need;
                        }
                    }
                    j += j < 0 ? nphi : 0;
                    j -= j >= nphi ? nphi : 0;
                    const int jt = j - J0;
                    tile_vote_if<CELL>(rowp, stride, jt, W, act && (unsigned)jt < (unsigned)W, lbit);
                    if (qn >= 32) flush_refines();   // at most 63 queued
                }
            }
            __syncwarp();   // the buffer is read before the next chunk overwrites it
        }
    }
    if (qn) flush_refines();
    if (refined) atomicAdd(&s_refined, refined);
    if (GENERAL_ONLY) pdl_enter();   // the gathered accumulator is complete
    __syncthreads();

    // flush the tile: 8 cells of a row per thread, consecutive threads on consecutive rows (one
    // bank each in the column-major tile), one 16-byte store (ORed into the gathered layers' bits,
    // or added to their counts, when only the layers of several radii were voted here)
    uint16_t *M = p.w.M + (int64_t)e * ax.n_qpt * nphi;
    const int v8 = W >> 3;
    for (int q = threadIdx.x; q < nrows * v8; q += TPB) {
        const int c8 = q / nrows, rr = q - c8 * nrows;
        uint4 *dst = reinterpret_cast<uint4 *>(M + (int64_t)(i0 + rr) * nphi + J0 + c8 * 8);
        if (COUNTS) {
            uint32_t cnt[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) cnt[k] = tile[(c8 * 8 + k) * pitch + rr];
            if (GENERAL_ONLY) {
                const uint4 old = *dst;
                const uint32_t ow[4] = {old.x, old.y, old.z, old.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    cnt[2 * k] += ow[k] & 0xFFFFu;
                    cnt[2 * k + 1] += ow[k] >> 16;
                }
            }
            auto pack = [](uint32_t lo, uint32_t hi) { return min(lo, 65535u) | (min(hi, 65535u) << 16); };
            *dst = make_uint4(pack(cnt[0], cnt[1]), pack(cnt[2], cnt[3]), pack(cnt[4], cnt[5]), pack(cnt[6], cnt[7]));
            continue;
        }
        uint4 v;
        if (CELL == 1) {   // a mask a word: pairs of cells into one word
            uint32_t m[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) m[k] = tile[(c8 * 8 + k) * pitch + rr];
            v = make_uint4(m[0] | (m[1] << 16), m[2] | (m[3] << 16), m[4] | (m[5] << 16), m[6] | (m[7] << 16));
        } else {
            v = make_uint4(tile[(c8 * 4) * pitch + rr], tile[(c8 * 4 + 1) * pitch + rr], tile[(c8 * 4 + 2) * pitch + rr],
                           tile[(c8 * 4 + 3) * pitch + rr]);
        }
        if (GENERAL_ONLY) {
            const uint4 old = *dst;
            v.x |= old.x;
            v.y |= old.y;
            v.z |= old.z;
            v.w |= old.w;
        }
        *dst = v;
    }
    if (threadIdx.x == 0 && s_refined) atomicAdd(&p.w.stats[e].refined_votes, s_refined);
}

// Gather: one tile of `rows` rows x `cols` columns of the accumulator from the per-bucket f
// extrema and the table.  On row i a layer's cells read the bucket entries shifted by I_i, which
// grows with i, so the tile reads one contiguous window of each layer's entries:
// [c0 + min_i I_i, c0 + cols + 2 + max_i I_i).  Thread 0 copies every layer's window into shared
// memory with bulk asynchronous copies (one or two pieces, the second when the window wraps
// around phi) completing on one mbarrier, while the other threads wait; a layer whose window does
// not fit its slot reads global memory instead.  A warp then takes a strip of up to 256 cells of a
// row, 8 per lane at a stride of 32; the staging put bucket J+1's smallest fraction beside bucket
// J's largest, so a layer's bit of cell j reads the one 8-byte entry j + I: conflict-free shared
// loads, one per (cell, voting layer), the layer's shift and threshold read once per 8 cells.
struct GatherParams {
    Axes ax;
    Workspace w;
    int rows, cols, col_tiles, tiles_per_event;
    int cap;   // entries of a layer's staging slot (even)
};

constexpr int kGatherRowsMax = 32;
constexpr long long kCopyWaitCycles = 2000000000LL;   // about a second: bulk copies take microseconds

// The first bound on the wait for a CTA's bulk copies: about a second, or none at all when a test of
// the error path asked for it (Workspace::copy_wait < 0).  On expiry the CTA reports
// HOUGH_DEVERR_TIMEOUT and waits once more, with the full bound, for its copies to land, so that it
// leaves no copy writing into shared memory after it has exited (unless that wait expires too).
__device__ __forceinline__ bool first_copy_wait(const Workspace &w, uint64_t *bar)
{
    if (w.copy_wait < 0) return false;
    return mbar_wait_bounded(bar, 0, kCopyWaitCycles);
}

template <int NL, int TPB>
__global__ void __launch_bounds__(TPB, 1) gather_kernel(GatherParams p)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char gather_smem[];
    __shared__ int rowI[kGatherRowsMax * 16];
    __shared__ unsigned rowG[kGatherRowsMax * 16];
    __shared__ unsigned rowMask[kGatherRowsMax];
    __shared__ int s_wbase[16], s_wlen[16];
    __shared__ unsigned s_staged;
    __shared__ __align__(8) uint64_t s_bar;
    const Axes &ax = p.ax;
    const Workspace &w = p.w;
    const int e = blockIdx.x / p.tiles_per_event;
    const int t = blockIdx.x - e * p.tiles_per_event;
    const int rt = t / p.col_tiles, ct = t - rt * p.col_tiles;
    const int i0 = rt * p.rows, c0 = ct * p.cols;
    const int nrows = min(p.rows, ax.n_qpt - i0);
    const int L = ax.n_layers, nphi = ax.n_phi;

    // per (row, layer): the table entry and whether the layer votes on that row by the gather
    // (whole warps, so that the ballot sees full warps; TPB is a multiple of 32)
    for (int q = threadIdx.x; q < ((p.rows * 16 + 31) & ~31); q += TPB) {
        const int rr = q >> 4, l = q & 15, i = i0 + rr;
        int I = 0;
        unsigned gb = 0u, valid = 0u;
        if (l < L && rr < nrows) {
            const LayerInfo li = w.info[l];
            const TabEntry te = w.tab[l * ax.n_qpt + i];   // requested with the layer record: one round trip
            if (li.present && li.uniform && i >= li.lo && i <= li.hi) {
                if (te.I != kNoVote) {
                    I = te.I;
                    gb = __float_as_uint(te.g);
                    valid = 1u;
                }
            }
        }
        const unsigned m = __ballot_sync(0xFFFFFFFFu, valid) >> (threadIdx.x & 16);
        rowI[q] = I;
        rowG[q] = gb;
        if ((threadIdx.x & 15) == 0) rowMask[rr] = m & 0xFFFFu;
    }
    __syncthreads();
    // each layer's window of bucket entries (unwrapped indices, start even)
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        bool staged = false;
        if (l < L) {
            int lo = INT_MAX, hi = INT_MIN;
            for (int rr = 0; rr < nrows; ++rr)
                if ((rowMask[rr] >> l) & 1u) {
                    lo = min(lo, rowI[rr * 16 + l]);
                    hi = max(hi, rowI[rr * 16 + l]);
                }
            if (lo <= hi) {
                const int ws = (c0 + lo) - ((c0 + lo) & 1);
                int len = c0 + p.cols + 2 + hi - ws;
                len += len & 1;
                staged = len <= p.cap && len <= nphi;
                s_wbase[l] = ws;
                s_wlen[l] = len;
            }
        }
        const unsigned sm = __ballot_sync(0xFFFFFFFFu, staged);
        if (l == 0) {
            s_staged = sm;
            if (sm) mbar_init(&s_bar, 1);
        }
    }
    __syncthreads();
    const unsigned staged = s_staged;
    const uint2 *prof = w.prof + (int64_t)e * prof_event_entries(ax);
    const int pstride = prof_stride(ax);
    uint2 *win = reinterpret_cast<uint2 *>(gather_smem);
    if (staged) {
        if (threadIdx.x == 0) {
            unsigned bytes = 0;
            for (int l = 0; l < L; ++l)
                if ((staged >> l) & 1u) bytes += 8u * (unsigned)s_wlen[l];
            mbar_arrive_expect(&s_bar, bytes);
            for (int l = 0; l < L; ++l) {
                if (!((staged >> l) & 1u)) continue;
                const int len = s_wlen[l];
                const int a = ((s_wbase[l] % nphi) + nphi) % nphi;   // even, as nphi is
                const uint2 *src = prof + (int64_t)l * pstride;
                uint2 *dst = win + (int64_t)l * p.cap;
                const int first = min(len, nphi - a);
                bulk_copy_g2s(dst, src + a, 8u * (unsigned)first, &s_bar);
                if (first < len) bulk_copy_g2s(dst + first, src, 8u * (unsigned)(len - first), &s_bar);
            }
        }
        const bool ok = first_copy_wait(w, &s_bar);
        if (!__syncthreads_and(ok)) {
            // the copies did not land in time: report it, give them one more bound, write nothing
            if (threadIdx.x == 0) atomicOr(&w.stats[e].device_error, HOUGH_DEVERR_TIMEOUT);
            mbar_wait_bounded(&s_bar, 0, kCopyWaitCycles);
            return;
        }
    }
    // one warp per strip of up to 256 cells of a row, lane t taking cells t, t + 32, ...: a layer's
    // bit of cell j is the comparison of bucket entry j + I alone, so each of the lane's loads is
    // one 8-byte entry and a warp's loads cover consecutive entries
    constexpr int kCells = 8;
    uint16_t *M = w.M + (int64_t)e * ax.n_qpt * nphi;
    const int kc = min(kCells, p.cols >> 5);   // cells per lane (cols is a multiple of 64)
    const int strip = kc * 32;
    const int per_row = p.cols / strip;
    const int nstrips = nrows * per_row;
    const int lane = threadIdx.x & 31;
    for (int sidx = threadIdx.x >> 5; sidx < nstrips; sidx += TPB / 32) {
        const int rr = sidx / per_row;
        const int jb = c0 + (sidx - rr * per_row) * strip + lane;
        const unsigned vm = rowMask[rr];
        const int *rI = rowI + rr * 16;
        const unsigned *rG = rowG + rr * 16;
        unsigned mask[kCells];
#pragma unroll
        for (int c = 0; c < kCells; ++c) mask[c] = 0u;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            if (!((vm >> l) & 1u)) continue;   // the same for the whole warp: the row's layers
            const int I = rI[l];
            const unsigned gb = rG[l], ngb = ~gb;
            if ((staged >> l) & 1u) {
                const uint2 *src = win + (int64_t)l * p.cap + (jb + I - s_wbase[l]);   // inside the window
#pragma unroll
                for (int c = 0; c < kCells; ++c)
                    if (c < kc) {
                        const uint2 v = src[32 * c];
                        mask[c] |= (unsigned)((v.x > gb) | (v.y > ngb)) << l;
                    }
            } else {
                const uint2 *src = prof + (int64_t)l * pstride;
#pragma unroll
                for (int c = 0; c < kCells; ++c)
                    if (c < kc) {
                        const uint2 v = __ldg(&src[wrap_col(jb + 32 * c + I, nphi)]);
                        mask[c] |= (unsigned)((v.x > gb) | (v.y > ngb)) << l;
                    }
            }
        }
        uint16_t *row = M + (int64_t)(i0 + rr) * nphi + jb;
#pragma unroll
        for (int c = 0; c < kCells; ++c)
            if (c < kc) row[32 * c] = (uint16_t)mask[c];
    }
}


// Fused vote and peak search (vote_mode HOUGH_VOTE_FUSED): a CTA per band of band_rows full rows.
// A cell of a layer of one radius is a function of its row's table entry and two bucket-profile
// entries alone, so the CTA computes the band's masks and those of the row above and below it
// (the 3 x 3 neighbourhoods; phi wraps within the full rows) into shared memory, searches the
// band for peaks there and writes the band's candidate list and count as the peak kernel does --
// the accumulator never goes to device memory.  Full rows read every bucket of a layer, so when
// they fit (STAGE) the voting layers' whole profiles are first copied into shared memory with
// bulk asynchronous copies; otherwise they are read through the cache.  When a present layer's
// hits lie at several radii the scatter kernel adds that layer's votes afterwards: the CTA then
// writes the band's rows to the accumulator instead, and the peak kernel searches it.

__device__ __forceinline__ bool all_layers_uniform(const Axes &ax, const Workspace &w)
{
    for (int l = 0; l < ax.n_layers; ++l) {
        const LayerInfo li = w.info[l];
        if (li.present && !li.uniform) return false;
    }
    return true;
}

template <int NL, int TPB, bool STAGE>
__global__ void __launch_bounds__(TPB) fused_kernel(GatherParams p)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char fused_smem[];
    __shared__ int rowI[kGatherRowsMax * 16];
    __shared__ unsigned rowG[kGatherRowsMax * 16];
    __shared__ unsigned rowMask[kGatherRowsMax];
    __shared__ __align__(8) uint64_t s_bar;
    const Axes &ax = p.ax;
    const Workspace &w = p.w;
    const int nb = p.tiles_per_event;
    const int e = blockIdx.x / nb, band = blockIdx.x - e * nb;
    const int R = p.rows, i0 = band * R;
    const int nrows = min(R, ax.n_qpt - i0);
    const int L = ax.n_layers, nphi = ax.n_phi;
    const bool search = all_layers_uniform(ax, w);
    // computed rows: i0 - 1 .. i0 + nrows (halo included) when searching, else the band's own
    const int first = search ? i0 - 1 : i0;
    const int S = search ? nrows + 2 : nrows;
    for (int q = threadIdx.x; q < ((S * 16 + 31) & ~31); q += TPB) {
        const int s = q >> 4, l = q & 15, i = first + s;
        int I = 0;
        unsigned gb = 0u, valid = 0u;
        if (l < L && s < S && i >= 0 && i < ax.n_qpt) {   // rows outside the grid hold no votes
            const LayerInfo li = w.info[l];
            const TabEntry te = w.tab[l * ax.n_qpt + i];   // requested with the layer record: one round trip
            if (li.present && li.uniform && i >= li.lo && i <= li.hi) {
                if (te.I != kNoVote) {
                    I = te.I;
                    gb = __float_as_uint(te.g);
                    valid = 1u;
                }
            }
        }
        const unsigned m = __ballot_sync(0xFFFFFFFFu, valid) >> (threadIdx.x & 16);
        rowI[q] = I;
        rowG[q] = gb;
        if ((threadIdx.x & 15) == 0) rowMask[s] = m & 0xFFFFu;
    }
    __syncthreads();
    constexpr bool stage = STAGE;
    const uint2 *prof = w.prof + (int64_t)e * prof_event_entries(ax);
    const int pstride = prof_stride(ax);
    uint2 *win = reinterpret_cast<uint2 *>(fused_smem);   // staged: layer l's profile at l * n_phi
    uint16_t *tm = reinterpret_cast<uint16_t *>(fused_smem + (stage ? (size_t)L * nphi * sizeof(uint2) : 0));
    unsigned used = 0u;   // layers voting on any computed row
    for (int q = 0; q < S; ++q) used |= rowMask[q];
    if (stage && used) {
        if (threadIdx.x == 0) mbar_init(&s_bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_expect(&s_bar, (unsigned)__popc(used) * (unsigned)nphi * 8u);
            for (int l = 0; l < L; ++l)
                if ((used >> l) & 1u)
                    bulk_copy_g2s(win + (int64_t)l * nphi, prof + (int64_t)l * pstride, 8u * (unsigned)nphi, &s_bar);
        }
        const bool ok = first_copy_wait(w, &s_bar);
        if (!__syncthreads_and(ok)) {
            // the copies did not land in time: report it, give them one more bound, find nothing
            if (threadIdx.x == 0) {
                atomicOr(&w.stats[e].device_error, HOUGH_DEVERR_TIMEOUT);
                if (search) w.band_counts[(int64_t)e * nb + band] = 0;
            }
            mbar_wait_bounded(&s_bar, 0, kCopyWaitCycles);
            return;
        }
    }
    // a warp per strip of 256 cells of a row (the last strip of a row may be shorter: n_phi is a
    // multiple of 64), lane t taking cells t, t + 32, ...; a layer's bit of cell j compares the
    // profile entry j + I of that layer
    constexpr int kCells = 8;
    const int per_row = (nphi + 32 * kCells - 1) / (32 * kCells);
    const int lane = threadIdx.x & 31;
    for (int sidx = threadIdx.x >> 5; sidx < S * per_row; sidx += TPB / 32) {
        const int s = sidx / per_row;
        const int jb = (sidx - s * per_row) * 32 * kCells + lane;
        const unsigned vm = rowMask[s];
        unsigned mask[kCells];
#pragma unroll
        for (int c = 0; c < kCells; ++c) mask[c] = 0u;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            if (!((vm >> l) & 1u)) continue;   // the same for the whole warp: the row's layers
            const int I = rowI[s * 16 + l];
            const unsigned gb = rowG[s * 16 + l], ngb = ~gb;
            if (stage) {
                const uint2 *src = win + (int64_t)l * nphi;
#pragma unroll
                for (int c = 0; c < kCells; ++c)
                    if (jb + 32 * c < nphi) {
                        const uint2 v = src[wrap_col(jb + 32 * c + I, nphi)];
                        mask[c] |= (unsigned)((v.x > gb) | (v.y > ngb)) << l;
                    }
            } else {
                const uint2 *src = prof + (int64_t)l * pstride;
#pragma unroll
                for (int c = 0; c < kCells; ++c)
                    if (jb + 32 * c < nphi) {
                        const uint2 v = __ldg(&src[wrap_col(jb + 32 * c + I, nphi)]);
                        mask[c] |= (unsigned)((v.x > gb) | (v.y > ngb)) << l;
                    }
            }
        }
#pragma unroll
        for (int c = 0; c < kCells; ++c)
            if (jb + 32 * c < nphi) tm[s * nphi + jb + 32 * c] = (uint16_t)mask[c];
    }
    __syncthreads();
    if (!search) {
        // the scatter adds the other layers' votes: hand the band's rows to the peak kernel
        uint16_t *M = w.M + (int64_t)e * ax.n_qpt * nphi;
        const int v8 = nphi >> 3;
        for (int q = threadIdx.x; q < nrows * v8; q += TPB) {
            const int rr = q / v8, c8 = q - rr * v8;
            *reinterpret_cast<uint4 *>(M + (int64_t)(i0 + rr) * nphi + c8 * 8) =
                *reinterpret_cast<const uint4 *>(tm + rr * nphi + c8 * 8);
        }
        return;
    }
    uint2 *out = w.band_cands + ((int64_t)e * nb + band) * w.band_cap;
    const int cnt = band_peak_search<TPB, uint16_t, false, true>(tm, nrows, i0, nphi, ax.threshold, nullptr, out,
                                                                 w.band_cap);
    if (threadIdx.x == 0) w.band_counts[(int64_t)e * nb + band] = cnt;
}

// Count accumulator by gather.  On row i a layer of one radius adds to cell j the hits of bucket
// J' = (j + I_i) mod Nphi with f >= g_i and the hits of bucket J' + 1 with f < g_i: exactly the
// hits whose vote J - I_i - (f < g_i) is j, by the same FP32 comparison, so the same counts as the
// scatter -- with no atomics.  A CTA owns `rows` x `cols` cells.  It first stages, for every layer
// at once, the window of buckets its tile reads: the buckets' offsets (the bucket offsets are a
// prefix sum already, so a window's are a difference of two, or three when it wraps around phi)
// and the f values of their hits (the sorted hits of consecutive buckets are contiguous: one
// range, or two when the window wraps).  Then a lane per cell sums, over the layers, the hits of
// the two buckets its cell reads, and writes the saturated count.  A window too wide or too full
// for its slot is read from global memory.  Layers whose hits lie at several radii are added by
// the scatter kernel afterwards.
constexpr int kCountWinPad = 128;    // window buckets beyond cols + 2 held in a layer's slot
constexpr int kCountSmemBudget = 96 * 1024;

__host__ __device__ inline int count_win_cap(int cols) { return cols + 2 + kCountWinPad; }

template <int TPB>
__global__ void __launch_bounds__(TPB) gather_count_kernel(GatherParams p, int fcap)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char count_smem[];
    __shared__ int rowI[kGatherRowsMax * 16];
    __shared__ float rowG[kGatherRowsMax * 16];
    __shared__ unsigned rowMask[kGatherRowsMax];
    __shared__ int s_lo[HOUGH_MAX_LAYERS], s_len[HOUGH_MAX_LAYERS], s_a[HOUGH_MAX_LAYERS];
    __shared__ int s_total[HOUGH_MAX_LAYERS], s_first[HOUGH_MAX_LAYERS], s_fbase[HOUGH_MAX_LAYERS];
    __shared__ unsigned s_staged;
    const Axes &ax = p.ax;
    const Workspace &w = p.w;
    const int e = blockIdx.x / p.tiles_per_event;
    const int t = blockIdx.x - e * p.tiles_per_event;
    const int rt = t / p.col_tiles, ct = t - rt * p.col_tiles;
    const int i0 = rt * p.rows, c0 = ct * p.cols;
    const int nrows = min(p.rows, ax.n_qpt - i0);
    const int C = p.cols, L = ax.n_layers, nphi = ax.n_phi;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wcap = count_win_cap(C);
    int *bpre = reinterpret_cast<int *>(count_smem);          // L slots of wcap + 1 bucket offsets
    float *fs = reinterpret_cast<float *>(bpre + L * (wcap + 1));   // fcap f values, layer after layer
    const int64_t hstart = w.hit_start[e];
    const float *fsort = w.fsort + hstart;
    const int32_t *offs = w.offs + (int64_t)e * (n_keys(ax) + 1);

    for (int q = threadIdx.x; q < ((p.rows * 16 + 31) & ~31); q += TPB) {
        const int rr = q >> 4, l = q & 15, i = i0 + rr;
        int I = 0;
        float g = 0.f;
        unsigned valid = 0u;
        if (l < L && rr < nrows) {
            const LayerInfo li = w.info[l];
            const TabEntry te = w.tab[l * ax.n_qpt + i];   // requested with the layer record: one round trip
            if (li.present && li.uniform && i >= li.lo && i <= li.hi) {
                if (te.I != kNoVote) {
                    I = te.I;
                    g = te.g;
                    valid = 1u;
                }
            }
        }
        const unsigned m = __ballot_sync(0xFFFFFFFFu, valid) >> (threadIdx.x & 16);
        rowI[q] = I;
        rowG[q] = g;
        if ((threadIdx.x & 15) == 0) rowMask[rr] = m & 0xFFFFu;
    }
    __syncthreads();
    // each layer's window: buckets [c0 + min I, c0 + C + max I] over the rows it votes on
    if (threadIdx.x < HOUGH_MAX_LAYERS) {
        const int l = threadIdx.x;
        int lo = INT_MAX, hi = INT_MIN, len = 0, a = 0, total = 0, first = 0;
        if (l < L) {
            for (int rr = 0; rr < nrows; ++rr)
                if ((rowMask[rr] >> l) & 1u) {
                    lo = min(lo, rowI[rr * 16 + l]);
                    hi = max(hi, rowI[rr * 16 + l]);
                }
            if (lo <= hi) {
                len = C + 2 + (hi - lo);   // buckets J' and J' + 1 of every cell
                a = wrap_col(c0 + lo, nphi);
                if (len <= wcap && len <= nphi) {   // one pass over the ring at most
                    const int32_t *lofs = offs + l * nphi;
                    const int end = a + len;          // unwrapped end bucket
                    first = end <= nphi ? lofs[end] - lofs[a] : lofs[nphi] - lofs[a];
                    total = first + (end <= nphi ? 0 : lofs[end - nphi] - lofs[0]);
                } else {
                    len = -len;   // not staged
                }
            }
        }
        s_lo[l] = lo;
        s_len[l] = len;
        s_a[l] = a;
        s_total[l] = total;
        s_first[l] = first;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned staged = 0u;
        int fbase = 0;
        for (int l = 0; l < L; ++l) {
            s_fbase[l] = fbase;
            if (s_len[l] > 0 && fbase + s_total[l] <= fcap) {
                staged |= 1u << l;
                fbase += s_total[l];
            }
        }
        s_staged = staged;
    }
    __syncthreads();
    const unsigned staged = s_staged;
    // staging: every staged layer's bucket offsets (relative to its f values) and f values
    for (int l = 0; l < L; ++l) {
        if (!((staged >> l) & 1u)) continue;
        const int32_t *lofs = offs + l * nphi;
        const int a = s_a[l], len = s_len[l], first = s_first[l], total = s_total[l], fb = s_fbase[l];
        int *bp = bpre + l * (wcap + 1);
        for (int q = threadIdx.x; q <= len; q += TPB) {
            const int J = a + q;   // unwrapped
            bp[q] = fb + (J <= nphi ? lofs[J] - lofs[a] : first + lofs[J - nphi] - lofs[0]);
        }
        for (int q = threadIdx.x; q < total; q += TPB)
            fs[fb + q] = q < first ? fsort[lofs[a] + q] : fsort[lofs[0] + (q - first)];
    }
    __syncthreads();
    // a lane per cell, 32 cells of one row per warp pass, every layer summed in a register
    uint16_t *M = w.M + (int64_t)e * ax.n_qpt * nphi;
    const int per_row = C >> 5;
    for (int task = warp; task < nrows * per_row; task += TPB / 32) {
        const int rr = task / per_row;
        const int c = (task - rr * per_row) * 32 + lane;
        const unsigned vm = rowMask[rr];
        uint32_t count = 0;
        for (int l = 0; l < L; ++l) {
            if (!((vm >> l) & 1u)) continue;   // the same for the whole warp: the row's layers
            const int I = rowI[rr * 16 + l];
            const float g = rowG[rr * 16 + l];
            if ((staged >> l) & 1u) {
                const int *bp = bpre + l * (wcap + 1) + (c + I - s_lo[l]);   // bucket J' of the window
                const int s0 = bp[0], s1 = bp[1], s2 = bp[2];
                for (int q = s0; q < s1; ++q) count += fs[q] < g ? 0u : 1u;
                for (int q = s1; q < s2; ++q) count += fs[q] < g ? 1u : 0u;
            } else {
                const int32_t *lofs = offs + l * nphi;
                const int J0 = wrap_col(c0 + c + I, nphi), J1 = wrap_col(c0 + c + I + 1, nphi);
                for (int q = lofs[J0]; q < lofs[J0 + 1]; ++q) count += fsort[q] < g ? 0u : 1u;
                for (int q = lofs[J1]; q < lofs[J1 + 1]; ++q) count += fsort[q] < g ? 1u : 0u;
            }
        }
        // saturated to 16 bits; even lanes store their cell and the next one as one word
        const uint32_t v = min(count, 65535u);
        const uint32_t next = __shfl_down_sync(0xFFFFFFFFu, v, 1);
        if (!(lane & 1))
            *reinterpret_cast<uint32_t *>(M + (int64_t)(i0 + rr) * nphi + c0 + c) = v | (next << 16);
    }
}

__device__ void compact_if_last(const Axes &ax, const Workspace &w, void *buf, size_t buf_bytes);

// A context's bucket profile is read for the last time by the vote, which the peak search follows:
// zero it here for the next event (Workspace::recycle).
__device__ __forceinline__ void recycle_profile(const Axes &ax, const Workspace &w)
{
    if (!w.recycle || !w.prof) return;
    uint4 *p4 = reinterpret_cast<uint4 *>(w.prof);
    const int64_t n4 = (int64_t)w.n_events * prof_event_entries(ax) / 2;   // two entries a vector
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x)
        p4[q] = make_uint4(0u, 0u, 0u, 0u);
}

// Peak search of one band of band_rows rows from the accumulator (plus a halo row on each side).
// COUNTS: the cells are vote counts, staged as they are (2 bytes each); otherwise layer masks,
// staged as their layer counts (1 byte each).
template <bool COUNTS>
__global__ void __launch_bounds__(kPeakThreads) peaks_kernel(Axes ax, Workspace w)
{
    pdl_enter();
    recycle_profile(ax, w);
    if (!COUNTS && w.fused && all_layers_uniform(ax, w)) return;   // the fused vote searched the bands
    extern __shared__ __align__(16) unsigned char pc[];
    const int R = w.band_rows;
    const int nb = n_bands(ax, R);
    const int e = blockIdx.x / nb, band = blockIdx.x - e * nb;
    const int nphi = ax.n_phi;
    const int i0 = band * R;
    const int nrows = min(R, ax.n_qpt - i0);
    const uint16_t *M = w.M + (int64_t)e * ax.n_qpt * nphi;
    const int v8 = nphi >> 3;
    uint2 *out = w.band_cands + ((int64_t)e * nb + band) * w.band_cap;
    if (COUNTS) {
        uint16_t *pv = reinterpret_cast<uint16_t *>(pc);
        for (int q = threadIdx.x; q < (nrows + 2) * v8; q += kPeakThreads) {
            const int rr = q / v8, c8 = q - rr * v8;
            const int i = i0 - 1 + rr;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (i >= 0 && i < ax.n_qpt) v = *reinterpret_cast<const uint4 *>(M + (int64_t)i * nphi + c8 * 8);
            *reinterpret_cast<uint4 *>(pv + rr * nphi + c8 * 8) = v;
        }
        __syncthreads();
        const int cnt = band_peak_search<kPeakThreads>(pv, nrows, i0, nphi, ax.threshold, M, out, w.band_cap);
        if (threadIdx.x == 0) w.band_counts[(int64_t)e * nb + band] = cnt;
        __syncthreads();   // the band buffer is free
        compact_if_last(ax, w, pc, band_smem_bytes(ax, R));
        return;
    }
    uint16_t *pm = reinterpret_cast<uint16_t *>(pc + (size_t)(R + 2) * nphi);   // the band's own rows' masks
    for (int q = threadIdx.x; q < (nrows + 2) * v8; q += kPeakThreads) {
        const int rr = q / v8, c8 = q - rr * v8;
        const int i = i0 - 1 + rr;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (i >= 0 && i < ax.n_qpt) v = *reinterpret_cast<const uint4 *>(M + (int64_t)i * nphi + c8 * 8);
        if (rr >= 1 && rr <= nrows) *reinterpret_cast<uint4 *>(pm + (rr - 1) * nphi + c8 * 8) = v;
        const uint32_t words[4] = {v.x, v.y, v.z, v.w};
        uint32_t packed[2] = {0u, 0u};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t lo = (uint32_t)__popc(words[u] & 0xFFFFu), hi = (uint32_t)__popc(words[u] >> 16);
            packed[u >> 1] |= (lo | (hi << 8)) << ((u & 1) * 16);
        }
        *reinterpret_cast<uint2 *>(pc + rr * nphi + c8 * 8) = make_uint2(packed[0], packed[1]);
    }
    __syncthreads();
    const int cnt = band_peak_search<kPeakThreads, unsigned char, false, false, true>(pc, nrows, i0, nphi, ax.threshold,
                                                                                     pm, out, w.band_cap);
    if (threadIdx.x == 0) w.band_counts[(int64_t)e * nb + band] = cnt;
    __syncthreads();   // the band buffer is free
    compact_if_last(ax, w, pc, band_smem_bytes(ax, R));
}

// Peak search of one band of band_rows q/pT rows of one d0 slice m of a grid with a d0 axis: the
// rows of its cells' 3 x 3 x 3 blocks -- rows i0 - 1 .. i0 + nrows of slices m - 1, m, m + 1 --
// are staged as cell values (layer counts as bytes, or 16-bit counts), rows outside the slice and
// slices outside the grid as empty.  Bands never cross a slice, so the band lists concatenate in
// raster order.
template <bool COUNTS>
__global__ void __launch_bounds__(kPeakThreads) peaks3_kernel(Axes ax, Workspace w)
{
    pdl_enter();
    recycle_profile(ax, w);
    extern __shared__ __align__(16) unsigned char pc[];
    const int R = w.band_rows, Q = ax.q_rows;
    const int bps = (Q + R - 1) / R;   // bands per slice
    const int nb = n_bands(ax, R);
    const int e = blockIdx.x / nb, band = blockIdx.x - e * nb;
    const int m = band / bps, i0 = (band - m * bps) * R;
    const int nrows = min(R, Q - i0);
    const int S = nrows + 2;
    const int nphi = ax.n_phi;
    const uint16_t *M = w.M + (int64_t)e * ax.n_qpt * nphi;
    const int v8 = nphi >> 3;
    for (int q = threadIdx.x; q < 3 * S * v8; q += kPeakThreads) {
        const int sidx = q / v8, c8 = q - sidx * v8;
        const int slice = sidx / S;
        const int mm = m + slice - 1, ii = i0 - 1 + (sidx - slice * S);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (mm >= 0 && mm < ax.n_d0 && ii >= 0 && ii < Q)
            v = *reinterpret_cast<const uint4 *>(M + (int64_t)(mm * Q + ii) * nphi + c8 * 8);
        if (COUNTS) {
            *reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(pc) + sidx * nphi + c8 * 8) = v;
        } else {
            const uint32_t words[4] = {v.x, v.y, v.z, v.w};
            uint32_t packed[2] = {0u, 0u};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t lo = (uint32_t)__popc(words[u] & 0xFFFFu), hi = (uint32_t)__popc(words[u] >> 16);
                packed[u >> 1] |= (lo | (hi << 8)) << ((u & 1) * 16);
            }
            *reinterpret_cast<uint2 *>(pc + sidx * nphi + c8 * 8) = make_uint2(packed[0], packed[1]);
        }
    }
    __syncthreads();
    uint2 *out = w.band_cands + ((int64_t)e * nb + band) * w.band_cap;
    const int row0 = m * Q + i0;   // stacked row of the band's first row
    int cnt;
    if (COUNTS)
        cnt = band_peak_search<kPeakThreads, uint16_t, true>(reinterpret_cast<const uint16_t *>(pc), nrows, row0, nphi,
                                                             ax.threshold, M, out, w.band_cap);
    else
        cnt = band_peak_search<kPeakThreads, unsigned char, true>(pc, nrows, row0, nphi, ax.threshold, M, out,
                                                                  w.band_cap);
    if (threadIdx.x == 0) w.band_counts[(int64_t)e * nb + band] = cnt;
    __syncthreads();   // the band buffer is free
    compact_if_last(ax, w, pc, band_smem_bytes(ax, R));
}

// One event's candidate list: exclusive scan of the band counts, then the band lists concatenated
// into the raster-ordered candidate list (the first max_cand of them).  With the band offsets in
// shared memory every thread copies candidates by their index (the band found by binary search
// over the offsets), so the copy costs one round trip however the candidates fall into bands.
// `parts` CTAs may share an event, each copying its slice (this one is `part`); part 0 also records
// the event's totals (and handles band counts too many to stage).  `single`: the batch is one
// event, whose flattened candidate base this CTA then writes itself.  Called by all TPB threads.
// The band offsets are staged in shared memory when they fit (`offs_smem`, `offs_cap` entries);
// otherwise they go through device memory and a warp copies a band at a time.
constexpr int kCompactSmemBands = 4096;

template <int TPB>
__device__ void compact_event(const Axes &ax, const Workspace &w, int e, int part, int parts, int single,
                              int *s_offs, int offs_cap)
{
    __shared__ int s_warp[TPB / 32];
    const int nb = n_bands(ax, w.band_rows);
    const bool staged = nb + 1 <= offs_cap;
    const int32_t *counts = w.band_counts + (int64_t)e * nb;
    int32_t *offs = w.band_offs + (int64_t)e * nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int chunk = (nb + TPB - 1) / TPB;
    const int k0 = min(nb, (int)threadIdx.x * chunk), k1 = min(nb, k0 + chunk);
    int sum = 0;
    for (int k = k0; k < k1; ++k) sum += counts[k];
    int incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int wv = lane < TPB / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, wv, d);
            if (lane >= d) wv += t;
        }
        if (lane < TPB / 32) s_warp[lane] = wv;
    }
    __syncthreads();
    int run = (warp > 0 ? s_warp[warp - 1] : 0) + incl - sum;
    for (int k = k0; k < k1; ++k) {
        if (staged) s_offs[k] = run;
        else if (part == 0) offs[k] = run;
        run += counts[k];
    }
    const int total = s_warp[TPB / 32 - 1];
    const int kept = min(total, w.max_cand);
    if (part == 0 && threadIdx.x == 0) {
        w.stats[e].n_candidates = (unsigned)total;
        if (total > w.max_cand) atomicOr(&w.stats[e].device_error, HOUGH_DEVERR_CAND);
        if (single) {
            w.cand_base[0] = 0;
            w.cand_base[1] = kept;
            w.counters->total_cands = (unsigned)kept;
        }
    }
    __syncthreads();
    hough_candidate *cands = w.cands + (int64_t)e * w.max_cand;
    const uint2 *lists = w.band_cands + (int64_t)e * nb * w.band_cap;
    auto emit = [&](int c, uint2 v) {
        hough_candidate cd;
        cd.iq = v.x / (unsigned)ax.n_phi;
        cd.jphi = v.x % (unsigned)ax.n_phi;
        cd.mask = v.y;
        cd.n_members = 0u;
        cd.icot = cd.jz0 = cd.mask2 = cd.flags = 0u;
        cands[c] = cd;
    };
    if (staged) {
        const int per = (kept + parts - 1) / parts;
        const int c_end = min(kept, (part + 1) * per);
        for (int c = part * per + threadIdx.x; c < c_end; c += TPB) {
            // the band holding candidate c: the last b with offs[b] <= c (empty bands share offsets)
            int lo = 0, hi = nb - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_offs[mid] <= c) lo = mid; else hi = mid - 1;
            }
            emit(c, lists[(int64_t)lo * w.band_cap + (c - s_offs[lo])]);
        }
        return;
    }
    if (part != 0) return;
    __syncthreads();   // the offsets in device memory are complete
    for (int b = warp; b < nb; b += TPB / 32) {
        const int n = counts[b], o = offs[b];
        for (int k = lane; k < n; k += 32) {
            const int c = o + k;
            if (c >= w.max_cand) break;
            emit(c, lists[(int64_t)b * w.band_cap + k]);
        }
    }
}

__global__ void __launch_bounds__(kCompactThreads) compact_kernel(Axes ax, Workspace w, int single, int parts)
{
    pdl_enter();
    __shared__ int s_offs[kCompactSmemBands + 1];
    compact_event<kCompactThreads>(ax, w, blockIdx.x / parts, blockIdx.x % parts, parts, single, s_offs,
                                   kCompactSmemBands + 1);
}

// One event in one context: the CTA of the peak search that finishes last compacts the candidate
// list itself, saving the launch of the compaction (the band counts and lists of every CTA are
// visible to it after their fences).  Its band buffer (`buf`, `buf_bytes`), no longer needed,
// holds the band offsets.
__device__ void compact_if_last(const Axes &ax, const Workspace &w, void *buf, size_t buf_bytes)
{
    __shared__ int s_last;
    if (!w.compact_in_peaks) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&w.counters->peaks_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    compact_event<kPeakThreads>(ax, w, 0, 0, 1, 1, static_cast<int *>(buf), (int)(buf_bytes / sizeof(int)));
    if (threadIdx.x == 0) w.counters->peaks_done = 0u;   // ready for the next event
}

// One CTA: the first flattened candidate index of every event (kept candidates only), so that
// later kernels can spread all events' candidates over the whole device.
__global__ void __launch_bounds__(kCompactThreads) cand_scan_kernel(Workspace w)
{
    pdl_enter();
    __shared__ int s_warp[kCompactThreads / 32];
    __shared__ int s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < w.n_events; base += kCompactThreads) {
        const int e = base + threadIdx.x;
        const int v = e < w.n_events ? (int)min((unsigned)w.max_cand, w.stats[e].n_candidates) : 0;
        int incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int sv = s_warp[lane];
            int si = sv;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(0xFFFFFFFFu, si, d);
                if (lane >= d) si += t;
            }
            s_warp[lane] = si - sv;
        }
        __syncthreads();
        const int excl = s_carry + s_warp[warp] + incl - v;
        if (e < w.n_events) w.cand_base[e] = excl;
        __syncthreads();
        if (threadIdx.x == kCompactThreads - 1) s_carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        w.cand_base[w.n_events] = s_carry;
        w.counters->total_cands = (unsigned)s_carry;
    }
}

// All events' candidate lists, concatenated in event order into `out` (positions from cand_base).
// (the first `limit` to `out`, the rest -- when `rest` is given -- to rest at the same index)
// When `stats_out` is given, block 0 also copies the first event's counters there.
__global__ void pack_candidates_kernel(Workspace w, hough_candidate *out, long long limit, hough_candidate *rest,
                                       DevStats *stats_out)
{
    pdl_enter();
    static_assert(sizeof(DevStats) % 4 == 0, "the counters are copied as 32-bit words");
    if (stats_out && blockIdx.x == 0) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(w.stats);
        uint32_t *dst = reinterpret_cast<uint32_t *>(stats_out);
        for (int q = threadIdx.x; q < (int)(sizeof(DevStats) / 4); q += blockDim.x) dst[q] = src[q];
    }
    const int total = w.cand_base[w.n_events];
    const int n = rest ? total : (int)min((long long)total, limit);
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < n; f += gridDim.x * blockDim.x) {
        const int e = upper_index(w.cand_base, w.n_events, f);
        const hough_candidate cd = w.cands[(int64_t)e * w.max_cand + (f - w.cand_base[e])];
        if (f < limit) out[f] = cd;
        else rest[f] = cd;
    }
}

template <int TPB, bool GENERAL_ONLY, int CELL>
cudaError_t launch_scatter(const VoteParams &p, size_t smem, int grid, cudaStream_t stream)
{
    cudaError_t err = cudaFuncSetAttribute(scatter_kernel<TPB, GENERAL_ONLY, CELL>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err) return err;
    return launch_chained(scatter_kernel<TPB, GENERAL_ONLY, CELL>, dim3(grid), dim3(TPB), smem, stream, p);
}

template <bool GENERAL_ONLY, int CELL>
cudaError_t launch_scatter_tpb(const VoteParams &p, int threads, size_t smem, int grid, cudaStream_t stream)
{
    switch (threads) {
    case 128: return launch_scatter<128, GENERAL_ONLY, CELL>(p, smem, grid, stream);
    case 256: return launch_scatter<256, GENERAL_ONLY, CELL>(p, smem, grid, stream);
    case 512: return launch_scatter<512, GENERAL_ONLY, CELL>(p, smem, grid, stream);
    case 1024: return launch_scatter<1024, GENERAL_ONLY, CELL>(p, smem, grid, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// Bucket-offset slots of every layer, then the f values (at least 16 KB, the rest of the budget).
static size_t gather_count_base_bytes(const Axes &ax, const Tiling &t)
{
    return (size_t)ax.n_layers * (count_win_cap(t.gather_cols) + 1) * 4;
}

size_t gather_count_smem_bytes(const Axes &ax, const Tiling &t)
{
    const size_t base = gather_count_base_bytes(ax, t);
    const size_t fbytes = base + 16384 > (size_t)kCountSmemBudget ? 16384 : (size_t)kCountSmemBudget - base;
    return base + fbytes;
}

// Shared memory of the scatter kernel: the column-major tile, the slab's table rows and q/pT centres,
// then a 32-hit buffer and a queue of FP64 votes per warp.  wide: a 32-bit word a cell.
static size_t scatter_smem_bytes(const Axes &ax, const Tiling &t, bool wide)
{
    return scatter_hit_offset(t.tile_qpt, t.tile_phi, ax.n_layers, wide) + (size_t)t.threads * sizeof(uint4) +
           (size_t)(t.threads / 32) * kRefineQueue * sizeof(uint2) + 32 * sizeof(uint32_t);
}

// The smallest form the tile can take: two 16-bit masks a word, or 32-bit counters.
size_t vote_smem_bytes(const Axes &ax, const Tiling &t) { return scatter_smem_bytes(ax, t, ax.counts != 0); }


static VoteParams vote_params(const Axes &ax, const Workspace &w, const Tiling &t, float refine_eps)
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
    return p;
}

template <int NL>
cudaError_t launch_gather_nl(const GatherParams &p, int threads, size_t smem, int blocks, cudaStream_t stream)
{
    cudaError_t err;
    switch (threads) {
    case 256:
        if ((err = cudaFuncSetAttribute(gather_kernel<NL, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return err;
        return launch_chained(gather_kernel<NL, 256>, dim3(blocks), dim3(256), smem, stream, p);
    case 1024:
        if ((err = cudaFuncSetAttribute(gather_kernel<NL, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return err;
        return launch_chained(gather_kernel<NL, 1024>, dim3(blocks), dim3(1024), smem, stream, p);
    default:
        if ((err = cudaFuncSetAttribute(gather_kernel<NL, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return err;
        return launch_chained(gather_kernel<NL, 512>, dim3(blocks), dim3(512), smem, stream, p);
    }
}

size_t fused_smem_bytes(const Axes &ax, int band_rows)
{
    return (size_t)(band_rows + 2) * ax.n_phi * sizeof(uint16_t);
}

// Whether the fused kernel's CTA also holds every layer's whole bucket profile (8 bytes a bucket)
// beside its masks and row tables.
bool fused_stages_profiles(const Axes &ax, int band_rows)
{
    static std::atomic<int> optin{0};
    int m = optin.load(std::memory_order_relaxed);
    if (!m) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&m, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
        optin.store(m, std::memory_order_relaxed);
    }
    return fused_smem_bytes(ax, band_rows) + (size_t)ax.n_layers * ax.n_phi * sizeof(uint2) + 6144 + 1024 <= (size_t)m;
}

size_t gather_smem_bytes(const Axes &ax, const Tiling &t)
{
    return (size_t)ax.n_layers * (size_t)(t.gather_cols + 64) * sizeof(uint2);
}

static cudaError_t launch_gather_tiled(const Axes &ax, const Workspace &w, const Tiling &t, cudaStream_t stream)
{
    GatherParams p;
    p.ax = ax;
    p.w = w;
    p.rows = t.gather_rows;
    p.cols = t.gather_cols;
    p.cap = t.gather_cols + 64;
    p.col_tiles = ax.n_phi / p.cols;
    p.tiles_per_event = ((ax.n_qpt + p.rows - 1) / p.rows) * p.col_tiles;
    const int blocks = w.n_events * p.tiles_per_event;
    const size_t smem = gather_smem_bytes(ax, t);
    // layer loops unrolled to the next multiple of four
    if (ax.n_layers <= 4) return launch_gather_nl<4>(p, t.gather_threads, smem, blocks, stream);
    if (ax.n_layers <= 8) return launch_gather_nl<8>(p, t.gather_threads, smem, blocks, stream);
    if (ax.n_layers <= 12) return launch_gather_nl<12>(p, t.gather_threads, smem, blocks, stream);
    return launch_gather_nl<16>(p, t.gather_threads, smem, blocks, stream);
}

template <int NL, int TPB>
cudaError_t launch_fused_tpb(const GatherParams &p, size_t smem, int blocks, cudaStream_t stream)
{
    auto kernel = p.cap ? fused_kernel<NL, TPB, true> : fused_kernel<NL, TPB, false>;
    cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err) return err;
    return launch_chained(kernel, dim3(blocks), dim3(TPB), smem, stream, p);
}

template <int NL>
cudaError_t launch_fused_nl(const GatherParams &p, int threads, size_t smem, int blocks, cudaStream_t stream)
{
    switch (threads) {
    case 256: return launch_fused_tpb<NL, 256>(p, smem, blocks, stream);
    case 1024: return launch_fused_tpb<NL, 1024>(p, smem, blocks, stream);
    default: return launch_fused_tpb<NL, 512>(p, smem, blocks, stream);
    }
}

// One CTA per band of the peak search (w.band_rows full rows).
static cudaError_t launch_fused(const Axes &ax, const Workspace &w, const Tiling &t, cudaStream_t stream)
{
    GatherParams p;
    p.ax = ax;
    p.w = w;
    p.rows = w.band_rows;
    p.cols = ax.n_phi;
    p.cap = fused_stages_profiles(ax, w.band_rows) ? 1 : 0;
    p.col_tiles = 1;
    p.tiles_per_event = n_bands(ax, w.band_rows);
    const int blocks = w.n_events * p.tiles_per_event;
    const size_t smem = fused_smem_bytes(ax, w.band_rows) + (p.cap ? (size_t)ax.n_layers * ax.n_phi * sizeof(uint2) : 0);
    if (ax.n_layers <= 4) return launch_fused_nl<4>(p, t.gather_threads, smem, blocks, stream);
    if (ax.n_layers <= 8) return launch_fused_nl<8>(p, t.gather_threads, smem, blocks, stream);
    if (ax.n_layers <= 12) return launch_fused_nl<12>(p, t.gather_threads, smem, blocks, stream);
    return launch_fused_nl<16>(p, t.gather_threads, smem, blocks, stream);
}

template <int TPB>
cudaError_t launch_gather_count_tpb(const GatherParams &p, size_t smem, int fcap, int blocks, cudaStream_t stream)
{
    cudaError_t err = cudaFuncSetAttribute(gather_count_kernel<TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err) return err;
    return launch_chained(gather_count_kernel<TPB>, dim3(blocks), dim3(TPB), smem, stream, p, fcap);
}

cudaError_t launch_gather(const Axes &ax, const Workspace &w, const Tiling &t, cudaStream_t stream)
{
    if (t.vote_mode == HOUGH_VOTE_FUSED) return launch_fused(ax, w, t, stream);
    if (!ax.counts) return launch_gather_tiled(ax, w, t, stream);
    if (!w.fsort) return cudaErrorInvalidValue;   // the count gather reads the sorted f values
    GatherParams p;
    p.ax = ax;
    p.w = w;
    p.rows = t.gather_rows;
    p.cols = t.gather_cols;
    p.cap = 0;
    p.col_tiles = ax.n_phi / p.cols;
    p.tiles_per_event = ((ax.n_qpt + p.rows - 1) / p.rows) * p.col_tiles;
    const int blocks = w.n_events * p.tiles_per_event;
    const size_t smem = gather_count_smem_bytes(ax, t);
    const int fcap = (int)((smem - gather_count_base_bytes(ax, t)) / 4);
    switch (t.gather_threads) {
    case 256: return launch_gather_count_tpb<256>(p, smem, fcap, blocks, stream);
    case 1024: return launch_gather_count_tpb<1024>(p, smem, fcap, blocks, stream);
    default: return launch_gather_count_tpb<512>(p, smem, fcap, blocks, stream);
    }
}

cudaError_t launch_scatter(const Axes &ax, const Workspace &w, const Tiling &t, float refine_eps, bool general_only,
                           cudaStream_t stream)
{
    const VoteParams p = vote_params(ax, w, t, refine_eps);
    const int grid = w.n_events * p.tiles_per_event;
    if (ax.counts) {
        const size_t smem = scatter_smem_bytes(ax, t, true);
        return general_only ? launch_scatter_tpb<true, 2>(p, t.threads, smem, grid, stream)
                            : launch_scatter_tpb<false, 2>(p, t.threads, smem, grid, stream);
    }
    // a mask a word when that tile fits (no shift to place the bit), else two a word
    static std::atomic<int> optin{0};
    int m = optin.load(std::memory_order_relaxed);
    if (!m) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&m, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) m = 48 * 1024;
        optin.store(m, std::memory_order_relaxed);
    }
    const size_t wide = scatter_smem_bytes(ax, t, true);
    if (wide + 1024 <= (size_t)m)
        return general_only ? launch_scatter_tpb<true, 1>(p, t.threads, wide, grid, stream)
                            : launch_scatter_tpb<false, 1>(p, t.threads, wide, grid, stream);
    const size_t smem = scatter_smem_bytes(ax, t, false);
    return general_only ? launch_scatter_tpb<true, 0>(p, t.threads, smem, grid, stream)
                        : launch_scatter_tpb<false, 0>(p, t.threads, smem, grid, stream);
}

cudaError_t launch_vote(const Axes &ax, const Workspace &w, const Tiling &t, float refine_eps,
                        cudaStream_t stream)
{
    if (t.vote_mode == HOUGH_VOTE_SCATTER || (ax.counts && !w.fsort)) return launch_scatter(ax, w, t, refine_eps, false, stream);
    // gather every table layer (fused with the peak search under HOUGH_VOTE_FUSED), then let the
    // scatter kernel add the layers whose radii differ
    cudaError_t err = launch_gather(ax, w, t, stream);
    if (err) return err;
    return launch_scatter(ax, w, t, refine_eps, true, stream);
}


cudaError_t launch_band_peaks(const Axes &ax, const Workspace &w, const Tiling &t, cudaStream_t stream)
{
    const int nb = n_bands(ax, w.band_rows);
    const size_t smem = band_smem_bytes(ax, w.band_rows);
    auto kernel = ax.n_d0 ? (ax.counts ? peaks3_kernel<true> : peaks3_kernel<false>)
                          : (ax.counts ? peaks_kernel<true> : peaks_kernel<false>);
    cudaError_t err;
    if ((err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return err;
    if ((err = launch_chained(kernel, dim3(w.n_events * nb), dim3(kPeakThreads), smem, stream, ax, w))) return err;
    return cudaGetLastError();
}

cudaError_t launch_compact(const Axes &ax, const Workspace &w, cudaStream_t stream)
{
    const int single = w.n_events == 1;
    // about two CTAs per SM over all events (the copy of a dense event's tens of thousands of
    // candidates is latency-bound in one CTA)
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int parts = std::max(1, std::min(16, (2 * sms + w.n_events - 1) / w.n_events));
    cudaError_t err = launch_chained(compact_kernel, dim3(w.n_events * parts), dim3(kCompactThreads), 0, stream, ax, w,
                                     single, parts);
    if (!err && !single) err = launch_chained(cand_scan_kernel, dim3(1), dim3(kCompactThreads), 0, stream, w);
    return err;
}

cudaError_t launch_pack_candidates(const Axes &ax, const Workspace &w, hough_candidate *out, cudaStream_t stream,
                                   long long limit, hough_candidate *rest, DevStats *stats_out, int blocks)
{
    (void)ax;
    return launch_chained(pack_candidates_kernel, dim3(blocks), dim3(256), 0, stream, w, out, limit, rest, stats_out);
}

cudaError_t launch_peaks(const Axes &ax, const Workspace &w, const Tiling &t, cudaStream_t stream)
{
    cudaError_t err = launch_band_peaks(ax, w, t, stream);
    if (err) return err;
    return launch_compact(ax, w, stream);
}

}  // namespace hough
