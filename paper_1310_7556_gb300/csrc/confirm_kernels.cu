// Confirmation of the candidates (Sec. 4: candidates found as local maxima are confirmed by "more
// expensive computations"): for each candidate, the hits whose stage-1 vote fell in its cell
// (membership) and their vote in a (cot theta, z0) grid of layer masks (stage 2).
//
// Work scales with a candidate's votes, not with the size of the stage-2 grid.  Each confirming
// warp owns a clear n_cot x n_z0 grid in shared memory (16-bit masks; in batches of a detector of
// at most 10 layers, 10-bit masks three to a word, which lets more warps share an SM).  A member's z0 coordinate is linear in the
// cot row, so only a run of rows can vote inside the z0 range; the (member, row) pairs of all
// runs are spread over the lanes and voted with a shared atomicOr, whose returned word also
// judges the cell (stage2_vote): the arg-max falls out of the one pass.
//
// member_kernel (a warp per candidate, all events' candidates flattened) enumerates a candidate's
// members once, in a fixed order, into the event's member pool, and finishes stage 2 itself for
// candidates of up to kMemberCap members (in chunks of 32, one member per lane).  Larger
// candidates -- the saturated cells of very dense events -- are filed for stage2_large_kernel,
// a CTA each, which re-reads them from the pool (or re-enumerates them, when the pool overflowed)
// in chunks of kLargeChunk.
//
// Membership: only layers present in the candidate's mask can hold members (with the count
// accumulator the cell holds a count, and every layer is scanned).  For a table layer
// the vote inverts exactly -- a hit of bucket J votes into column j on row i when
// J = j + I_i + (f < g_i) -- so two buckets of the sorted hits hold all of that layer's members;
// other layers scan the buckets their radius range allows and redo the vote per hit (FP32 with
// FP64 refinement, as in the vote kernel).
//
// Stage-2 arithmetic: for a member with arc length s the z0 coordinate
// w(m) = n_z0 (z - s t_m - z0_min) / (z0_max - z0_min) is evaluated in FP32 around the row m_ref
// where it crosses z0_min, from coefficients formed in two-float arithmetic (member_coefficients),
// to within 2e-5 bin of its exact value (stage2_cell).
#include <atomic>
#include <climits>

#include "hough_internal.cuh"

namespace hough {

namespace {

constexpr int kConfirmWarpsMax = 8;
constexpr int kMemberCap = 128;        // members a warp holds at a time
constexpr int kSmallMembers = 32;      // candidates up to this size are finished by one warp
constexpr int kLargeChunk = 1024;      // members a CTA holds at a time for a large candidate

// The (up to two) ranges of staged hits of layer l that can hold members of candidate (i, j).
struct LayerScan {
    int nr;
    int st[2], en[2];
    int table;          // table layer: range 0 needs f >= g, range 1 needs f < g
    float g;
};

__device__ LayerScan layer_scan(const Axes &ax, const Workspace &w, const int32_t *offs, int l, int i, int j, float s32)
{
    LayerScan sc;
    sc.nr = 0;
    sc.table = 0;
    sc.g = 0.f;
    const int nphi = ax.n_phi;
    // both records at once (the table entry's address does not depend on the layer record)
    const LayerInfo li = w.info[l];
    const TabEntry te = w.tab[l * ax.n_qpt + i];
    if (!li.present) return sc;
    if (li.uniform) {
        if (i < li.lo || i > li.hi || te.I == kNoVote) return sc;
        sc.table = 1;
        sc.g = te.g;
        sc.nr = 2;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int J = wrap_col(j + te.I + side, nphi);   // |I| <= nphi / 4 + 1: within one wrap
            sc.st[side] = offs[l * nphi + J];
            sc.en[side] = offs[l * nphi + J + 1];
        }
        return sc;
    }
    const int lstart = offs[l * nphi], lend = offs[(l + 1) * nphi];
    if (ax.n_d0) {   // per-vote layer on a grid with a d0 axis: every hit of the layer
        sc.nr = 1; sc.st[0] = lstart; sc.en[0] = lend;
        return sc;
    }
    // per-vote layer: the buckets allowed by the layer's radius range on row i
    const float k = w.kq32[i];
    const float c_lo = 0.15f * (float)ax.b / 100.f * __uint_as_float(w.radii->rmin[l]) * 0.999f;
    const float c_hi = 0.15f * (float)ax.b / 100.f * __uint_as_float(w.radii->rmax[l]) * 1.001f;
    const float a1 = asinf(fminf(fmaxf(c_lo * k, -1.f), 1.f));
    const float a2 = asinf(fminf(fmaxf(c_hi * k, -1.f), 1.f));
    const int ja = (int)floorf(j + s32 * fminf(a1, a2)) - 2;
    const int jb = (int)floorf(j + 1 + s32 * fmaxf(a1, a2)) + 2;
    if (jb - ja + 1 >= nphi) {
        sc.nr = 1; sc.st[0] = lstart; sc.en[0] = lend;
    } else {
        const int a = wrap_col(ja, nphi), b = wrap_col(jb, nphi);   // within nphi / 4 + 3 of [0, nphi)
        if (a <= b) {
            sc.nr = 1; sc.st[0] = offs[l * nphi + a]; sc.en[0] = offs[l * nphi + b + 1];
        } else {
            sc.nr = 2; sc.st[0] = offs[l * nphi + a]; sc.en[0] = lend; sc.st[1] = lstart; sc.en[1] = offs[l * nphi + b + 1];
        }
    }
    return sc;
}

// Per-warp scratch of the enumeration: the candidate's (up to two per layer) bucket ranges in the
// fixed order (layer ascending, range 0 before range 1), with their exclusive prefix.
struct SegTable {
    int start[2 * HOUGH_MAX_LAYERS];
    int pre[2 * HOUGH_MAX_LAYERS + 1];
    float g[HOUGH_MAX_LAYERS];
    unsigned char kind[2 * HOUGH_MAX_LAYERS];   // 0: table side f >= g, 1: table side f < g, 2: per-vote test
};

// Members of candidate (i, j) enumerated by one warp in the fixed order (layer, bucket, position).
// Lanes first find every layer's bucket ranges in parallel, then test the flattened union of their
// hits together.  Returns the number of members; stores the staged position of the member of rank
// r in [lo, lo + cap) in pos[r - lo], and, when pool is given, in pool[r] for r < pool_n.
__device__ int warp_enumerate(const Axes &ax, const Workspace &w, const int32_t *offs, const HotHit *hot,
                              const ColdHit *cold, uint32_t mask, int i, int j, float s32, float refine_eps,
                              int lo, int cap, int *pos, int32_t *pool, int pool_n, SegTable &seg,
                              unsigned char *lay = nullptr)
{
    const int lane = threadIdx.x & 31;
    // a count says nothing of which layers voted: every layer may hold members
    if (ax.counts) mask = 0xFFFFu;
    // lane l < 16: layer l's ranges
    int st0 = 0, len0 = 0, st1 = 0, len1 = 0;
    unsigned char k0 = 0, k1 = 0;
    if (lane < HOUGH_MAX_LAYERS && lane < ax.n_layers && ((mask >> lane) & 1u)) {
        const LayerScan sc = layer_scan(ax, w, offs, lane, i, j, s32);
        if (sc.nr >= 1) { st0 = sc.st[0]; len0 = sc.en[0] - sc.st[0]; }
        if (sc.nr >= 2) { st1 = sc.st[1]; len1 = sc.en[1] - sc.st[1]; }
        k0 = sc.table ? 0 : 2;
        k1 = sc.table ? 1 : 2;
        seg.g[lane] = sc.g;
    }
    const int tot = len0 + len1;
    int incl = tot;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane < HOUGH_MAX_LAYERS) {
        const int base = incl - tot;
        seg.start[2 * lane] = st0;
        seg.start[2 * lane + 1] = st1;
        seg.pre[2 * lane] = base;
        seg.pre[2 * lane + 1] = base + len0;
        seg.kind[2 * lane] = k0;
        seg.kind[2 * lane + 1] = k1;
    }
    const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (lane == 0) seg.pre[2 * HOUGH_MAX_LAYERS] = total;
    __syncwarp();
    int count = 0;
    // the hit record of flattened index v, with its segment: the last q with pre[q] <= v
    auto locate = [&](int v, int &q) {
        q = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
            if (q + step < 2 * HOUGH_MAX_LAYERS && seg.pre[q + step] <= v) q += step;
        return seg.start[q] + (v - seg.pre[q]);
    };
    // software-pipelined: the next round's record is requested before this round is tested
    int q = 0, p = 0;
    HotHit hh{};
    if (lane < total) {
        p = locate(lane, q);
        hh = hot[p];
    }
    for (int base = 0; base < total; base += 32) {
        const int v = base + lane;
        const int vn = v + 32;
        int qn = 0, pn = 0;
        HotHit hn{};
        if (vn < total) {
            pn = locate(vn, qn);
            hn = hot[pn];
        }
        bool mem = false;
        if (v < total) {
            const int kind = seg.kind[q];
            if (kind == 0) {
                mem = !(hh.f < seg.g[q >> 1]);
            } else if (kind == 1) {
                mem = hh.f < seg.g[q >> 1];
            } else {
                const int rlo = (int)(hh.rows & 0xFFFFu), rhi = (int)(hh.rows >> 16);
                if (ax.n_d0) {   // every vote in FP64 on a grid with a d0 axis
                    const ColdHit ch = cold[p];
                    int jj = 0;
                    mem = exact_vote(ax, (double)ch.r, (double)ch.phi, i, &jj) && jj == j;
                } else if (i >= rlo && i <= rhi) {
                    const float x = fminf(fmaxf(hh.c * w.kq32[i], -1.f), 1.f);
                    const float vq = fmaf(-asinf(x), s32, hh.f);
                    const float fl = floorf(vq);
                    const float d = vq - fl;
                    int jj = (int)(hh.jl & 0xFFFFu) + (int)fl;
                    if (d < refine_eps || d > 1.f - refine_eps || fabsf(x) > kRefineXLim) {
                        const ColdHit ch = cold[p];
                        jj = exact_bin(ax, (double)ch.phi, __dmul_rn(sagitta_coef(ax, (double)ch.r), qpt_centre(ax, i)));
                    }
                    mem = wrap_col(jj, ax.n_phi) == j;
                }
            }
        }
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, mem);
        if (mem) {
            const int r = count + __popc(ball & ((1u << lane) - 1u));
            if (r >= lo && r < lo + cap) {
                pos[r - lo] = p;
                if (lay) lay[r - lo] = (unsigned char)(q >> 1);
            }
            if (pool && r < pool_n) pool[r] = p;
        }
        count += __popc(ball);
        q = qn;
        p = pn;
        hh = hn;
    }
    __syncwarp();
    return count;
}

// Arc length of a member at row i: from the table for a uniform layer, else from the closest
// approach in FP64 (r asin(|x|) / |x| for prompt tracks).
__device__ __forceinline__ double member_arc(const Axes &ax, const Workspace &w, int l, int i, float r)
{
    const LayerInfo li = w.info[l];
    if (li.uniform) return w.arc[l * ax.n_qpt + i];
    const double rd = (double)r;
    const double x = __dmul_rn(sagitta_coef(ax, rd), qpt_centre(ax, i));
    const double d0 = d0_centre(ax, i);
    double y = x;
    track_sin(rd, x, d0, &y);   // a member's track passes its radius: its vote was cast
    return track_arc(rd, x, d0, y);
}

// Stage-2 coefficients of one member at row i: z0 coordinate w(m) = a - (m - m_ref) b in FP32.
// For a layer of one radius the per-row terms S = zscale s t_0 and B = zscale s dt come from the
// table and w(m_ref) = zscale (z - z0_min) - S - m_ref B is formed in two-float arithmetic (about
// 2^-44 relative before the final rounding), which keeps a within a few 1e-6 bins of the exact
// value.  Other layers take the FP64 route.
__device__ __forceinline__ void member_coefficients(const Axes &ax, const Workspace &w, const HotHit *hot,
                                                    const ColdHit *cold, int p, int i, float *a_out, float *b_out,
                                                    int *mrl_out, int layer = -1)
{
    // the layer from the enumeration when given: then the layer record, the stage-2 terms and the
    // hit's coordinates are requested together
    const int l = layer >= 0 ? layer : (int)((hot[p].jl >> 16) & 0xFu);
    const ColdHit ch = cold[p];
    if (w.info[l].uniform) {
        const float4 zc = w.zco[l * ax.n_qpt + i];
        // d = z - z0_min and Z = zscale d as two-float values
        float2 d = two_sum(ch.z, -ax.zmin_hi);
        d.y = __fsub_rn(d.y, ax.zmin_lo);
        const float2 zp = two_prod(d.x, ax.zs_hi);
        const float zlo = zp.y + d.x * ax.zs_lo + d.y * ax.zs_hi;
        // A = Z - S
        float2 A = two_sum(zp.x, -zc.x);
        A.y = A.y + (zlo - zc.y);
        int mref = 0;
        if (zc.z > 0.f) mref = (int)fminf(fmaxf(rintf(__fdividef(A.x, zc.z)), 0.f), (float)(ax.n_cot - 1));
        // a = A - m_ref B; m_ref B.hi is exact as a two-float product
        const float fm = (float)mref;
        const float2 q = two_prod(fm, zc.z);
        *a_out = __fsub_rn(A.x, q.x) + (A.y - q.y - fm * zc.w);
        *b_out = zc.z;
        *mrl_out = mref | (l << 16);
        return;
    }
    const double s = member_arc(ax, w, l, i, ch.r);
    const double t0 = __dadd_rn(ax.cot_min, __dmul_rn(0.5, ax.dt));
    const double A = __dmul_rn(ax.zscale, __dsub_rn(__dsub_rn((double)ch.z, ax.z0_min), __dmul_rn(s, t0)));
    const double B = __dmul_rn(ax.zscale, __dmul_rn(s, ax.dt));
    int mref = 0;
    if (B > 0.0) mref = (int)fminf(fmaxf(rintf((float)A / (float)B), 0.f), (float)(ax.n_cot - 1));
    *a_out = (float)(A - (double)mref * B);
    *b_out = (float)B;
    *mrl_out = mref | (l << 16);
}

// z0 bin of a member's vote at cot row m, -1 outside the grid: w(m) = a - (m - m_ref) b in FP32,
// one fused multiply-add from the two-float coefficients.  Its error stays below 2e-5 bin (a to
// ~4e-6, the rounding of b times |m - m_ref| <= 128 / b rows to ~8e-6, the final rounding to
// ~4e-6), so every vote farther than that from a z0 edge -- in particular every vote the exact
// definition would not flag within 1e-4 bin -- lands in the bin the definition gives.
__device__ __forceinline__ int stage2_cell(const Axes &ax, float a, float b, int mrl, int m)
{
    const float wv = fmaf(-(float)(m - (mrl & 0xFFFF)), b, a);
    return (wv >= 0.f && wv < (float)ax.n_z0) ? (int)wv : -1;   // truncation is the floor here
}

// Cot rows [*lo, *hi] whose vote of the member can fall inside the z0 range: w(m) = a - (m - m_ref) b
// is monotone in m, so the rows form one run; the bounds are widened by a row on each side and
// every pair is still tested by stage2_cell.
__device__ __forceinline__ void member_rows(const Axes &ax, float a, float b, int mrl, int *lo, int *hi)
{
    const int mref = mrl & 0xFFFF;
    const float top = (float)(ax.n_cot - 1);
    if (!(b > 0.f)) {
        const bool in = a > -1.f && a < (float)ax.n_z0 + 1.f;
        *lo = in ? 0 : 1;
        *hi = in ? ax.n_cot - 1 : 0;
        return;
    }
    // approximate quotients: the run is widened by a row each side and every pair is tested exactly
    const float flo = floorf((float)mref + __fdividef(a - (float)ax.n_z0, b));
    const float fhi = floorf((float)mref + __fdividef(a, b)) + 1.f;
    *lo = (int)fminf(fmaxf(flo, 0.f), top + 1.f);
    *hi = (int)fminf(fmaxf(fhi, -1.f), top);
}

struct Best {
    unsigned cnt, cell, mask;
};

// One stage-2 vote: OR the member's layer bit into cell (m, nz) of `grid` and judge the cell by
// the mask the OR produced.  The contributions to a cell are serialised by the atomic, so the last
// one sees the cell's final mask; every other sees a subset of it.  Hence the largest popcount
// seen over all votes is the grid's maximum, the cells seen with it are exactly the cells that
// reach it, and the lowest of them -- with the mask seen there, which is its final mask -- is the
// row-major-first arg-max.  No second pass over the votes is needed.  Returns the word index.
// P10: the grid packs three 10-bit masks a word (detectors of at most 10 layers), else two 16-bit.
template <bool P10 = false>
__device__ __forceinline__ int stage2_vote(const Axes &ax, uint32_t *grid, int m, int nz, int layer, Best &best)
{
    const unsigned cell = (unsigned)(m * ax.n_z0 + nz);
    const unsigned word = P10 ? cell / 3u : cell >> 1;
    const unsigned shift = P10 ? (cell - word * 3u) * 10u : (cell & 1u) << 4;
    const uint32_t bit = 1u << layer;
    const uint32_t old = atomicOr(&grid[word], bit << shift);
    const uint32_t m16 = ((old >> shift) & (P10 ? 0x3FFu : 0xFFFFu)) | bit;
    const unsigned cnt = (unsigned)__popc(m16);
    if (cnt > best.cnt || (cnt == best.cnt && cell < best.cell)) {
        best.cnt = cnt;
        best.cell = cell;
        best.mask = m16;
    }
    return (int)word;
}

__device__ __forceinline__ void warp_best(Best &best)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned oc = __shfl_xor_sync(0xFFFFFFFFu, best.cnt, d);
        const unsigned ol = __shfl_xor_sync(0xFFFFFFFFu, best.cell, d);
        const unsigned om = __shfl_xor_sync(0xFFFFFFFFu, best.mask, d);
        if (oc > best.cnt || (oc == best.cnt && ol < best.cell)) {
            best.cnt = oc;
            best.cell = ol;
            best.mask = om;
        }
    }
}

__device__ __forceinline__ hough_candidate finished(const Axes &ax, hough_candidate cd, int n, int written, const Best &b)
{
    cd.n_members = (uint32_t)n;
    cd.icot = b.cell / (unsigned)ax.n_z0;
    cd.jz0 = b.cell % (unsigned)ax.n_z0;
    cd.mask2 = b.mask;
    cd.flags = ((int)b.cnt >= min(ax.threshold, ax.n_layers) ? 1u : 0u) | (written < n ? 2u : 0u);
    return cd;
}

// Per-warp scratch of the small-candidate stage 2 (member positions stay in the warp's position
// buffer).
struct SmallStage2 {
    float a[kSmallMembers], b[kSmallMembers];
    int mrl[kSmallMembers], mlo[kSmallMembers];
    int start[kSmallMembers + 1];
};

// The enumeration table and the small stage 2 are never live at the same time: a warp fills the
// latter only after its enumeration has finished (and synchronised), and enumerates again only
// after its stage 2 has.
union WarpScratch {
    SegTable seg;
    SmallStage2 small;
};

// Stage 2 of up to 32 members in the warp's private grid: lane q prepares member q and its run of
// cot rows; the (member, row) pairs of all runs are then spread over the lanes and voted in one pass
// (stage2_vote).  Returns, through rlo / rhi, the rows the runs cover (rlo > rhi when none): every
// touched cell lies in them, which is what the caller clears afterwards.  One simple loop keeps the
// code small: with few warps resident, instruction fetch of a large body is what a candidate waits on.
__device__ __forceinline__ int small_pair_member(const SmallStage2 &sm, int n, int v)
{
    // the member whose run holds pair v: the last q with start[q] <= v
    int q = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (q + step < n && sm.start[q + step] <= v) q += step;
    return q;
}

// K pairs per lane, v0 + 32 u for u < K, straight-line and independent of each other (an index
// past the end is clamped and its result masked): a lone warp (few candidates) is bound by the
// latency of this chain, not by issue.
template <int K, bool P10>
__device__ __forceinline__ void vote_pairs(const Axes &ax, uint32_t *grid, const SmallStage2 &sm, int n, int total,
                                           int v0, Best &best, unsigned long long &votes)
{
    int m[K], nz[K], ly[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
        const int v = v0 + 32 * u;
        const int vc = min(v, total - 1);
        const int q = small_pair_member(sm, n, vc);
        const int mrl = sm.mrl[q];
        m[u] = sm.mlo[q] + (vc - sm.start[q]);
        ly[u] = mrl >> 16;
        const int cell = stage2_cell(ax, sm.a[q], sm.b[q], mrl, m[u]);
        nz[u] = v < total ? cell : -1;
    }
#pragma unroll
    for (int u = 0; u < K; ++u)
        if (nz[u] >= 0) {
            stage2_vote<P10>(ax, grid, m[u], nz[u], ly[u], best);
            ++votes;
        }
}

template <bool P10>
__device__ void warp_stage2_small(const Axes &ax, const Workspace &w, const ColdHit *cold, uint32_t *grid,
                                  SmallStage2 &sm, const int *pos, int n, int i, Best &best,
                                  unsigned long long &votes, int &rlo, int &rhi)
{
    const int lane = threadIdx.x & 31;
    int len = 0, lo = ax.n_cot, hi = -1;
    if (lane < n) {
        member_rows(ax, sm.a[lane], sm.b[lane], sm.mrl[lane], &lo, &hi);
        sm.mlo[lane] = lo;
        len = max(0, hi - lo + 1);
        if (!len) {
            lo = ax.n_cot;
            hi = -1;
        }
    }
    int incl = len;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += t;
        lo = min(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, d));
        hi = max(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, d));
    }
    rlo = min(rlo, lo);
    rhi = max(rhi, hi);
    if (lane < kSmallMembers) sm.start[lane] = incl - len;
    const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (lane == 0) sm.start[kSmallMembers] = total;
    __syncwarp();
    // rounds of four pairs per lane while more than two lanes' worth remain, then one pair per lane:
    // a masked four-pair round costs a full round's instructions however few pairs it holds
    constexpr int kIlp = 4;
    int base = 0;
    for (; total - base > 64; base += 32 * kIlp)
        vote_pairs<kIlp, P10>(ax, grid, sm, n, total, base + lane, best, votes);
    for (; base < total; base += 32) vote_pairs<1, P10>(ax, grid, sm, n, total, base + lane, best, votes);
    __syncwarp();
}

// Zero the grid words of rows [rlo, rhi] (16-byte stores over a span rounded out to whole vectors:
// the extra words hold only cells outside the touched rows, already zero).
template <bool P10>
__device__ __forceinline__ void clear_rows(const Axes &ax, uint32_t *grid, int rlo, int rhi)
{
    if (rlo > rhi) return;
    const int lane = threadIdx.x & 31;
    const int c0 = rlo * ax.n_z0, c1 = (rhi + 1) * ax.n_z0 - 1;   // first and last cell
    const int w0 = (P10 ? c0 / 3 : c0 >> 1) & ~3;
    const int w1 = ((P10 ? c1 / 3 : c1 >> 1) | 3) + 1;   // <= grid words (a multiple of 4)
    uint4 *g4 = reinterpret_cast<uint4 *>(grid);
    for (int q = (w0 >> 2) + lane; q < (w1 >> 2); q += 32) g4[q] = make_uint4(0u, 0u, 0u, 0u);
}

// Membership and, for candidates of at most kSmallMembers members, stage 2: one warp per candidate
// over all events' candidates.  Members go once, in the fixed order, to the member pool; a larger
// candidate is filed for the CTA stage-2 kernel.
// P10: 10-bit masks, three to a word (at most 10 layers): a 64 x 64 grid takes 5.3 KB instead of
// 8 KB, which with 64 registers a thread lets four CTAs share an SM instead of three.
template <bool P10>
__global__ void __launch_bounds__(kConfirmWarpsMax * 32, P10 ? 4 : 3)
    member_kernel(Axes ax, Workspace w, float s32, float refine_eps, int grid_words)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_m[];
    __shared__ int s_pos[kConfirmWarpsMax][kMemberCap];
    __shared__ unsigned char s_lay[kConfirmWarpsMax][kMemberCap];
    __shared__ WarpScratch s_scratch[kConfirmWarpsMax];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    int *pos = s_pos[warp];
    unsigned char *lay = s_lay[warp];
    SegTable &seg = s_scratch[warp].seg;
    SmallStage2 &sm = s_scratch[warp].small;
    uint32_t *grid = reinterpret_cast<uint32_t *>(smem_m) + warp * grid_words;   // warp-private, clear
    for (int q = lane; q < grid_words; q += 32) grid[q] = 0u;
    __syncwarp();
    const int nkeys = ax.n_layers * ax.n_phi;
    const int total = (int)w.counters->total_cands;
    // candidate f goes to CTA f mod gridDim, so that a few candidates spread over all SMs
    int e = 0, e_base = 0, e_next = w.n_events == 1 ? INT_MAX : -1;   // the event of the last candidate
    for (int f = warp * gridDim.x + blockIdx.x; f < total; f += gridDim.x * nwarps) {
        // a warp's candidates come in increasing flattened order, so its event only moves forward:
        // a short forward step instead of a binary search (none at all for a one-event batch)
        if (e_next < 0) {
            e = upper_index(w.cand_base, w.n_events, f);
            e_base = w.cand_base[e];
            e_next = w.cand_base[e + 1];
        }
        while (f >= e_next) {
            ++e;
            e_base = e_next;
            e_next = w.cand_base[e + 1];
        }
        const int c = f - e_base;
        const int64_t hstart = w.hit_start[e];
        const HotHit *hot = w.hot + hstart;
        const ColdHit *cold = w.cold + hstart;
        const int32_t *offs = w.offs + (int64_t)e * (nkeys + 1);
        int32_t *pool = w.mem_pool + (int64_t)e * w.max_members;
        hough_candidate *cands = w.cands + (int64_t)e * w.max_cand;
        const hough_candidate cd = cands[c];
        const int i = (int)cd.iq;
        const int n = warp_enumerate(ax, w, offs, hot, cold, cd.mask, i, (int)cd.jphi, s32, refine_eps, 0,
                                     kMemberCap, pos, nullptr, 0, seg, lay);
        // the event's member pool is shared by all its candidates: reserve the range now and use it
        // after stage 2, so that the contended atomic's round trip overlaps the vote
        unsigned reserved = 0u;
        if (lane == 0 && n) reserved = atomicAdd(&w.stats[e].pool_used, (unsigned)n);
        Best best = {0u, 0u, 0u};
        unsigned long long votes = 0;
        if (n <= kMemberCap) {
            // members in chunks of 32 into the one grid, then the rows their runs covered cleared
            int rlo = ax.n_cot, rhi = -1;
            for (int c0 = 0; c0 < n; c0 += kSmallMembers) {
                const int nc = min(kSmallMembers, n - c0);
                if (lane < nc)
                    member_coefficients(ax, w, hot, cold, pos[c0 + lane], i, &sm.a[lane], &sm.b[lane], &sm.mrl[lane],
                                        lay[c0 + lane]);
                __syncwarp();
                warp_stage2_small<P10>(ax, w, cold, grid, sm, pos + c0, nc, i, best, votes, rlo, rhi);
            }
            clear_rows<P10>(ax, grid, rlo, rhi);
            __syncwarp();
            warp_best(best);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) votes += __shfl_xor_sync(0xFFFFFFFFu, votes, d);
        }
        int base = 0, written = 0;
        if (lane == 0) {
            const long long room = (long long)w.max_members - (long long)reserved;
            base = (int)min((long long)reserved, (long long)w.max_members);
            written = n ? (int)max(0LL, min((long long)n, room)) : 0;
            w.mem_start[(int64_t)e * w.max_cand + c] = base;
            w.mem_count[(int64_t)e * w.max_cand + c] = written;
            if (n) atomicAdd(&w.stats[e].n_members, (unsigned)n);
            if (n > kMemberCap) {
                cands[c].n_members = (uint32_t)n;
                w.large_list[atomicAdd(&w.counters->n_large, 1u)] = make_int2(e, c);
            } else {
                cands[c] = finished(ax, cd, n, written, best);
                if (votes) atomicAdd(&w.stats[e].stage2_votes, votes);
            }
        }
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        written = __shfl_sync(0xFFFFFFFFu, written, 0);
        if (n <= kMemberCap) {
            for (int q = lane; q < written; q += 32) pool[base + q] = pos[q];
        } else if (written > 0) {
            warp_enumerate(ax, w, offs, hot, cold, cd.mask, i, (int)cd.jphi, s32, refine_eps, 0, 0, pos, pool + base,
                           written, seg);
        }
        __syncwarp();
    }
}

struct Stage2Ctx {
    const HotHit *hot;
    const ColdHit *cold;
    const int32_t *offs;
    const int32_t *pool;
    hough_candidate *cands;
};

__device__ __forceinline__ Stage2Ctx stage2_ctx(const Axes &ax, const Workspace &w, int e)
{
    Stage2Ctx x;
    const int64_t hstart = w.hit_start[e];
    x.hot = w.hot + hstart;
    x.cold = w.cold + hstart;
    x.offs = w.offs + (int64_t)e * (ax.n_layers * ax.n_phi + 1);
    x.pool = w.mem_pool + (int64_t)e * w.max_members;
    x.cands = w.cands + (int64_t)e * w.max_cand;
    return x;
}

// Stage 2 of the large candidates: one CTA each, members in chunks of kLargeChunk, every chunk's
// (member, cot row) pairs voted in one pass (stage2_vote); the grid is cleared whole afterwards.
__global__ void __launch_bounds__(kConfirmWarpsMax * 32, 2) stage2_large_kernel(Axes ax, Workspace w, float s32,
                                                                                 float refine_eps)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem2[];
    __shared__ int s_pos[kLargeChunk];
    __shared__ float s_a[kLargeChunk], s_b[kLargeChunk];
    __shared__ int s_mrl[kLargeChunk];
    __shared__ int s_mlo[kLargeChunk], s_len[kLargeChunk], s_start[kLargeChunk + 1];
    __shared__ Best s_best[kConfirmWarpsMax];
    __shared__ SegTable s_seg;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    uint32_t *grid = reinterpret_cast<uint32_t *>(smem2);
    const int nlarge = (int)w.counters->n_large;
    if (blockIdx.x >= nlarge) return;
    const int grid_words = (((ax.n_cot * ax.n_z0 + 1) >> 1) + 3) & ~3;
    for (int q = threadIdx.x; q < grid_words; q += blockDim.x) grid[q] = 0u;
    for (int idx = blockIdx.x; idx < nlarge; idx += gridDim.x) {
        unsigned long long votes = 0;
        const int2 ec = w.large_list[idx];
        const int e = ec.x, c = ec.y;
        const Stage2Ctx x = stage2_ctx(ax, w, e);
        const hough_candidate cd = x.cands[c];
        const int i = (int)cd.iq, n = (int)cd.n_members;
        const int base = w.mem_start[(int64_t)e * w.max_cand + c], written = w.mem_count[(int64_t)e * w.max_cand + c];
        const int nchunks = (n + kLargeChunk - 1) / kLargeChunk;
        Best best = {0u, 0u, 0u};
        for (int k = 0; k < nchunks; ++k) {
            const int lo = k * kLargeChunk;
            const int nm = min(kLargeChunk, n - lo);
            __syncthreads();
            if (written == n) {
                for (int q = threadIdx.x; q < nm; q += blockDim.x) s_pos[q] = x.pool[base + lo + q];
            } else if (warp == 0) {
                warp_enumerate(ax, w, x.offs, x.hot, x.cold, cd.mask, i, (int)cd.jphi, s32, refine_eps, lo,
                               kLargeChunk, s_pos, nullptr, 0, s_seg);
            }
            __syncthreads();
            for (int q = threadIdx.x; q < nm; q += blockDim.x) {
                member_coefficients(ax, w, x.hot, x.cold, s_pos[q], i, &s_a[q], &s_b[q], &s_mrl[q]);
                int rlo, rhi;
                member_rows(ax, s_a[q], s_b[q], s_mrl[q], &rlo, &rhi);
                s_mlo[q] = rlo;
                s_len[q] = max(0, rhi - rlo + 1);
            }
            __syncthreads();
            // exclusive scan of the runs' lengths
            if (warp == 0) {
                int carry = 0;
                for (int b0 = 0; b0 < nm; b0 += 32) {
                    const int q = b0 + lane;
                    const int v = q < nm ? s_len[q] : 0;
                    int inc = v;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int t = __shfl_up_sync(0xFFFFFFFFu, inc, d);
                        if (lane >= d) inc += t;
                    }
                    if (q < nm) s_start[q] = carry + inc - v;
                    carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
                }
                if (lane == 0) s_start[nm] = carry;
            }
            __syncthreads();
            // (member, cot row) pairs of the chunk's runs, spread over the CTA
            const int npairs = s_start[nm];
            for (int v = threadIdx.x; v < npairs; v += blockDim.x) {
                int qlo = 0, qhi = nm - 1;
                while (qlo < qhi) {
                    const int mid = (qlo + qhi + 1) >> 1;
                    if (s_start[mid] <= v) qlo = mid; else qhi = mid - 1;
                }
                const int m = s_mlo[qlo] + (v - s_start[qlo]);
                const int mrl = s_mrl[qlo];
                const int nz = stage2_cell(ax, s_a[qlo], s_b[qlo], mrl, m);
                if (nz >= 0) {
                    stage2_vote(ax, grid, m, nz, mrl >> 16, best);
                    ++votes;
                }
            }
        }
        warp_best(best);
        if (lane == 0) s_best[warp] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            Best b = s_best[0];
            for (int q = 1; q < nwarps; ++q) {
                const Best o = s_best[q];
                if (o.cnt > b.cnt || (o.cnt == b.cnt && o.cell < b.cell)) b = o;
            }
            x.cands[c] = finished(ax, cd, n, written, b);
        }
        for (int q = threadIdx.x; q < grid_words; q += blockDim.x) grid[q] = 0u;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) votes += __shfl_xor_sync(0xFFFFFFFFu, votes, d);
        if (lane == 0 && votes) atomicAdd(&w.stats[e].stage2_votes, votes);
        __syncthreads();
    }
}

__global__ void member_index_kernel(Workspace w, int32_t *idx_out, int64_t total)
{
    pdl_enter();
    const ColdHit *cold = w.cold + w.hit_start[0];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
        idx_out[q] = cold[w.mem_pool[q]].idx;
}

int confirm_grid_words(const Axes &ax) { return (((ax.n_cot * ax.n_z0 + 1) >> 1) + 3) & ~3; }

// Words of a warp's grid of 10-bit masks, three to a word, rounded up to whole 16-byte vectors.
int packed_grid_words(const Axes &ax) { return (((ax.n_cot * ax.n_z0 + 2) / 3) + 3) & ~3; }


}  // namespace

size_t stage2_smem_bytes(const Axes &ax) { return (size_t)confirm_grid_words(ax) * 4; }

namespace {

// Resident CTAs per SM of a kernel at a block size and dynamic shared-memory size, asked once per
// pair (the answer depends on the kernel and the device only; the library drives one device model).
template <typename K>
int resident_ctas(K kernel, int threads, size_t smem, std::atomic<unsigned long long> &memo)
{
    const unsigned long long key = (unsigned long long)smem | ((unsigned long long)threads << 20);
    const unsigned long long m = memo.load(std::memory_order_relaxed);
    if (m && (m >> 32) == key) return (int)(m & 0xFFFFFFFFull);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) n = 1;
    memo.store((key << 32) | (unsigned)n, std::memory_order_relaxed);
    return n;
}

std::atomic<unsigned long long> g_member_ctas{0}, g_member_p10_ctas{0}, g_large_ctas{0};
std::atomic<int> g_member_static{-1}, g_smem_optin{-1};

// Warps per member CTA: kConfirmWarpsMax, or as many as shared memory holds when each warp's grid
// is large (n_cot * n_z0 up to 16384 cells, 32 KB a warp).
int member_warps(size_t grid_bytes)
{
    if (g_member_static.load(std::memory_order_relaxed) < 0) {
        cudaFuncAttributes fa{};
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        if (cudaFuncGetAttributes(&fa, member_kernel<false>) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return kConfirmWarpsMax;   // the launch itself then reports what is wrong
        g_smem_optin.store(optin, std::memory_order_relaxed);
        g_member_static.store((int)fa.sharedSizeBytes, std::memory_order_relaxed);
    }
    const long long room = (long long)g_smem_optin.load(std::memory_order_relaxed) -
                           (long long)g_member_static.load(std::memory_order_relaxed);
    return (int)std::max(1LL, std::min((long long)kConfirmWarpsMax, room / (long long)std::max<size_t>(grid_bytes, 1)));
}

}  // namespace

cudaError_t launch_stage2(const Axes &ax, const Workspace &w, int sms, float refine_eps, cudaStream_t stream,
                          cudaEvent_t between)
{
    const float s32 = (float)(ax.n_phi * kInvTwoPi);
    // the number of candidates is known on the device only: persistent grids of exactly the
    // resident CTAs, each warp or CTA striding over the flattened (event, candidate) work
    const size_t large_smem = (size_t)confirm_grid_words(ax) * 4;
    // a warp's grid: 10-bit masks three to a word when the layers fit and a batch of events keeps
    // every warp busy (the fourth CTA an SM then holds is worth more than the 64-register cap
    // costs); otherwise, and for one event, whose candidates are spread one to a CTA and whose
    // time is one warp's chain, 16-bit masks and 80 registers
    const bool p10 = ax.n_layers <= 10 && w.n_events > 1;
    const int words = p10 ? packed_grid_words(ax) : confirm_grid_words(ax);
    const int warps = member_warps((size_t)words * 4);
    const size_t member_smem = (size_t)warps * words * 4;
    auto member = p10 ? member_kernel<true> : member_kernel<false>;
    cudaError_t err = cudaFuncSetAttribute(member, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)member_smem);
    if (!err) err = cudaFuncSetAttribute(member, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (err) return err;
    const int member_threads = warps * 32;
    const int member_ctas = resident_ctas(member, member_threads, member_smem, p10 ? g_member_p10_ctas : g_member_ctas);
    if ((err = launch_chained(member, dim3(member_ctas * sms), dim3(member_threads), member_smem, stream, ax, w, s32,
                              refine_eps, words)))
        return err;
    if (between && (err = cudaEventRecord(between, stream))) return err;
    err = cudaFuncSetAttribute(stage2_large_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)large_smem);
    if (!err) err = cudaFuncSetAttribute(stage2_large_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (err) return err;
    const int threads = kConfirmWarpsMax * 32;
    const int large_ctas = resident_ctas(stage2_large_kernel, threads, large_smem, g_large_ctas);
    return launch_chained(stage2_large_kernel, dim3(large_ctas * sms), dim3(threads), large_smem, stream, ax, w, s32,
                          refine_eps);
}

cudaError_t launch_member_index(const Workspace &w, int32_t *idx_out, int64_t total, cudaStream_t stream)
{
    if (total <= 0) return cudaSuccess;
    const int g = (int)min((total + 255) / 256, (int64_t)4096);
    cudaError_t err = launch_chained(member_index_kernel, dim3(g), dim3(256), 0, stream, w, idx_out, total);
    if (err) return err;
    return cudaGetLastError();
}

}  // namespace hough
