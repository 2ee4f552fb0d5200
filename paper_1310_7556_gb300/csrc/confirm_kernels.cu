// Confirmation of the candidates (Sec. 4: candidates found as local maxima are confirmed by "more
// expensive computations"): for each candidate, the hits whose stage-1 vote fell in its cell
// (membership) and their vote in a (cot theta, z0) grid of layer masks (stage 2).
//
// One kernel, confirm_kernel, with a group of threads per candidate: a warp in batches (thousands
// of candidates keep every SM busy), a CTA of four warps for a single event (a few hundred
// candidates, whose time is the chain of one candidate).  Groups stride over all events'
// candidates, flattened.  Per candidate:
//
//   1. Segments.  Only layers present in the candidate's mask can hold members (with the count
//      accumulator every layer is scanned).  For a layer whose hits share one radius the vote
//      inverts exactly -- a hit of bucket J votes into column j on row i when
//      J = j + I_i + (f < g_i) -- so two buckets of the (layer, azimuth bucket)-sorted hits hold
//      all of that layer's members: bucket j + I_i with f >= g_i and bucket j + I_i + 1 with
//      f < g_i.  Other layers give the buckets their radius range allows, whose hits redo the vote
//      (FP32 with FP64 refinement, as in the vote kernel).  Lane t of the first warp computes
//      range t = (layer t / 2, side t % 2); the non-empty ones are compacted with their exclusive
//      prefix, so their starts strictly increase.
//   2. Membership.  The group tests the flattened union of the ranges, a lane per hit.  A lane's
//      range is found without a search: the ranges starting inside the warp's window of 32 hits
//      are OR-reduced into one bit mask (a redux), and a population count below the lane gives its
//      range.  Members are ranked by ballot in the fixed order (layer, bucket, position) and
//      listed, each with its z, in the group's shared memory.
//   3. Coefficients.  A lane per listed member (so this arithmetic runs once per 32 members, not
//      once per 32 hits scanned): the z0 coordinate of its vote on cot row m,
//      w(m) = n_z0 (z - s t_m - z0_min) / (z0_max - z0_min) = a - (m - m_ref) b, evaluated in FP32
//      around the row m_ref where it crosses z0_min, from coefficients formed in two-float
//      arithmetic (to within 2e-5 bin of its exact value), and the exact run of rows whose vote
//      falls inside the z0 range (w is monotone in m, so they form one run).  Members with a
//      non-empty run are compacted in place with the exclusive prefix of the run lengths.
//   4. Stage-2 vote.  The (member, row) pairs of all runs are spread over the lanes -- a pair's
//      member found like a hit's range above -- and voted with a shared atomicOr into the group's
//      own n_cot x n_z0 grid (16-bit masks, or in batches of a detector of at most 10 layers
//      10-bit masks three to a word, 5.3 KB for 64 x 64).  The word the atomic returns judges the
//      cell: the last OR into a cell sees its final mask and every earlier one a subset, so the
//      largest popcount seen is the grid's maximum and the lowest cell seen with it the
//      row-major-first arg-max.  Each lane keeps the best as one 32-bit key (popcount, then the
//      complement of the cell index), and a redux finds the group's.
//   5. The cell's final mask is read back, the touched rows cleared, the candidate written.
//
// A candidate with more members than the list holds (kBatchCap, kEventCap), or whose runs hold more
// pairs than a chunk votes at a time, is done in chunks, the membership pass repeated for each,
// all chunks voting into the one grid.  The member lists are kept for contexts (hough_get_members
// reads them), in the event's member pool, where a slot is reserved once the membership pass has
// counted the members and step 3 stores each member as it reads it; a batch keeps none.  The event's member and stage-2
// vote counters are summed per group and added once per event a group visits.
#include <atomic>
#include <climits>

#include "hough_internal.cuh"

namespace hough {

namespace {

constexpr int kBatchCap = 40;      // members a warp holds at a time (batches)
constexpr int kBatchPairs = 1024;  // (member, row) pairs a warp votes at a time (batches)
constexpr int kEventCap = 256;     // members a four-warp group holds at a time (single events)
constexpr int kEventPairs = 4096;  // pairs it votes at a time
constexpr int kEventWarps = 4;     // warps per candidate for a single event
constexpr int kBatchGroups = 4;    // one-warp groups per CTA at most (batches)
constexpr int kMaxBandsRead = 8192;   // band offsets a single event's CTA may hold to read the band lists
constexpr int kManyPerCta = 2;        // one event with more candidates than this per CTA: a warp per candidate

// Per-group scratch of a group of WPC warps, for detectors of at most NL layers.  Kind of a range: bits 0..3 the layer, bit 4 the side (1: f < g), bit 5 a
// layer whose hits lie at several radii (each hit's vote recomputed).
template <int WPC, int CAP, int MAXP, int NL>
struct __align__(16) Scratch {
    // chunk member with a run of cot rows: a, b (float bits); (first row - first pair - m_ref) +
    // kDmBias in bits 0..19 and the layer in bits 20..23; (first row - first pair) * n_z0
    int4 par[CAP];
    float4 zco[NL];                 // stage-2 terms {S hi, S lo, B hi, B lo} of each table layer at this row
    float rb[NL];                   // 1 / B hi of each table layer at this row (approximate)
    unsigned starts[MAXP / 32];     // bit v: a chunk member's run starts at pair v
    int seg_pre[2 * NL], seg_start[2 * NL];   // the ranges, two a layer at most
    unsigned seg_kind[2 * NL];
    float seg_g[2 * NL];
    int wtmp[4 * WPC];
    int n_seg, total, pool_base, pool_written;
};

constexpr int kDmBias = 1 << 19;

template <int WPC>
__device__ __forceinline__ void group_sync()
{
    if (WPC == 1) __syncwarp(); else __syncthreads();
}

template <int WPC>
__device__ __forceinline__ int group_tid() { return WPC == 1 ? (int)(threadIdx.x & 31) : (int)threadIdx.x; }

template <int WPC>
__device__ __forceinline__ int group_warp() { return WPC == 1 ? 0 : (int)(threadIdx.x >> 5); }

__device__ __forceinline__ unsigned lanes_below() { return (1u << (threadIdx.x & 31)) - 1u; }

// Rank of this thread among the group's threads with `pred` set (group order: warp, then lane);
// *total receives their number.  Called by every thread of the group.
template <int WPC>
__device__ __forceinline__ int group_excl_count(bool pred, int *total, int *wtmp)
{
    const unsigned b = __ballot_sync(0xFFFFFFFFu, pred);
    const int within = __popc(b & lanes_below());
    if (WPC == 1) {
        *total = __popc(b);
        return within;
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) wtmp[w] = __popc(b);
    __syncthreads();
    int pre = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < WPC; ++k) {
        const int t = wtmp[k];
        pre += k < w ? t : 0;
        tot += t;
    }
    __syncthreads();
    *total = tot;
    return pre + within;
}

// Exclusive prefix of v over the group; *total receives the sum.  Called by every thread of the group.
template <int WPC>
__device__ __forceinline__ int group_excl_scan(int v, int *total, int *wtmp)
{
    const int lane = threadIdx.x & 31;
    int incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += t;
    }
    if (WPC == 1) {
        *total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        return incl - v;
    }
    const int w = threadIdx.x >> 5;
    if (lane == 31) wtmp[w] = incl;
    __syncthreads();
    int pre = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < WPC; ++k) {
        const int t = wtmp[k];
        pre += k < w ? t : 0;
        tot += t;
    }
    __syncthreads();
    *total = tot;
    return pre + incl - v;
}

// Maximum (MAX) or minimum of v over the group, returned to every thread.
template <int WPC, bool MAX>
__device__ __forceinline__ unsigned group_reduce(unsigned v, int *wtmp)
{
    v = MAX ? __reduce_max_sync(0xFFFFFFFFu, v) : __reduce_min_sync(0xFFFFFFFFu, v);
    if (WPC == 1) return v;
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) wtmp[w] = (int)v;
    __syncthreads();
    unsigned r = (unsigned)wtmp[0];
#pragma unroll
    for (int k = 1; k < WPC; ++k) r = MAX ? max(r, (unsigned)wtmp[k]) : min(r, (unsigned)wtmp[k]);
    __syncthreads();
    return r;
}

// Warp totals v of N quantities made group-wide: the sums over the warps before this one (pre)
// and over all (tot), in one exchange through shared memory (wx: WPC * N words).
template <int WPC, int N>
__device__ __forceinline__ void group_exchange(const int (&v)[N], int (&pre)[N], int (&tot)[N], int *wx)
{
#pragma unroll
    for (int n = 0; n < N; ++n) {
        pre[n] = 0;
        tot[n] = v[n];
    }
    if (WPC == 1) return;
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int n = 0; n < N; ++n) wx[w * N + n] = v[n];
    }
    __syncthreads();
#pragma unroll
    for (int n = 0; n < N; ++n) {
        int p = 0, t = 0;
#pragma unroll
        for (int k = 0; k < WPC; ++k) {
            const int x = wx[k * N + n];
            p += k < w ? x : 0;
            t += x;
        }
        pre[n] = p;
        tot[n] = t;
    }
    __syncthreads();
}

// Sum of v over the group, returned to every thread.
template <int WPC>
__device__ __forceinline__ unsigned group_reduce_add(unsigned v, int *wtmp)
{
    v = __reduce_add_sync(0xFFFFFFFFu, v);
    if (WPC == 1) return v;
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) wtmp[w] = (int)v;
    __syncthreads();
    unsigned r = 0u;
#pragma unroll
    for (int k = 0; k < WPC; ++k) r += (unsigned)wtmp[k];
    __syncthreads();
    return r;
}

// The index, within a sorted list of strictly increasing starts held one per lane (lane t: entry
// base_idx + t, INT_MAX past the end), of the entry owning position pos0 + lane, given that entry
// q_base owns pos0.  The entries starting inside the window (pos0, pos0 + 32) are OR-reduced into
// a bit mask; the count of those at or below the lane's position is its offset from q_base.
__device__ __forceinline__ int window_owner(int st_next, int pos0, int q_base)
{
    const int d = st_next - pos0;   // st_next: start of entry q_base + 1 + lane (no overflow: pos0 >= 0)
    const unsigned bits = __reduce_or_sync(0xFFFFFFFFu, (d > 0 && d < 32) ? 1u << d : 0u);
    const int lane = threadIdx.x & 31;
    return q_base + __popc(bits & ((2u << lane) - 1u));
}

// The (up to two) ranges of staged hits of a layer whose hits lie at several radii that can hold
// members of candidate (i, j): the buckets its radius range allows on row i.  Returns the count.
__device__ int general_ranges(const Axes &ax, const Workspace &w, const int32_t *offs, int l, int i, int j, float s32,
                              int st[2], int en[2])
{
    const int nphi = ax.n_phi;
    const int lstart = offs[l * nphi], lend = offs[(l + 1) * nphi];
    if (ax.n_d0) {   // a grid with a d0 axis: every hit of the layer
        st[0] = lstart;
        en[0] = lend;
        return 1;
    }
    const float k = w.kq32[i];
    const float c_lo = 0.15f * (float)ax.b / 100.f * __uint_as_float(w.radii->rmin[l]) * 0.999f;
    const float c_hi = 0.15f * (float)ax.b / 100.f * __uint_as_float(w.radii->rmax[l]) * 1.001f;
    const float a1 = asinf(fminf(fmaxf(c_lo * k, -1.f), 1.f));
    const float a2 = asinf(fminf(fmaxf(c_hi * k, -1.f), 1.f));
    const int ja = (int)floorf(j + s32 * fminf(a1, a2)) - 2;
    const int jb = (int)floorf(j + 1 + s32 * fmaxf(a1, a2)) + 2;
    if (jb - ja + 1 >= nphi) {
        st[0] = lstart;
        en[0] = lend;
        return 1;
    }
    const int a = wrap_col(ja, nphi), b = wrap_col(jb, nphi);   // within nphi / 4 + 3 of [0, nphi)
    if (a <= b) {
        st[0] = offs[l * nphi + a];
        en[0] = offs[l * nphi + b + 1];
        return 1;
    }
    st[0] = offs[l * nphi + a];
    en[0] = lend;
    st[1] = lstart;
    en[1] = offs[l * nphi + b + 1];
    return 2;
}

// Whether the staged hit at position p of a layer whose hits lie at several radii votes into cell
// (i, j): the vote redone per hit, as the vote kernel casts it.
__device__ __forceinline__ bool general_member(const Axes &ax, const Workspace &w, const HotHit *hot,
                                               const ColdHit *cold, int p, int i, int j, float s32, float refine_eps)
{
    const HotHit hh = hot[p];
    int jj = 0;
    if (ax.n_d0) {   // every vote in FP64 on a grid with a d0 axis
        const ColdHit ch = cold[p];
        return exact_vote(ax, (double)ch.r, (double)ch.phi, i, &jj) && jj == j;
    }
    const int rlo = (int)(hh.rows & 0xFFFFu), rhi = (int)(hh.rows >> 16);
    if (i < rlo || i > rhi) return false;
    const float x = fminf(fmaxf(hh.c * w.kq32[i], -1.f), 1.f);
    const float vq = fmaf(-asinf(x), s32, hh.f);
    const float fl = floorf(vq);
    const float d = vq - fl;
    jj = (int)(hh.jl & 0xFFFFu) + (int)fl;
    if (d < refine_eps || d > 1.f - refine_eps || fabsf(x) > kRefineXLim) {
        const ColdHit ch = cold[p];
        jj = exact_bin(ax, (double)ch.phi, __dmul_rn(sagitta_coef(ax, (double)ch.r), qpt_centre(ax, i)));
    }
    return wrap_col(jj, ax.n_phi) == j;
}

// Stage-2 coefficients of a member of a layer of one radius at row i: z0 coordinate
// w(m) = a - (m - m_ref) b in FP32.  The per-row terms S = zscale s t_0 and B = zscale s dt come
// from the table and w(m_ref) = zscale (z - z0_min) - S - m_ref B is formed in two-float
// arithmetic (about 2^-44 relative before the final rounding), which keeps a within a few 1e-6
// bins of the exact value.
__device__ __forceinline__ void table_coefficients(const Axes &ax, const float4 zc, float rb, float z, int l,
                                                   float *a_out, float *b_out, int *mrl_out)
{
    // d = z - z0_min and Z = zscale d as two-float values
    float2 d = two_sum(z, -ax.zmin_hi);
    d.y = __fsub_rn(d.y, ax.zmin_lo);
    const float2 zp = two_prod(d.x, ax.zs_hi);
    const float zlo = zp.y + d.x * ax.zs_lo + d.y * ax.zs_hi;
    // A = Z - S
    float2 A = two_sum(zp.x, -zc.x);
    A.y = A.y + (zlo - zc.y);
    // any nearby row will do
    const int mref = zc.z > 0.f ? (int)fminf(fmaxf(rintf(A.x * rb), 0.f), (float)(ax.n_cot - 1)) : 0;
    // a = A - m_ref B; m_ref B.hi is exact as a two-float product
    const float fm = (float)mref;
    const float2 q = two_prod(fm, zc.z);
    *a_out = __fsub_rn(A.x, q.x) + (A.y - q.y - fm * zc.w);
    *b_out = zc.z;
    *mrl_out = mref | (l << 16);
}

// The same for a member of a layer whose hits lie at several radii: the arc length from the
// closest approach in FP64 (r asin(|x|) / |x| for prompt tracks).
__device__ __forceinline__ void exact_coefficients(const Axes &ax, int l, int i, const ColdHit &ch, float *a_out,
                                                   float *b_out, int *mrl_out)
{
    const double rd = (double)ch.r;
    const double x = __dmul_rn(sagitta_coef(ax, rd), qpt_centre(ax, i));
    const double d0 = d0_centre(ax, i);
    double y = x;
    track_sin(rd, x, d0, &y);   // a member's track passes its radius: its vote was cast
    const double s = track_arc(rd, x, d0, y);
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

// The run of cot rows whose vote of the member can fall inside the z0 range.  w(m) is the rounding
// of a quantity strictly decreasing in m (b > 0), so it is non-increasing and the rows with
// 0 <= w(m) < n_z0 form one run.  Approximate quotients bound the run from outside by about a row
// on each side; one step at each end then drops a bound whose own vote falls outside, which
// leaves the exact run in all but rare cases (a row of an outer bound still outside: every pair
// is tested again when it votes).  *len receives the length (0: no row).
__device__ __forceinline__ void member_run(const Axes &ax, float a, float b, float rb, int mrl, int *lo_out,
                                           int *len_out)
{
    const int mref = mrl & 0xFFFF;
    const float top = (float)(ax.n_cot - 1);
    const float flo = floorf((float)mref + (a - (float)ax.n_z0) * rb);   // rb: about 1 / b
    const float fhi = floorf((float)mref + a * rb) + 1.f;
    int lo = (int)fminf(fmaxf(flo, 0.f), top + 1.f);
    int hi = (int)fminf(fmaxf(fhi, -1.f), top);
    lo += (lo <= hi && stage2_cell(ax, a, b, mrl, lo) < 0) ? 1 : 0;
    hi -= (hi >= lo && stage2_cell(ax, a, b, mrl, hi) < 0) ? 1 : 0;
    if (!(b > 0.f)) {   // w constant in m: every row or none
        const bool in = a >= 0.f && a < (float)ax.n_z0;
        lo = 0;
        hi = in ? ax.n_cot - 1 : -1;
    }
    *lo_out = lo;
    *len_out = max(0, hi - lo + 1);
}

// One stage-2 vote (when `in`): OR the member's layer bit into `cell` = m n_z0 + nz of `grid`; returns
// the key of the cell as the OR left it (0 when not `in`): its popcount above the complement of the cell index, so that the larger
// key is the larger popcount and, on a tie, the lower cell.  P10: the grid packs three 10-bit
// masks a word (detectors of at most 10 layers), else two 16-bit ones.
template <bool P10>
__device__ __forceinline__ unsigned stage2_vote(uint32_t *grid, unsigned cell, int layer, bool in)
{
    const unsigned word = P10 ? cell / 3u : cell >> 1;
    const unsigned shift = P10 ? (cell - word * 3u) * 10u : (cell & 1u) << 4;
    const uint32_t bit = 1u << layer;
    uint32_t old = 0u;
    if (in) old = atomicOr(&grid[word], bit << shift);
    const uint32_t msk = ((old >> shift) & (P10 ? 0x3FFu : 0xFFFFu)) | bit;
    return in ? ((unsigned)__popc(msk) << 16) | (0xFFFFu - cell) : 0u;
}

template <bool P10>
__device__ __forceinline__ uint32_t grid_mask(const uint32_t *grid, unsigned cell)
{
    const unsigned word = P10 ? cell / 3u : cell >> 1;
    const unsigned shift = P10 ? (cell - word * 3u) * 10u : (cell & 1u) << 4;
    return (grid[word] >> shift) & (P10 ? 0x3FFu : 0xFFFFu);
}

// Zero the grid words of rows [rlo, rhi] (16-byte stores over a span rounded out to whole vectors:
// the extra words hold only cells outside the touched rows, already zero).
template <int WPC, bool P10>
__device__ __forceinline__ void clear_rows(const Axes &ax, uint32_t *grid, int rlo, int rhi)
{
    if (rlo > rhi) return;
    const int c0 = rlo * ax.n_z0, c1 = (rhi + 1) * ax.n_z0 - 1;   // first and last cell
    const int w0 = (P10 ? c0 / 3 : c0 >> 1) & ~3;
    const int w1 = ((P10 ? c1 / 3 : c1 >> 1) | 3) + 1;   // <= grid words (a multiple of 4)
    uint4 *g4 = reinterpret_cast<uint4 *>(grid);
#pragma unroll 4
    for (int q = (w0 >> 2) + group_tid<WPC>(); q < (w1 >> 2); q += 32 * WPC) g4[q] = make_uint4(0u, 0u, 0u, 0u);
}

// A candidate record as two 16-byte vectors (the arrays are 16-byte aligned, 32 bytes an entry).
__device__ __forceinline__ void store_candidate(hough_candidate *p, const hough_candidate &c)
{
    reinterpret_cast<uint4 *>(p)[0] = make_uint4(c.iq, c.jphi, c.mask, c.n_members);
    reinterpret_cast<uint4 *>(p)[1] = make_uint4(c.icot, c.jz0, c.mask2, c.flags);
}

// Step 2: one pass over the candidate's ranges, a lane per hit, software-pipelined (the next
// round's hit is requested before this round is tested).  Members are ranked in the fixed order
// (layer, bucket, position) and sink(r, p, kd, z) receives member r: its staged position, the kind
// of its range and (Z) its z.  Returns the number of members.
template <int WPC, int CAP, int MAXP, int NL, bool GEN, bool Z, typename Sink>
__device__ int scan_members(const Axes &ax, const Workspace &w, Scratch<WPC, CAP, MAXP, NL> &S, const HotHit *hot,
                            const float *fsort, const float *zsort, const ColdHit *cold, int i, int j, float s32,
                            float refine_eps, Sink &&sink)
{
    const int lane = threadIdx.x & 31;
    const int T = S.total, nseg = S.n_seg;
    const int pre_t = lane < nseg ? S.seg_pre[lane] : INT_MAX;
    const int start_t = lane < nseg ? S.seg_start[lane] : 0;
    const unsigned kind_t = lane < nseg ? S.seg_kind[lane] : 0u;
    const float g_t = lane < nseg ? S.seg_g[lane] : 0.f;
    // the hit at flattened index base + lane: its staged position, range kind and threshold
    auto locate = [&](int base, int &p, unsigned &kd, float &gg) {
        const int qb = __popc(__ballot_sync(0xFFFFFFFFu, pre_t <= base)) - 1;   // range 0 starts at 0 <= base
        const int src = qb + 1 + lane;   // the range after qb that this lane inspects
        const int pn = __shfl_sync(0xFFFFFFFFu, pre_t, src & 31);
        const int sg = min(window_owner(src < 32 ? pn : INT_MAX, base, qb), 31);
        p = __shfl_sync(0xFFFFFFFFu, start_t, sg) + (base + lane - __shfl_sync(0xFFFFFFFFu, pre_t, sg));
        kd = __shfl_sync(0xFFFFFFFFu, kind_t, sg);
        gg = __shfl_sync(0xFFFFFFFFu, g_t, sg);
    };
    const int G = 32 * WPC;
    const int wb = 32 * group_warp<WPC>();
    int n = 0;
    int p = 0;
    unsigned kd = 0u;
    float gg = 0.f, f = 0.f, z = 0.f;
    if (wb < T) {
        locate(wb, p, kd, gg);
        if (wb + lane < T && !(kd & 32u)) {
            f = __ldg(&fsort[p]);
            if (Z) z = __ldg(&zsort[p]);
        }
    }
    for (int b0 = 0; b0 < T; b0 += G) {
        const int v = b0 + wb + lane;
        const int bn = b0 + G + wb;
        int pn = 0;
        unsigned kdn = 0u;
        float ggn = 0.f, fn = 0.f, zn = 0.f;
        if (bn < T) {
            locate(bn, pn, kdn, ggn);
            if (bn + lane < T && !(kdn & 32u)) {
                fn = __ldg(&fsort[pn]);
                if (Z) zn = __ldg(&zsort[pn]);
            }
        }
        bool mem = v < T && (f < gg) == ((kd & 16u) != 0u);   // side 1: f < g; side 0: f >= g
        if (GEN && v < T && (kd & 32u)) mem = general_member(ax, w, hot, cold, p, i, j, s32, refine_eps);
        int nm;
        const int r = n + group_excl_count<WPC>(mem, &nm, S.wtmp);
        if (mem) sink(r, p, kd, z);
        n += nm;
        p = pn;
        kd = kdn;
        gg = ggn;
        f = fn;
        z = zn;
    }
    return n;
}

// Totals of a chunk's runs.
struct ChunkOut {
    int npairs;     // (member, row) pairs of the members kept
    int consumed;   // members of the list the chunk has dealt with (kept, or without a run)
};

// Step 3 for the chunk's m members listed in par as {position, kind, z bits}: each one's stage-2
// coefficients and run of cot rows, a lane per member.  The members with a run are kept, in order,
// while their pairs fit MAXP: par is rewritten in place from slot 0 (a slot never lies past the
// entry it comes from, and a round's entries are all read before any is written), and the bit of
// each kept member's first pair is set in starts.  rlo / rhi widen to the rows the runs cover.
// pool (contexts): the member list, whose first `written` ranks are stored as the entries are read.
template <int WPC, int CAP, int MAXP, int NL, bool GEN, bool KEEP>
__device__ ChunkOut chunk_runs(const Axes &ax, Scratch<WPC, CAP, MAXP, NL> &S, const ColdHit *cold, int i, int m, int &rlo,
                               int &rhi, int32_t *pool, int rank0, int written)
{
    const int tid = group_tid<WPC>();
    const int G = 32 * WPC;
    for (int q = tid; q < MAXP / 32; q += G) S.starts[q] = 0u;
    int pairs = 0, kept = 0, consumed = 0;
    for (int b0 = 0; b0 < m; b0 += G) {
        const int idx = b0 + tid;
        const bool valid = idx < m;
        int4 e = make_int4(0, 0, 0, 0);
        if (valid) e = S.par[idx];
        // a context lists the member (rank rank0 + idx, its staged position) in its pool slot; a
        // member a later chunk lists again writes the same value
        if (KEEP && valid && rank0 + idx < written) pool[rank0 + idx] = e.x;
        group_sync<WPC>();   // the round's entries are read (and starts cleared) before any write
        // every lane forms coefficients (a lane past the list from entry 0's zeros) and the run is
        // dropped where not valid: no divergent branch on the table path
        float a, bb;
        int mrl, mlo, len;
        const unsigned kd = (unsigned)e.y;
        const int l = (int)(kd & 15u);
        float rb = S.rb[l];
        table_coefficients(ax, S.zco[l], rb, __int_as_float(e.z), l, &a, &bb, &mrl);
        if (GEN && valid && (kd & 32u)) {
            exact_coefficients(ax, l, i, cold[e.x], &a, &bb, &mrl);
            rb = bb > 0.f ? __frcp_rn(bb) : 0.f;
        }
        member_run(ax, a, bb, rb, mrl, &mlo, &len);
        if (!valid) len = 0;
        // pair prefix over the round (members without a run add nothing); a member whose pairs end
        // past MAXP, and every one after it (their prefixes only grow), waits for the next chunk
        int tot_len;
        const int st = pairs + group_excl_scan<WPC>(len, &tot_len, S.wtmp);
        const bool after = valid && st + len > MAXP;
        const bool keep = len > 0 && !after;
        const unsigned bkeep = __ballot_sync(0xFFFFFFFFu, keep);
        int pre[3], tot[3];
        group_exchange<WPC, 3>({__popc(bkeep), (int)__reduce_add_sync(0xFFFFFFFFu, keep ? (unsigned)len : 0u),
                                __popc(__ballot_sync(0xFFFFFFFFu, after))},
                               pre, tot, S.wtmp);
        if (WPC == 1) __syncwarp();
        if (keep) {
            const int slot = kept + pre[0] + __popc(bkeep & lanes_below());
            const int c0 = mlo - st;
            S.par[slot] = make_int4(__float_as_int(a), __float_as_int(bb),
                                    (c0 - (mrl & 0xFFFF) + kDmBias) | ((mrl >> 16) << 20), c0 * ax.n_z0);
            atomicOr(&S.starts[st >> 5], 1u << (st & 31));
            rlo = min(rlo, mlo);
            rhi = max(rhi, mlo + len - 1);
        }
        kept += tot[0];
        pairs += tot[1];
        consumed += min(G, m - b0) - tot[2];
        if (tot[2] > 0) break;
    }
    return {pairs, consumed};
}

// Stage-2 vote of the chunk's pairs (step 4); best keeps the lane's largest key and votes its
// count of votes cast.  Each warp takes windows of 32 consecutive pairs, one word of the start bits:
// the member owning pair bw + lane is the number of runs starting at or before it, less one -- the
// runs starting before the window (counted as the windows go by) plus a population count of the
// window's bits up to the lane.  A lane's owner is a kept member past npairs too (pair 0 starts a
// run), so every lane reads a valid entry and only the atomic is predicated.
template <int WPC, int CAP, int MAXP, int NL, bool P10>
__device__ void vote_pairs(const Axes &ax, const Scratch<WPC, CAP, MAXP, NL> &S, uint32_t *grid, int npairs,
                           unsigned &best, unsigned &votes)
{
    const int lane = threadIdx.x & 31;
    const unsigned upto = (2u << lane) - 1u;
    const float nz0 = (float)ax.n_z0;
    const int wg = group_warp<WPC>();
    auto vote = [&](int v, int owner) {
        const int4 pr = S.par[owner];
        // w(m) = a - (m - m_ref) b at the pair's row m, as stage2_cell evaluates it
        const float wv = fmaf(-(float)(v + (pr.z & 0xFFFFF) - kDmBias), __int_as_float(pr.y), __int_as_float(pr.x));
        const bool in = v < npairs && wv >= 0.f && wv < nz0;
        best = max(best, stage2_vote<P10>(grid, (unsigned)(v * ax.n_z0 + pr.w + (int)wv), pr.z >> 20, in));
        votes += in ? 1u : 0u;
    };
    int before = 0;   // runs starting in the windows before this warp's current one
    if constexpr (WPC == 1) {
        // two windows an iteration: two independent chains for the scheduler to interleave
        for (int bw = 0; bw < npairs; bw += 64) {
            const int q = bw >> 5;
            const unsigned b0 = S.starts[q], b1 = q + 1 < MAXP / 32 ? S.starts[q + 1] : 0u;
            const int n0 = __popc(b0);
            vote(bw + lane, before + __popc(b0 & upto) - 1);
            if (bw + 32 < npairs) vote(bw + 32 + lane, before + n0 + __popc(b1 & upto) - 1);   // (warp-uniform)
            before += n0 + __popc(b1);
        }
    } else {
        for (int k = 0; k < wg; ++k) before += __popc(S.starts[k]);
        for (int bw = 32 * wg; bw < npairs; bw += 32 * WPC) {
            const unsigned bits = S.starts[bw >> 5];
            const int owner = before + __popc(bits & upto) - 1;
#pragma unroll
            for (int k = 0; k < WPC; ++k)
                if ((bw >> 5) + k < MAXP / 32) before += __popc(S.starts[(bw >> 5) + k]);
            vote(bw + lane, owner);
        }
    }
}

// Exclusive prefix of counts[0, n) into out[0, n] (out[n]: the sum, also returned), by the whole CTA.
__device__ int block_excl_scan(const int32_t *counts, int n, int *out)
{
    __shared__ int s_w[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const int chunk = (n + blockDim.x - 1) / blockDim.x;
    const int k0 = min(n, (int)threadIdx.x * chunk), k1 = min(n, k0 + chunk);
    int sum = 0;
    for (int k = k0; k < k1; ++k) sum += counts[k];
    int incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    int before = 0, all = 0;
    for (int k = 0; k < nw; ++k) {
        before += k < warp ? s_w[k] : 0;
        all += s_w[k];
    }
    int run = before + incl - sum;
    for (int k = k0; k < k1; ++k) {
        out[k] = run;
        run += counts[k];
    }
    if (threadIdx.x == 0) out[n] = all;
    __syncthreads();
    return all;
}

// Membership and stage 2 of every candidate a group takes.  GEN: some layer's hits lie at several
// radii (their votes are redone per hit, partly in FP64); without it that code is left out, which
// spares the common path its registers.  KEEP: the member lists may be kept (Workspace::keep_members
// decides; single events only), code the batches' one-warp kernels leave out for the same reason.
template <int WPC, int CAP, int MAXP, int NL, bool P10, bool GEN, bool KEEP>
__device__ __forceinline__ void confirm_all(const Axes &ax, const Workspace &w, float s32, float refine_eps,
                                            Scratch<WPC, CAP, MAXP, NL> &S, uint32_t *grid, const LayerInfo *s_info,
                                            int ngroups, int gidx, int total, const int *band_offs)
{
    const int tid = group_tid<WPC>(), lane = threadIdx.x & 31, wg = group_warp<WPC>();
    const int L = ax.n_layers, nphi = ax.n_phi, nkeys = L * nphi;
    // the event's counters, summed by the group's first thread over the event's candidates it takes
    int acc_e = -1;
    unsigned acc_members = 0u;
    unsigned long long acc_votes = 0ull;
    // candidate f goes to CTA f mod gridDim, so that a few candidates spread over all SMs; a group's
    // candidates come in increasing flattened order, so its event only moves forward
    int e = 0, e_base = 0, e_next = w.n_events == 1 ? INT_MAX : -1;   // the event of the last candidate fetched
    // (i, j, mask) of candidate f, whose event becomes e; the next candidate's is requested while
    // this one is confirmed, taking its loads off the candidate's chain
    auto fetch = [&](int f) {
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
        if (band_offs) {
            // one event whose candidate list was not compacted: candidate c from its band's list
            int b = 0, hi = n_bands(ax, w.band_rows) - 1;   // the last band with offset <= c (shared memory)
            while (b < hi) {
                const int mid = (b + hi + 1) >> 1;
                if (band_offs[mid] <= c) b = mid; else hi = mid - 1;
            }
            const uint2 v = w.band_cands[(int64_t)b * w.band_cap + (c - band_offs[b])];
            return make_uint3(v.x / (unsigned)nphi, v.x % (unsigned)nphi, v.y);
        }
        const uint4 v = *reinterpret_cast<const uint4 *>(w.cands + (int64_t)e * w.max_cand + c);
        return make_uint3(v.x, v.y, v.z);
    };
    const int stride = gridDim.x * ngroups;
    int f = gidx * gridDim.x + blockIdx.x;
    uint3 rec = f < total ? fetch(f) : make_uint3(0u, 0u, 0u);
    for (; f < total; f += stride) {
        const int ev = e, c = f - e_base;
        hough_candidate cd;
        cd.iq = rec.x;
        cd.jphi = rec.y;
        cd.mask = rec.z;
        cd.n_members = cd.icot = cd.jz0 = cd.mask2 = cd.flags = 0u;
        if (f + stride < total) rec = fetch(f + stride);
        const int64_t hstart = ev == 0 ? 0 : w.hit_start[ev];   // hit_start[0] is 0
        const HotHit *hot = w.hot + hstart;
        const float *fsort = w.fsort + hstart;
        const float *zsort = w.zsort + hstart;
        const ColdHit *cold = w.cold + hstart;
        const int32_t *offs = w.offs + (int64_t)ev * (nkeys + 1);
        hough_candidate *cands = w.cands + (int64_t)ev * w.max_cand;
        const int i = (int)cd.iq, j = (int)cd.jphi;
        // step 1: the candidate's ranges, lane t of the first warp taking range t = (layer t/2, side t%2)
        if (wg == 0) {
            const int l = lane >> 1, side = lane & 1;
            const uint32_t mask = ax.counts ? 0xFFFFu : cd.mask;   // a count names no layers
            int st = 0, len = 0;
            unsigned kind = 0u;
            float gv = 0.f;
            if (l < L && ((mask >> l) & 1u)) {
                const LayerInfo li = s_info[l];
                if (li.present && li.uniform) {
                    if (i >= li.lo && i <= li.hi) {
                        const TabEntry te = w.tab[l * ax.n_qpt + i];
                        const float4 zc = w.zco[l * ax.n_qpt + i];
                        if (te.I != kNoVote) {
                            const int J = wrap_col(j + te.I + side, nphi);   // |I| <= nphi / 4 + 1
                            st = offs[l * nphi + J];
                            len = offs[l * nphi + J + 1] - st;
                            kind = (unsigned)l | ((unsigned)side << 4);
                            gv = te.g;
                            if (side == 0) {
                                S.zco[l] = zc;
                                S.rb[l] = zc.z > 0.f ? __fdividef(1.f, zc.z) : 0.f;   // approximate suffices
                            }
                        }
                    }
                } else if (GEN && li.present) {
                    int sts[2] = {0, 0}, ens[2] = {0, 0};
                    const int nr = general_ranges(ax, w, offs, l, i, j, s32, sts, ens);
                    if (side < nr) {
                        st = sts[side];
                        len = ens[side] - sts[side];
                        kind = (unsigned)l | ((unsigned)side << 4) | 32u;
                    }
                }
            }
            int incl = len;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
                if (lane >= d) incl += t;
            }
            const unsigned ne = __ballot_sync(0xFFFFFFFFu, len > 0);
            if (len > 0) {
                const int ct = __popc(ne & lanes_below());
                S.seg_pre[ct] = incl - len;
                S.seg_start[ct] = st;
                S.seg_kind[ct] = kind;
                S.seg_g[ct] = gv;
            }
            if (lane == 31) {
                S.n_seg = __popc(ne);
                S.total = incl;
            }
        }
        group_sync<WPC>();
        // steps 2-4, chunk by chunk: a membership pass lists the members of ranks [lo, lo + CAP)
        // (the first also counts them all), their runs are formed, and the kept members vote
        unsigned best = 0u, votes = 0u;
        int rlo = INT_MAX, rhi = -1;
        int lo = 0;
        auto to_chunk = [&](int r, int p, unsigned kd, float z) {
            if (r >= lo && r < lo + CAP) S.par[r - lo] = make_int4(p, (int)kd, __float_as_int(z), 0);
        };
        const int n = scan_members<WPC, CAP, MAXP, NL, GEN, true>(ax, w, S, hot, fsort, zsort, cold, i, j, s32, refine_eps,
                                                             to_chunk);
        int written = n, listed = 0;   // members in the pool slot / written by step 3
        int32_t *pool = nullptr;
        if (KEEP && w.keep_members) {
            // the event's member pool is shared by all its candidates: the count known, a slot is
            // reserved now, and the runs' pass lists each member as it reads the member's entry
            if (tid == 0) {
                const unsigned reserved = n ? atomicAdd(&w.stats[ev].pool_used, (unsigned)n) : 0u;
                const long long room = (long long)w.max_members - (long long)reserved;
                S.pool_base = (int)min((long long)reserved, (long long)w.max_members);
                S.pool_written = n ? (int)max(0LL, min((long long)n, room)) : 0;
            }
            group_sync<WPC>();
            const int base = S.pool_base;
            written = S.pool_written;
            if (tid == 0) {
                w.mem_start[(int64_t)ev * w.max_cand + c] = base;
                w.mem_count[(int64_t)ev * w.max_cand + c] = written;
            }
            pool = w.mem_pool + (int64_t)ev * w.max_members + base;
            listed = written;
        }
        while (lo < n) {
            if (lo > 0) {
                group_sync<WPC>();   // the previous chunk's votes have read its members
                scan_members<WPC, CAP, MAXP, NL, GEN, true>(ax, w, S, hot, fsort, zsort, cold, i, j, s32, refine_eps, to_chunk);
            }
            group_sync<WPC>();   // the chunk's list is complete
            const ChunkOut co = chunk_runs<WPC, CAP, MAXP, NL, GEN, KEEP>(ax, S, cold, i, min(n - lo, CAP), rlo, rhi, pool,
                                                                          lo, listed);
            group_sync<WPC>();   // its runs and start bits are complete
            vote_pairs<WPC, CAP, MAXP, NL, P10>(ax, S, grid, co.npairs, best, votes);
            lo += co.consumed;
        }
        // step 5: the group's best key and votes, the final mask of its cell, the touched rows cleared
        best = __reduce_max_sync(0xFFFFFFFFu, best);
        votes = __reduce_add_sync(0xFFFFFFFFu, votes);
        rlo = (int)__reduce_min_sync(0xFFFFFFFFu, (unsigned)rlo);
        rhi = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)(rhi + 1)) - 1;
        if (WPC > 1) {   // the warps' results combined in one exchange
            if (lane == 0) {
                S.wtmp[4 * wg] = (int)best;
                S.wtmp[4 * wg + 1] = (int)votes;
                S.wtmp[4 * wg + 2] = rlo;
                S.wtmp[4 * wg + 3] = rhi;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < WPC; ++k) {
                best = max(best, (unsigned)S.wtmp[4 * k]);
                votes += k == wg ? 0u : (unsigned)S.wtmp[4 * k + 1];
                rlo = min(rlo, S.wtmp[4 * k + 2]);
                rhi = max(rhi, S.wtmp[4 * k + 3]);
            }
            __syncthreads();
        }
        group_sync<WPC>();   // every vote has landed
        const unsigned cell = best ? 0xFFFFu - (best & 0xFFFFu) : 0u;
        const uint32_t mask2 = best ? grid_mask<P10>(grid, cell) : 0u;
        group_sync<WPC>();   // read before the clear
        clear_rows<WPC, P10>(ax, grid, rlo, rhi);
        if (tid == 0) {
            hough_candidate out = cd;
            out.n_members = (uint32_t)n;
            out.icot = cell / (unsigned)ax.n_z0;
            out.jz0 = cell % (unsigned)ax.n_z0;
            out.mask2 = mask2;
            out.flags = ((int)(best >> 16) >= min(ax.threshold, ax.n_layers) ? 1u : 0u) | (written < n ? 2u : 0u);
            store_candidate(cands + c, out);
            if (ev != acc_e) {
                if (acc_e >= 0) {
                    if (acc_members) atomicAdd(&w.stats[acc_e].n_members, acc_members);
                    if (acc_votes) atomicAdd(&w.stats[acc_e].stage2_votes, acc_votes);
                }
                acc_e = ev;
                acc_members = 0u;
                acc_votes = 0ull;
            }
            acc_members += (unsigned)n;
            acc_votes += (unsigned long long)votes;
        }
        group_sync<WPC>();   // the grid is clear and the scratch free for the next candidate
    }
    if (tid == 0 && acc_e >= 0) {
        if (acc_members) atomicAdd(&w.stats[acc_e].n_members, acc_members);
        if (acc_votes) atomicAdd(&w.stats[acc_e].stage2_votes, acc_votes);
    }
}

// Membership and stage 2 of every candidate of every event, a group of WPC warps per candidate.
template <int WPC, int CAP, int MAXP, int NL, bool P10>
__global__ void __launch_bounds__(WPC == 1 ? 32 * kBatchGroups : 32 * WPC, WPC == 1 ? (P10 ? 8 : 5) : 1)
    confirm_kernel(Axes ax, Workspace w, float s32, float refine_eps, int grid_words, int scratch_bytes,
                   int bands_at, int many_groups, int many_scratch_bytes)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_c[];
    __shared__ LayerInfo s_info[HOUGH_MAX_LAYERS];
    __shared__ int s_general;
    const int ngroups = WPC == 1 ? (int)(blockDim.x >> 5) : 1;
    const int gidx = WPC == 1 ? (int)(threadIdx.x >> 5) : 0;
    Scratch<WPC, CAP, MAXP, NL> &S = *reinterpret_cast<Scratch<WPC, CAP, MAXP, NL> *>(smem_c + (size_t)gidx * scratch_bytes);
    uint32_t *grid = reinterpret_cast<uint32_t *>(smem_c + (size_t)ngroups * scratch_bytes) + (size_t)gidx * grid_words;
    // the layer records are requested first and stored last, so that their round trip overlaps the
    // band counts' (or the candidate total's)
    LayerInfo li{};
    if (threadIdx.x < HOUGH_MAX_LAYERS) li = w.info[threadIdx.x];
    // one event of a context whose candidate list was not compacted: every CTA scans the band counts
    // into shared memory (behind the groups' scratch and grids) and reads its candidates from the
    // band lists; the first CTA records the totals the compaction would have
    int total;
    const int *band_offs = nullptr;
    if (WPC > 1 && w.cands_from_bands) {   // (batches use one-warp groups and a compacted list)
        int *bo = reinterpret_cast<int *>(smem_c + bands_at);
        const int nb = n_bands(ax, w.band_rows);
        const int found = block_excl_scan(w.band_counts, nb, bo);
        total = min(found, w.max_cand);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            w.stats[0].n_candidates = (unsigned)found;
            if (found > w.max_cand) atomicOr(&w.stats[0].device_error, HOUGH_DEVERR_CAND);
            w.cand_base[0] = 0;
            w.cand_base[1] = total;
            w.counters->total_cands = (unsigned)total;
        }
        band_offs = bo;
    } else {
        total = (int)w.counters->total_cands;
    }
    if constexpr (WPC > 1) {
        if (many_groups && total > kManyPerCta * (int)gridDim.x) {
            // one event with many candidates (a fine grid, a busy event): each warp confirms its
            // own candidates with its own scratch and grid, as in batches, instead of four warps
            // sharing one candidate's chain
            using S1 = Scratch<1, kBatchCap, kBatchPairs, NL>;
            const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
            S1 &s1 = *reinterpret_cast<S1 *>(smem_c + (size_t)g * many_scratch_bytes);
            uint32_t *grid1 = reinterpret_cast<uint32_t *>(smem_c + (size_t)many_groups * many_scratch_bytes) +
                              (size_t)g * grid_words;
            if (g < many_groups) {
                for (int q = lane; q < grid_words; q += 32) grid1[q] = 0u;
                for (int q = lane; q < (int)(sizeof(S1) / 4); q += 32) reinterpret_cast<uint32_t *>(&s1)[q] = 0u;
            }
            if (threadIdx.x < HOUGH_MAX_LAYERS) s_info[threadIdx.x] = li;
            __syncthreads();
            if (threadIdx.x == 0) {
                int gen = 0;
                for (int l = 0; l < ax.n_layers; ++l) gen |= s_info[l].present && !s_info[l].uniform;
                s_general = gen;
            }
            __syncthreads();
            if (g >= many_groups) return;
            if (s_general)
                confirm_all<1, kBatchCap, kBatchPairs, NL, P10, true, true>(ax, w, s32, refine_eps, s1, grid1, s_info,
                                                                            many_groups, g, total, band_offs);
            else
                confirm_all<1, kBatchCap, kBatchPairs, NL, P10, false, true>(ax, w, s32, refine_eps, s1, grid1, s_info,
                                                                             many_groups, g, total, band_offs);
            return;
        }
    }
    for (int q = group_tid<WPC>(); q < grid_words; q += 32 * WPC) grid[q] = 0u;
    // the scratch starts zeroed: lanes past a list read its terms without a branch
    for (int q = group_tid<WPC>(); q < (int)(sizeof(Scratch<WPC, CAP, MAXP, NL>) / 4); q += 32 * WPC)
        reinterpret_cast<uint32_t *>(&S)[q] = 0u;
    if (threadIdx.x < HOUGH_MAX_LAYERS) s_info[threadIdx.x] = li;
    __syncthreads();
    if (threadIdx.x == 0) {
        int g = 0;
        for (int l = 0; l < ax.n_layers; ++l) g |= s_info[l].present && !s_info[l].uniform;
        s_general = g;
    }
    __syncthreads();
    // (one-warp kernels run batches, which keep no member lists)
    if (s_general)
        confirm_all<WPC, CAP, MAXP, NL, P10, true, (WPC > 1)>(ax, w, s32, refine_eps, S, grid, s_info, ngroups, gidx, total,
                                                              band_offs);
    else
        confirm_all<WPC, CAP, MAXP, NL, P10, false, (WPC > 1)>(ax, w, s32, refine_eps, S, grid, s_info, ngroups, gidx, total,
                                                               band_offs);
}

__global__ void member_index_kernel(Workspace w, int32_t *idx_out, int64_t total)
{
    pdl_enter();
    const ColdHit *cold = w.cold + w.hit_start[0];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
        idx_out[q] = cold[w.mem_pool[q]].idx;
}

// Words of a grid of 16-bit masks, two to a word, or of 10-bit masks, three to a word, rounded up
// to whole 16-byte vectors.
int grid_words_for(const Axes &ax, bool p10)
{
    const int cells = ax.n_cot * ax.n_z0;
    return ((p10 ? (cells + 2) / 3 : (cells + 1) / 2) + 3) & ~3;
}

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

std::atomic<unsigned long long> g_ctas[4];
std::atomic<int> g_smem_optin{-1};

int smem_optin()
{
    int m = g_smem_optin.load(std::memory_order_relaxed);
    if (m < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&m, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) m = 48 * 1024;
        g_smem_optin.store(m, std::memory_order_relaxed);
    }
    return m;
}

template <int WPC, int CAP, int MAXP, int NL, bool P10>
cudaError_t launch_confirm(const Axes &ax, const Workspace &w, int sms, float s32, float refine_eps,
                           cudaStream_t stream, std::atomic<unsigned long long> &memo)
{
    auto kernel = confirm_kernel<WPC, CAP, MAXP, NL, P10>;
    const int words = grid_words_for(ax, P10);
    const size_t scratch = (sizeof(Scratch<WPC, CAP, MAXP, NL>) + 15) & ~(size_t)15;
    const size_t per_group = scratch + (size_t)words * 4;
    // one-warp groups: as many per CTA (up to kBatchGroups) as shared memory holds
    const int room = smem_optin() - (int)(sizeof(LayerInfo) * HOUGH_MAX_LAYERS) - 1024;
    const int groups = WPC == 1 ? std::max(1, std::min(kBatchGroups, room / (int)per_group)) : 1;
    // a group of several warps may split into one-warp groups when its event has many candidates:
    // room for WPC one-warp scratches and grids too, when they fit beside the bands
    const size_t many_scratch = (sizeof(Scratch<1, kBatchCap, kBatchPairs, NL>) + 15) & ~(size_t)15;
    const size_t many_bytes = (size_t)WPC * (many_scratch + (size_t)words * 4);
    const int many = WPC > 1 && many_bytes <= 128 * 1024 ? WPC : 0;
    const size_t layout = std::max((size_t)groups * per_group, many ? many_bytes : (size_t)0);
    const size_t smem = layout + (w.cands_from_bands ? ((size_t)n_bands(ax, w.band_rows) + 1) * sizeof(int) : 0);
    cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (!err) err = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (err) return err;
    const int threads = 32 * WPC * groups;
    const int ctas = resident_ctas(kernel, threads, smem, memo);
    // the number of candidates is known on the device only: a persistent grid of exactly the
    // resident CTAs, each group striding over the flattened (event, candidate) work
    return launch_chained(kernel, dim3(ctas * sms), dim3(threads), smem, stream, ax, w, s32, refine_eps, words,
                          (int)scratch, (int)layout, many, (int)many_scratch);
}

}  // namespace

size_t stage2_smem_bytes(const Axes &ax) { return (size_t)grid_words_for(ax, false) * 4; }

bool stage2_reads_bands(const Axes &ax, int band_rows) { return n_bands(ax, band_rows) <= kMaxBandsRead; }

cudaError_t launch_stage2(const Axes &ax, const Workspace &w, int sms, float refine_eps, cudaStream_t stream,
                          cudaEvent_t between)
{
    const float s32 = (float)(ax.n_phi * kInvTwoPi);
    if (w.keep_members && w.n_events != 1) return cudaErrorInvalidValue;   // only single events keep member lists
    cudaError_t err;
    if (w.n_events == 1) {
        // one event: a few hundred candidates, each a chain of dependent steps, so four warps share one
        err = launch_confirm<kEventWarps, kEventCap, kEventPairs, HOUGH_MAX_LAYERS, false>(ax, w, sms, s32, refine_eps, stream, g_ctas[0]);
    } else if (ax.n_layers <= 10) {
        // a batch: a warp per candidate, the grid's masks packed three to a word so more warps fit an SM
        err = launch_confirm<1, kBatchCap, kBatchPairs, 10, true>(ax, w, sms, s32, refine_eps, stream, g_ctas[1]);
    } else {
        err = launch_confirm<1, kBatchCap, kBatchPairs, HOUGH_MAX_LAYERS, false>(ax, w, sms, s32, refine_eps, stream, g_ctas[2]);
    }
    if (err) return err;
    if (between && (err = cudaEventRecord(between, stream))) return err;
    return cudaSuccess;
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
