// Peak search (Sec. 4, second step; Sec. 8: "regular memory access ... and a non-trivial
// reduction"), candidate membership and the confirmation vote in (cot theta, z0).
//
// Peaks: one CTA per (event, band of kPeakRows rows).  The band plus one halo row on each side
// is read once from HBM as 16-byte vectors and reduced to layer counts (popcount) in shared
// memory; each thread then tests cells in raster order and a block-wide ballot prefix gives every
// candidate its rank.  A first pass counts candidates per band, a per-event scan turns counts into
// offsets, and a second pass writes the candidates, so the list is in raster order without a sort.
//
// Membership: one warp per candidate.  Only layers present in the candidate's mask can hold
// members.  For a uniform-radius layer the table inverts the vote exactly: a hit of bin
// J votes into column j on row i when J = j + I_i + (f < g_i), so two buckets of the sorted
// hits hold all candidates' members.  Other layers scan the window of buckets their radius range
// allows and redo the vote per hit.
//
// Stage 2: one CTA per candidate with the n_cot x n_z0 grid of layer masks in shared memory.  For
// a member with arc length s the z0 coordinate w(m) = n_z0 (z - s t_m - z0_min) / (z0_max - z0_min)
// is linear in m; it is evaluated in FP32 around the member's own crossing row m_ref, and a vote
// within kStage2Eps of a z0 edge is recomputed in FP64 exactly as the definition reads.
#include "hough_internal.cuh"

namespace hough {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kMemberWarps = 8;
constexpr int kStage2Threads = 256;
constexpr int kStage2Chunk = 512;

__device__ __forceinline__ int wrap_col(int j, int n)
{
    j += j < 0 ? n : 0;
    return j >= n ? j - n : j;
}

template <bool WRITE>
__global__ void __launch_bounds__(kPeakThreads) peak_kernel(Axes ax, Workspace w)
{
    extern __shared__ __align__(16) unsigned char pc[];   // (kPeakRows + 2) x n_phi layer counts
    __shared__ int s_warp[kPeakThreads / 32];
    const int nb = n_bands(ax);
    const int e = blockIdx.x / nb, band = blockIdx.x - e * nb;
    const int nphi = ax.n_phi;
    const int i0 = band * kPeakRows;
    const int nrows = min(kPeakRows, ax.n_qpt - i0);
    const uint16_t *M = w.M + (int64_t)e * ax.n_qpt * nphi;

    // layer counts of rows i0-1 .. i0+nrows (rows outside the grid count as empty)
    const int v8 = nphi >> 3;
    for (int q = threadIdx.x; q < (nrows + 2) * v8; q += kPeakThreads) {
        const int rr = q / v8, c8 = q - rr * v8;
        const int i = i0 - 1 + rr;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (i >= 0 && i < ax.n_qpt) v = *reinterpret_cast<const uint4 *>(M + (int64_t)i * nphi + c8 * 8);
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

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ncell = nrows * nphi;
    int running = 0;
    const int out_base = WRITE ? w.band_offs[(int64_t)e * nb + band] : 0;
    hough_candidate *cands = w.cands + (int64_t)e * w.max_cand;
    for (int base = 0; base < ncell; base += kPeakThreads) {
        const int cell = base + threadIdx.x;
        bool is_peak = false;
        int rr = 0, j = 0;
        if (cell < ncell) {
            rr = cell / nphi;
            j = cell - rr * nphi;
            const unsigned char *row = pc + (rr + 1) * nphi;
            const int p = row[j];
            if (p >= ax.threshold) {
                const int jm = wrap_col(j - 1, nphi), jp = wrap_col(j + 1, nphi);
                const unsigned char *up = row - nphi, *dn = row + nphi;
                // the four raster-preceding neighbours must be strictly lower, the others not higher
                is_peak = up[jm] < p && up[j] < p && up[jp] < p && row[jm] < p &&
                          row[jp] <= p && dn[jm] <= p && dn[j] <= p && dn[jp] <= p;
            }
        }
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, is_peak);
        if (lane == 0) s_warp[warp] = __popc(ball);
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int q = 0; q < kPeakThreads / 32; ++q) {
            const int c = s_warp[q];
            before += q < warp ? c : 0;
            total += c;
        }
        if (WRITE && is_peak) {
            const int idx = out_base + running + before + __popc(ball & ((1u << lane) - 1u));
            if (idx < w.max_cand) {
                hough_candidate c;
                c.iq = (uint32_t)(i0 + rr);
                c.jphi = (uint32_t)j;
                c.mask = M[(int64_t)(i0 + rr) * nphi + j];
                c.n_members = 0u;
                c.icot = c.jz0 = c.mask2 = c.flags = 0u;
                cands[idx] = c;
            }
        }
        running += total;
        __syncthreads();
    }
    if (!WRITE && threadIdx.x == 0) w.band_counts[(int64_t)e * nb + band] = running;
}

// Block-wide exclusive scan of n int32 counts into offsets (int32 or int64); returns the total.
template <typename OffT>
__device__ long long block_exclusive_scan(const int32_t *counts, OffT *offs, int n)
{
    __shared__ long long s_warp[kScanThreads / 32];
    __shared__ long long s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += kScanThreads) {
        const int k = base + threadIdx.x;
        const long long v = k < n ? counts[k] : 0;
        long long incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            long long wv = s_warp[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const long long t = __shfl_up_sync(0xFFFFFFFFu, wv, d);
                if (lane >= d) wv += t;
            }
            s_warp[lane] = wv;
        }
        __syncthreads();
        const long long excl = s_carry + (warp > 0 ? s_warp[warp - 1] : 0) + incl - v;
        if (k < n) offs[k] = (OffT)excl;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) s_carry = excl + v;
        __syncthreads();
    }
    return s_carry;
}

__global__ void __launch_bounds__(kScanThreads) band_scan_kernel(Axes ax, Workspace w)
{
    const int e = blockIdx.x;
    const int nb = n_bands(ax);
    const long long total = block_exclusive_scan(w.band_counts + (int64_t)e * nb, w.band_offs + (int64_t)e * nb, nb);
    if (threadIdx.x == 0) {
        w.stats[e].n_candidates = (unsigned)total;
        if (total > w.max_cand) atomicOr(&w.stats[e].device_error, HOUGH_DEVERR_CAND);
    }
}

__device__ __forceinline__ int event_cands(const Workspace &w, int e)
{
    return (int)min((unsigned)w.max_cand, w.stats[e].n_candidates);
}

// Member hits of candidate (i, j) on one layer, visited by the 32 lanes of a warp.  `visit` is
// called with (has_member, staged position) once per lane per step, by all lanes together.
template <typename Visit>
__device__ void for_layer_members(const Axes &ax, const Workspace &w, int e, int l, int i, int j,
                                  float s32, float refine_eps, Visit visit)
{
    const int lane = threadIdx.x & 31;
    const int nphi = ax.n_phi;
    const int nkeys = ax.n_layers * nphi;
    const int32_t *offs = w.offs + (int64_t)e * (nkeys + 1);
    const int64_t hstart = w.hit_start[e];
    const HotHit *hot = w.hot + hstart;
    const LayerInfo li = w.info[l];
    if (li.uniform) {
        if (i < li.lo || i > li.hi) return;
        const TabEntry te = w.tab[l * ax.n_qpt + i];
        // J = j + I (f >= g) or J = j + I + 1 (f < g)
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int J = wrap_col(((j + te.I + side) % nphi + nphi) % nphi, nphi);
            const int a = offs[l * nphi + J], b = offs[l * nphi + J + 1];
            for (int base = a; base < b; base += 32) {
                const int pos = base + lane;
                bool mem = false;
                if (pos < b) {
                    const float f = hot[pos].f;
                    mem = side == 0 ? !(f < te.g) : (f < te.g);
                }
                visit(mem, pos);
            }
        }
        return;
    }
    // per-vote layer: the window of buckets allowed by the layer's radius range on row i
    const float k = w.kq32[i];
    const float c_lo = 0.15f * (float)ax.b / 100.f * __uint_as_float(w.radii->rmin[l]) * 0.999f;
    const float c_hi = 0.15f * (float)ax.b / 100.f * __uint_as_float(w.radii->rmax[l]) * 1.001f;
    const float a1 = asinf(fminf(fmaxf(c_lo * k, -1.f), 1.f));
    const float a2 = asinf(fminf(fmaxf(c_hi * k, -1.f), 1.f));
    const int ja = (int)floorf(j + s32 * fminf(a1, a2)) - 2;
    const int jb = (int)floorf(j + 1 + s32 * fmaxf(a1, a2)) + 2;
    const int lstart = offs[l * nphi], lend = offs[(l + 1) * nphi];
    int st[2], en[2], nr;
    if (jb - ja + 1 >= nphi) {
        nr = 1; st[0] = lstart; en[0] = lend;
    } else {
        const int a = ((ja % nphi) + nphi) % nphi, b = ((jb % nphi) + nphi) % nphi;
        if (a <= b) {
            nr = 1; st[0] = offs[l * nphi + a]; en[0] = offs[l * nphi + b + 1];
        } else {
            nr = 2; st[0] = offs[l * nphi + a]; en[0] = lend; st[1] = lstart; en[1] = offs[l * nphi + b + 1];
        }
    }
    const ColdHit *cold = w.cold + hstart;
    for (int q = 0; q < nr; ++q) {
        for (int base = st[q]; base < en[q]; base += 32) {
            const int pos = base + lane;
            bool mem = false;
            if (pos < en[q]) {
                const HotHit hh = hot[pos];
                const int rlo = (int)(hh.rows & 0xFFFFu), rhi = (int)(hh.rows >> 16);
                if (i >= rlo && i <= rhi) {
                    const float x = fminf(fmaxf(hh.c * k, -1.f), 1.f);
                    const float vq = fmaf(-asinf(x), s32, hh.f);
                    const float fl = floorf(vq);
                    const float d = vq - fl;
                    int jj = (int)(hh.jl & 0xFFFFu) + (int)fl;
                    if (d < refine_eps || d > 1.f - refine_eps || fabsf(x) > kRefineXLim) {
                        const ColdHit ch = cold[pos];
                        jj = exact_bin(ax, (double)ch.phi, __dmul_rn(sagitta_coef(ax, (double)ch.r), qpt_centre(ax, i)));
                    }
                    mem = wrap_col(jj, nphi) == j;
                }
            }
            visit(mem, pos);
        }
    }
}

template <bool WRITE>
__global__ void __launch_bounds__(kMemberWarps * 32) member_kernel(Axes ax, Workspace w, float s32, float refine_eps)
{
    const int e = blockIdx.y;
    const int ncand = event_cands(w, e);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const hough_candidate *cands = w.cands + (int64_t)e * w.max_cand;
    for (int c = blockIdx.x * kMemberWarps + warp; c < ncand; c += gridDim.x * kMemberWarps) {
        const hough_candidate cd = cands[c];
        int count = 0;
        long long base = WRITE ? w.mem_offs[(int64_t)e * (w.max_cand + 1) + c] : 0;
        int32_t *out = w.mem_pos + (int64_t)e * w.max_members;
        uint32_t layers = cd.mask;
        while (layers) {
            const int l = __ffs(layers) - 1;
            layers &= layers - 1;
            for_layer_members(ax, w, e, l, (int)cd.iq, (int)cd.jphi, s32, refine_eps, [&](bool mem, int pos) {
                const unsigned ball = __ballot_sync(0xFFFFFFFFu, mem);
                if (WRITE && mem) {
                    const long long at = base + count + __popc(ball & ((1u << lane) - 1u));
                    if (at < w.max_members) out[at] = pos;
                }
                count += __popc(ball);
            });
        }
        if (!WRITE && lane == 0) w.mem_counts[(int64_t)e * w.max_cand + c] = count;
    }
}

__global__ void __launch_bounds__(kScanThreads) member_scan_kernel(Workspace w)
{
    const int e = blockIdx.x;
    const int ncand = event_cands(w, e);
    int64_t *offs = w.mem_offs + (int64_t)e * (w.max_cand + 1);
    const long long total = block_exclusive_scan(w.mem_counts + (int64_t)e * w.max_cand, offs, ncand);
    if (threadIdx.x == 0) {
        offs[ncand] = total;
        w.stats[e].n_members = (unsigned)min(total, (long long)0xFFFFFFFFu);
        if (total > w.max_members) atomicOr(&w.stats[e].device_error, HOUGH_DEVERR_MEMBERS);
    }
}

// z0 coordinate of one stage-2 vote exactly as the definition reads (FP64, nothing fused).
__device__ __forceinline__ double exact_z0_coord(const Axes &ax, double z, double s, int m)
{
    const double t = __dadd_rn(ax.cot_min, __dmul_rn((double)m + 0.5, ax.dt));
    const double z0 = __dsub_rn(z, __dmul_rn(s, t));
    return __ddiv_rn(__dmul_rn((double)ax.n_z0, __dsub_rn(z0, ax.z0_min)), __dsub_rn(ax.z0_max, ax.z0_min));
}

__global__ void __launch_bounds__(kStage2Threads) stage2_kernel(Axes ax, Workspace w)
{
    extern __shared__ __align__(16) unsigned char smem2[];
    uint32_t *grid2 = reinterpret_cast<uint32_t *>(smem2);           // n_cot * n_z0 masks, 2 per word
    const int ncell = ax.n_cot * ax.n_z0;
    const int nwords = (ncell + 1) >> 1;
    double *m_s = reinterpret_cast<double *>(grid2 + ((nwords + 1) & ~1));
    float *m_z = reinterpret_cast<float *>(m_s + kStage2Chunk);
    float *m_a = m_z + kStage2Chunk;
    float *m_b = m_a + kStage2Chunk;
    int *m_ref = reinterpret_cast<int *>(m_b + kStage2Chunk);
    int *m_l = m_ref + kStage2Chunk;
    __shared__ unsigned long long s_best[kStage2Threads / 32];
    __shared__ unsigned long long s_votes;

    const int e = blockIdx.y;
    const int ncand = event_cands(w, e);
    const int64_t hstart = w.hit_start[e];
    const ColdHit *cold = w.cold + hstart;
    const HotHit *hot = w.hot + hstart;
    const int64_t *moffs = w.mem_offs + (int64_t)e * (w.max_cand + 1);
    const int32_t *mpos = w.mem_pos + (int64_t)e * w.max_members;
    hough_candidate *cands = w.cands + (int64_t)e * w.max_cand;
    const double zscale = __ddiv_rn((double)ax.n_z0, __dsub_rn(ax.z0_max, ax.z0_min));
    const double t0 = __dadd_rn(ax.cot_min, __dmul_rn(0.5, ax.dt));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_votes = 0ull;

    for (int c = blockIdx.x; c < ncand; c += gridDim.x) {
        const hough_candidate cd = cands[c];
        const int i = (int)cd.iq;
        const long long mb = moffs[c], me_full = moffs[c + 1];
        const long long me = min(me_full, (long long)w.max_members);
        const double k = qpt_centre(ax, i);
        for (int q = threadIdx.x; q < nwords; q += kStage2Threads) grid2[q] = 0u;
        unsigned long long votes = 0;
        for (long long cb = mb; cb < me; cb += kStage2Chunk) {
            const int nm = (int)min((long long)kStage2Chunk, me - cb);
            __syncthreads();
            // per member: arc length (FP64) and the linear z0 coordinate around its crossing row
            for (int q = threadIdx.x; q < nm; q += kStage2Threads) {
                const int pos = mpos[cb + q];
                const ColdHit ch = cold[pos];
                const int l = (int)((hot[pos].jl >> 16) & 0xFu);
                const LayerInfo li = w.info[l];
                double s;
                if (li.uniform) {
                    s = w.arc[l * ax.n_qpt + i];
                } else {
                    const double r = (double)ch.r;
                    const double axv = fabs(__dmul_rn(sagitta_coef(ax, r), k));
                    s = axv > 0.0 ? __ddiv_rn(__dmul_rn(r, asin(axv)), axv) : r;
                }
                const double A = __dmul_rn(zscale, __dsub_rn(__dsub_rn((double)ch.z, ax.z0_min), __dmul_rn(s, t0)));
                const double B = __dmul_rn(zscale, __dmul_rn(s, ax.dt));
                int mref = 0;
                if (B > 0.0) mref = (int)fmin(fmax(rint(A / B), 0.0), (double)(ax.n_cot - 1));
                m_s[q] = s;
                m_z[q] = ch.z;
                m_a[q] = (float)(A - (double)mref * B);
                m_b[q] = (float)B;
                m_ref[q] = mref;
                m_l[q] = l;
            }
            __syncthreads();
            for (int pq = threadIdx.x; pq < nm * ax.n_cot; pq += kStage2Threads) {
                const int q = pq / ax.n_cot, m = pq - q * ax.n_cot;
                const float wv = fmaf(-(float)(m - m_ref[q]), m_b[q], m_a[q]);
                const float fl = floorf(wv);
                const float d = wv - fl;
                int n;
                if (d < kStage2Eps || d > 1.f - kStage2Eps) {
                    n = (int)floor(exact_z0_coord(ax, (double)m_z[q], m_s[q], m));
                } else {
                    n = (int)fl;
                    if (wv < -1.f || wv > (float)ax.n_z0 + 1.f) n = -1;
                }
                if (n >= 0 && n < ax.n_z0) {
                    const int cell = m * ax.n_z0 + n;
                    atomicOr(&grid2[cell >> 1], (1u << m_l[q]) << ((cell & 1) << 4));
                    ++votes;
                }
            }
        }
        __syncthreads();
        // maximum layer count, lowest row-major cell on ties: key = count << 32 | (ncell - cell)
        unsigned long long best = 0ull;
        for (int cell = threadIdx.x; cell < ncell; cell += kStage2Threads) {
            const uint32_t m16 = (grid2[cell >> 1] >> ((cell & 1) << 4)) & 0xFFFFu;
            const unsigned long long key = ((unsigned long long)__popc(m16) << 32) | (unsigned)(ncell - cell);
            best = key > best ? key : best;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, best, d);
            best = o > best ? o : best;
        }
        if (lane == 0) s_best[warp] = best;
        if (votes) atomicAdd(&s_votes, votes);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long b = s_best[0];
            for (int q = 1; q < kStage2Threads / 32; ++q) b = s_best[q] > b ? s_best[q] : b;
            const int cell = ncell - (int)(b & 0xFFFFFFFFu);
            const uint32_t m16 = (grid2[cell >> 1] >> ((cell & 1) << 4)) & 0xFFFFu;
            hough_candidate out = cd;
            out.n_members = (uint32_t)(me_full - mb);
            out.icot = (uint32_t)(cell / ax.n_z0);
            out.jz0 = (uint32_t)(cell % ax.n_z0);
            out.mask2 = m16;
            out.flags = (__popc(m16) >= ax.threshold ? 1u : 0u) | (me < me_full ? 2u : 0u);
            cands[c] = out;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && s_votes) atomicAdd(&w.stats[e].stage2_votes, s_votes);
}

__global__ void member_index_kernel(Workspace w, int32_t *idx_out, int64_t total)
{
    const ColdHit *cold = w.cold + w.hit_start[0];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
        idx_out[q] = cold[w.mem_pos[q]].idx;
}

}  // namespace

cudaError_t launch_member_index(const Workspace &w, int32_t *idx_out, int64_t total, cudaStream_t stream)
{
    if (total <= 0) return cudaSuccess;
    const int g = (int)min((total + 255) / 256, (int64_t)4096);
    member_index_kernel<<<g, 256, 0, stream>>>(w, idx_out, total);
    return cudaGetLastError();
}

cudaError_t launch_peaks(const Axes &ax, const Workspace &w, cudaStream_t stream)
{
    const int nb = n_bands(ax);
    const size_t smem = (size_t)(kPeakRows + 2) * ax.n_phi;
    cudaError_t err;
    if ((err = cudaFuncSetAttribute(peak_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return err;
    if ((err = cudaFuncSetAttribute(peak_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return err;
    peak_kernel<false><<<w.n_events * nb, kPeakThreads, smem, stream>>>(ax, w);
    band_scan_kernel<<<w.n_events, kScanThreads, 0, stream>>>(ax, w);
    peak_kernel<true><<<w.n_events * nb, kPeakThreads, smem, stream>>>(ax, w);
    return cudaGetLastError();
}

size_t stage2_smem_bytes(const Axes &ax)
{
    const int nwords = (ax.n_cot * ax.n_z0 + 1) >> 1;
    return (size_t)((nwords + 1) & ~1) * 4 + (size_t)kStage2Chunk * (8 + 4 * 5);
}

cudaError_t launch_stage2(const Axes &ax, const Workspace &w, int sms, cudaStream_t stream)
{
    const float s32 = (float)(ax.n_phi * kInvTwoPi);
    const float eps = refine_eps_for(ax);
    // candidates per event are known on the device only: size the grids for the worst case and
    // let each CTA stride over the event's candidates
    int y = (4 * sms + w.n_events - 1) / w.n_events;
    y = max(1, min(y, (w.max_cand + kMemberWarps - 1) / kMemberWarps));
    dim3 gm(y, w.n_events);
    member_kernel<false><<<gm, kMemberWarps * 32, 0, stream>>>(ax, w, s32, eps);
    member_scan_kernel<<<w.n_events, kScanThreads, 0, stream>>>(w);
    member_kernel<true><<<gm, kMemberWarps * 32, 0, stream>>>(ax, w, s32, eps);
    const size_t smem = stage2_smem_bytes(ax);
    cudaError_t err = cudaFuncSetAttribute(stage2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err) return err;
    int y2 = (8 * sms + w.n_events - 1) / w.n_events;
    y2 = max(1, min(y2, w.max_cand));
    stage2_kernel<<<dim3(y2, w.n_events), kStage2Threads, smem, stream>>>(ax, w);
    return cudaGetLastError();
}

}  // namespace hough
