// Confirmation of the candidates (Sec. 4: candidates found as local maxima are confirmed by "more
// expensive computations"): for each candidate, the hits whose stage-1 vote fell in its cell
// (membership) and their vote in a (cot theta, z0) grid (stage 2), in one kernel.
//
// One CTA per candidate at a time.  Membership: only layers present in the candidate's mask can
// hold members.  For a table layer the vote inverts exactly -- a hit of bucket J votes into column
// j on row i when J = j + I_i + (f < g_i) -- so two buckets of the sorted hits hold all of that
// layer's members; other layers scan the buckets their radius range allows and redo the vote per
// hit (FP32 with FP64 refinement, as in the vote kernel).  Members are enumerated in a fixed order
// (layer, bucket, position), so chunks of them can be re-enumerated when a candidate has more
// members than shared memory holds.
//
// Stage 2: the n_cot x n_z0 grid of layer masks lives in shared memory.  For a member with arc
// length s the z0 coordinate w(m) = n_z0 (z - s t_m - z0_min) / (z0_max - z0_min) is linear in the
// cot row m; it is evaluated in FP32 around the member's own crossing row m_ref, and a vote within
// kStage2Eps of a z0 edge is recomputed in FP64 exactly as the definition reads.  The result is the
// cell with the most layers, the lowest row-major index on ties.
#include "hough_internal.cuh"

namespace hough {

namespace {

constexpr int kConfirmThreads = 256;
constexpr int kConfirmWarps = kConfirmThreads / 32;
constexpr int kMemberChunk = 1024;

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
    const LayerInfo li = w.info[l];
    if (!li.present) return sc;
    if (li.uniform) {
        if (i < li.lo || i > li.hi) return sc;
        const TabEntry te = w.tab[l * ax.n_qpt + i];
        sc.table = 1;
        sc.g = te.g;
        sc.nr = 2;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int J = ((j + te.I + side) % nphi + nphi) % nphi;
            sc.st[side] = offs[l * nphi + J];
            sc.en[side] = offs[l * nphi + J + 1];
        }
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
    const int lstart = offs[l * nphi], lend = offs[(l + 1) * nphi];
    if (jb - ja + 1 >= nphi) {
        sc.nr = 1; sc.st[0] = lstart; sc.en[0] = lend;
    } else {
        const int a = ((ja % nphi) + nphi) % nphi, b = ((jb % nphi) + nphi) % nphi;
        if (a <= b) {
            sc.nr = 1; sc.st[0] = offs[l * nphi + a]; sc.en[0] = offs[l * nphi + b + 1];
        } else {
            sc.nr = 2; sc.st[0] = offs[l * nphi + a]; sc.en[0] = lend; sc.st[1] = lstart; sc.en[1] = offs[l * nphi + b + 1];
        }
    }
    return sc;
}

// Members of one layer, enumerated by one warp in the fixed order.  Returns their number; when
// `s_pos` is given, stores the member of rank (rank_base + local rank) in s_pos[rank - lo] if it
// lies in [lo, hi), and in pool[rank] if rank < pool_n.
__device__ int warp_layer_members(const Axes &ax, const Workspace &w, const HotHit *hot, const ColdHit *cold,
                                  const LayerScan &sc, int i, int j, float s32, float refine_eps, int rank_base,
                                  int lo, int hi, int *s_pos, int32_t *pool, int pool_n)
{
    const int lane = threadIdx.x & 31;
    int count = 0;
    for (int q = 0; q < sc.nr; ++q) {
        for (int base = sc.st[q]; base < sc.en[q]; base += 32) {
            const int pos = base + lane;
            bool mem = false;
            if (pos < sc.en[q]) {
                const HotHit hh = hot[pos];
                if (sc.table) {
                    mem = q == 0 ? !(hh.f < sc.g) : (hh.f < sc.g);
                } else {
                    const int rlo = (int)(hh.rows & 0xFFFFu), rhi = (int)(hh.rows >> 16);
                    if (i >= rlo && i <= rhi) {
                        const float x = fminf(fmaxf(hh.c * w.kq32[i], -1.f), 1.f);
                        const float vq = fmaf(-asinf(x), s32, hh.f);
                        const float fl = floorf(vq);
                        const float d = vq - fl;
                        int jj = (int)(hh.jl & 0xFFFFu) + (int)fl;
                        if (d < refine_eps || d > 1.f - refine_eps || fabsf(x) > kRefineXLim) {
                            const ColdHit ch = cold[pos];
                            jj = exact_bin(ax, (double)ch.phi, __dmul_rn(sagitta_coef(ax, (double)ch.r), qpt_centre(ax, i)));
                        }
                        mem = wrap_col(jj, ax.n_phi) == j;
                    }
                }
            }
            const unsigned ball = __ballot_sync(0xFFFFFFFFu, mem);
            if (s_pos && mem) {
                const int r = rank_base + count + __popc(ball & ((1u << lane) - 1u));
                if (r >= lo && r < hi) {
                    s_pos[r - lo] = pos;
                    if (r < pool_n) pool[r] = pos;
                }
            }
            count += __popc(ball);
        }
    }
    return count;
}

// z0 coordinate of one stage-2 vote exactly as the definition reads (FP64, nothing fused).
__device__ __forceinline__ double exact_z0_coord(const Axes &ax, double z, double s, int m)
{
    const double t = __dadd_rn(ax.cot_min, __dmul_rn((double)m + 0.5, ax.dt));
    const double z0 = __dsub_rn(z, __dmul_rn(s, t));
    return __ddiv_rn(__dmul_rn((double)ax.n_z0, __dsub_rn(z0, ax.z0_min)), __dsub_rn(ax.z0_max, ax.z0_min));
}

__global__ void __launch_bounds__(kConfirmThreads) confirm_kernel(Axes ax, Workspace w, float s32, float refine_eps)
{
    extern __shared__ __align__(16) unsigned char smem2[];
    const int ncell = ax.n_cot * ax.n_z0;
    const int nwords = (((ncell + 1) >> 1) + 1) & ~1;
    uint32_t *grid2 = reinterpret_cast<uint32_t *>(smem2);           // n_cot x n_z0 masks, 2 per word
    double *m_s = reinterpret_cast<double *>(grid2 + nwords);
    float *m_z = reinterpret_cast<float *>(m_s + kMemberChunk);
    float *m_a = m_z + kMemberChunk;
    float *m_b = m_a + kMemberChunk;
    int *m_ref = reinterpret_cast<int *>(m_b + kMemberChunk);
    int *m_l = m_ref + kMemberChunk;
    int *s_pos = m_l + kMemberChunk;
    __shared__ int s_lcount[HOUGH_MAX_LAYERS], s_loff[HOUGH_MAX_LAYERS];
    __shared__ int s_total, s_base, s_written;
    __shared__ unsigned long long s_best[kConfirmWarps];
    __shared__ unsigned long long s_votes;

    const int e = blockIdx.y;
    const int ncand = (int)min((unsigned)w.max_cand, w.stats[e].n_candidates);
    const int nkeys = ax.n_layers * ax.n_phi;
    const int64_t hstart = w.hit_start[e];
    const HotHit *hot = w.hot + hstart;
    const ColdHit *cold = w.cold + hstart;
    const int32_t *offs = w.offs + (int64_t)e * (nkeys + 1);
    int32_t *pool = w.mem_pool + (int64_t)e * w.max_members;
    hough_candidate *cands = w.cands + (int64_t)e * w.max_cand;
    const double zscale = __ddiv_rn((double)ax.n_z0, __dsub_rn(ax.z0_max, ax.z0_min));
    const double t0 = __dadd_rn(ax.cot_min, __dmul_rn(0.5, ax.dt));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_votes = 0ull;
    unsigned members_total = 0;

    for (int c = blockIdx.x; c < ncand; c += gridDim.x) {
        const hough_candidate cd = cands[c];
        const int i = (int)cd.iq, j = (int)cd.jphi;
        // count the members of each layer in the candidate's mask (warp w: layers w and w + 8)
        for (int l = warp; l < HOUGH_MAX_LAYERS; l += kConfirmWarps) {
            int n = 0;
            if (l < ax.n_layers && ((cd.mask >> l) & 1u)) {
                const LayerScan sc = layer_scan(ax, w, offs, l, i, j, s32);
                n = warp_layer_members(ax, w, hot, cold, sc, i, j, s32, refine_eps, 0, 0, 0, nullptr, nullptr, 0);
            }
            if (lane == 0) s_lcount[l] = n;
        }
        for (int q = threadIdx.x; q < nwords; q += kConfirmThreads) grid2[q] = 0u;
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int l = 0; l < HOUGH_MAX_LAYERS; ++l) {
                s_loff[l] = acc;
                acc += s_lcount[l];
            }
            s_total = acc;
            const unsigned base = acc ? atomicAdd(&w.stats[e].pool_used, (unsigned)acc) : 0u;
            const long long room = (long long)w.max_members - (long long)base;
            s_base = (int)min((long long)base, (long long)w.max_members);
            s_written = (int)max(0LL, min((long long)acc, room));
            w.mem_start[(int64_t)e * w.max_cand + c] = s_base;
            w.mem_count[(int64_t)e * w.max_cand + c] = s_written;
        }
        __syncthreads();
        const int n = s_total;
        members_total += (unsigned)n;
        unsigned long long votes = 0;
        for (int lo = 0; lo < n; lo += kMemberChunk) {
            const int hi = min(n, lo + kMemberChunk);
            // the chunk's members, in the fixed order, into shared memory (and the pool)
            for (int l = warp; l < HOUGH_MAX_LAYERS; l += kConfirmWarps) {
                if (s_lcount[l] == 0) continue;
                if (s_loff[l] >= hi || s_loff[l] + s_lcount[l] <= lo) continue;
                const LayerScan sc = layer_scan(ax, w, offs, l, i, j, s32);
                warp_layer_members(ax, w, hot, cold, sc, i, j, s32, refine_eps, s_loff[l], lo, hi, s_pos,
                                   pool + s_base, s_written);
            }
            __syncthreads();
            const int nm = hi - lo;
            const double k = qpt_centre(ax, i);
            // per member: arc length (FP64) and the linear z0 coordinate around its crossing row
            for (int q = threadIdx.x; q < nm; q += kConfirmThreads) {
                const int pos = s_pos[q];
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
                if (B > 0.0) mref = (int)fminf(fmaxf(rintf((float)A / (float)B), 0.f), (float)(ax.n_cot - 1));
                m_s[q] = s;
                m_z[q] = ch.z;
                m_a[q] = (float)(A - (double)mref * B);
                m_b[q] = (float)B;
                m_ref[q] = mref;
                m_l[q] = l;
            }
            __syncthreads();
            for (int pq = threadIdx.x; pq < nm * ax.n_cot; pq += kConfirmThreads) {
                const int q = pq / ax.n_cot, m = pq - q * ax.n_cot;
                const float wv = fmaf(-(float)(m - m_ref[q]), m_b[q], m_a[q]);
                const float fl = floorf(wv);
                const float d = wv - fl;
                int nz;
                if (d < kStage2Eps || d > 1.f - kStage2Eps) {
                    nz = (int)floor(exact_z0_coord(ax, (double)m_z[q], m_s[q], m));
                } else {
                    nz = (int)fl;
                    if (wv < -1.f || wv > (float)ax.n_z0 + 1.f) nz = -1;
                }
                if (nz >= 0 && nz < ax.n_z0) {
                    const int cell = m * ax.n_z0 + nz;
                    atomicOr(&grid2[cell >> 1], (1u << m_l[q]) << ((cell & 1) << 4));
                    ++votes;
                }
            }
            __syncthreads();
        }
        // the cell of most layers, lowest row-major index on ties: key = count << 32 | (ncell - cell)
        unsigned long long best = 0ull;
        for (int cell = threadIdx.x; cell < ncell; cell += kConfirmThreads) {
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
            for (int q = 1; q < kConfirmWarps; ++q) b = s_best[q] > b ? s_best[q] : b;
            const int cell = ncell - (int)(b & 0xFFFFFFFFu);
            const uint32_t m16 = (grid2[cell >> 1] >> ((cell & 1) << 4)) & 0xFFFFu;
            hough_candidate out = cd;
            out.n_members = (uint32_t)n;
            out.icot = (uint32_t)(cell / ax.n_z0);
            out.jz0 = (uint32_t)(cell % ax.n_z0);
            out.mask2 = m16;
            out.flags = (__popc(m16) >= ax.threshold ? 1u : 0u) | (s_written < n ? 2u : 0u);
            cands[c] = out;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (s_votes) atomicAdd(&w.stats[e].stage2_votes, s_votes);
        if (members_total) atomicAdd(&w.stats[e].n_members, members_total);
    }
}

__global__ void member_index_kernel(Workspace w, int32_t *idx_out, int64_t total)
{
    const ColdHit *cold = w.cold + w.hit_start[0];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
        idx_out[q] = cold[w.mem_pool[q]].idx;
}

}  // namespace

size_t stage2_smem_bytes(const Axes &ax)
{
    const int ncell = ax.n_cot * ax.n_z0;
    const int nwords = (((ncell + 1) >> 1) + 1) & ~1;
    return (size_t)nwords * 4 + (size_t)kMemberChunk * (8 + 4 * 6);
}

cudaError_t launch_stage2(const Axes &ax, const Workspace &w, int sms, float refine_eps, cudaStream_t stream)
{
    const float s32 = (float)(ax.n_phi * kInvTwoPi);
    const size_t smem = stage2_smem_bytes(ax);
    cudaError_t err = cudaFuncSetAttribute(confirm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err) return err;
    // candidates per event are known on the device only: size the grid for the device and let
    // each CTA stride over its event's candidates
    int y = (4 * sms + w.n_events - 1) / w.n_events;
    y = max(1, min(y, w.max_cand));
    confirm_kernel<<<dim3(y, w.n_events), kConfirmThreads, smem, stream>>>(ax, w, s32, refine_eps);
    return cudaGetLastError();
}

cudaError_t launch_member_index(const Workspace &w, int32_t *idx_out, int64_t total, cudaStream_t stream)
{
    if (total <= 0) return cudaSuccess;
    const int g = (int)min((total + 255) / 256, (int64_t)4096);
    member_index_kernel<<<g, 256, 0, stream>>>(w, idx_out, total);
    return cudaGetLastError();
}

}  // namespace hough
