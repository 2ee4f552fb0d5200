/*
 * FP32 multi-core CPU implementation of the Hough-transform track finder: a context figure timed
 * beside the GPU numbers, written the way the paper describes its own CPU code (Sec. 6.2): OpenMP
 * threads over the outer loop of the transform (the hits) with thread-private accumulators merged
 * at the end, threads over the rows of the local-maximum search and over the candidates of the
 * confirmation, and inner loops kept free of dependences so the compiler can vectorise them.
 *
 * It is neither the FP64 oracle that the tests compare the CUDA path against nor part of that
 * path; the benchmark times it on the host cores.
 *
 * The method, per event, in FP32 (prompt tracks, layer-mask accumulator):
 *   vote     x = 0.15 B (r / 100) k_i on q/pT row i (k_i the row's centre), phi0 = phi - asin(x),
 *            j = floor(n_phi (phi0 + pi) / (2 pi)) mod n_phi; the hit's layer bit is ORed into
 *            cell (i, j) of every row with |x| <= 1 (Sec. 4);
 *   peaks    a cell with p >= threshold layers is a candidate when no cell of its 3 x 3 block
 *            (phi0 cyclic) has more, and those before it in raster order have fewer (Sec. 4);
 *   confirm  its members are the hits whose vote on its row fell in its column; each votes, for
 *            every cot(theta) row m, in the z0 column of z0 = z - s t_m, s = r asin|x| / |x| the
 *            transverse arc length; the result is the cell of most layers, the first in row-major
 *            order on ties (Sec. 4, the "more expensive computations" on each candidate).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CPU_PI 3.14159265358979323846f

typedef struct {
    int32_t n_layers, n_qpt, n_phi, threshold, n_cot, n_z0;
    float b_tesla, qpt_min, qpt_max, cot_min, cot_max, z0_min, z0_max;
} hough_cpu_binning;

/* Per candidate, eight int32: iq, jphi, layer mask, members, icot, jz0, stage-2 mask, confirmed. */
enum { CPU_OUT_FIELDS = 8 };

static int layer_count(uint16_t m) { return __builtin_popcount((unsigned)m); }

static int wrap(int j, int n) { j %= n; return j < 0 ? j + n : j; }

/* The phi0 column of a hit's vote for sagitta argument x (|x| <= 1). */
static int vote_col(const hough_cpu_binning *b, float phi, float x)
{
    const float u = (float)b->n_phi * (phi - asinf(x) + CPU_PI) / (2.f * CPU_PI);
    return wrap((int)floorf(u), b->n_phi);
}

/* Whether cell (i, j) with p layers is a local maximum: the neighbours before it in raster order
   (the row above, the cell to the left) have fewer layers, the others no more; phi0 wraps and rows
   outside the grid are empty. */
static int is_peak(const uint16_t *M, int R, int P, int i, int j, int p)
{
    const int jm = wrap(j - 1, P), jp = wrap(j + 1, P);
    const uint16_t *row = M + (size_t)i * P;
    if (i > 0) {
        const uint16_t *up = row - P;
        if (layer_count(up[jm]) >= p || layer_count(up[j]) >= p || layer_count(up[jp]) >= p) return 0;
    }
    if (layer_count(row[jm]) >= p || layer_count(row[jp]) > p) return 0;
    if (i + 1 < R) {
        const uint16_t *dn = row + P;
        if (layer_count(dn[jm]) > p || layer_count(dn[j]) > p || layer_count(dn[jp]) > p) return 0;
    }
    return 1;
}

/* Hits of one layer sorted by their own azimuth coordinate, for the membership search. */
typedef struct {
    int64_t *idx;     /* hit indices, by increasing u */
    float *u;         /* n_phi (phi + pi) / (2 pi) of each, in the same order */
    int64_t n;
    float c_min, c_max;   /* 0.15 B r / 100 over the layer's hits */
} layer_hits;

typedef struct { float u; int64_t h; } ukey;

static int key_cmp(const void *a, const void *b)
{
    const float x = ((const ukey *)a)->u, y = ((const ukey *)b)->u;
    if (x < y) return -1;
    if (x > y) return 1;
    const int64_t p = ((const ukey *)a)->h, q = ((const ukey *)b)->h;
    return p < q ? -1 : p > q;
}

/* First index of sorted u[0..n) with u >= v. */
static int64_t lower(const float *u, int64_t n, float v)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (u[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/*
 * One event.  Writes up to `cap` candidates (CPU_OUT_FIELDS int32 each, raster order) to out and,
 * when M_out is not NULL, the n_qpt x n_phi accumulator.  threads <= 0: OpenMP's default.
 * Returns the number of candidates found (which may exceed cap), or -1 on invalid input.
 */
int64_t hough_cpu_event(const hough_cpu_binning *b, const float *r, const float *phi, const float *z,
                        const uint8_t *layer, int64_t n, int threads, int32_t *out, int64_t cap, uint16_t *M_out)
{
    if (b->n_layers < 1 || b->n_layers > 16 || b->n_qpt < 1 || b->n_phi < 3 || b->n_cot < 1 || b->n_z0 < 1)
        return -1;
    for (int64_t h = 0; h < n; ++h)
        if (layer[h] >= b->n_layers) return -1;
    const int R = b->n_qpt, P = b->n_phi, L = b->n_layers;
    const size_t cells = (size_t)R * (size_t)P;
    const int T = threads > 0 ? threads : omp_get_max_threads();
    const float dk = (b->qpt_max - b->qpt_min) / (float)R;
    float *kq = (float *)malloc(sizeof(float) * (size_t)R);
    uint16_t *M = (uint16_t *)malloc(sizeof(uint16_t) * cells);
    uint16_t **priv = (uint16_t **)calloc((size_t)T, sizeof(uint16_t *));
    if (!kq || !M || !priv) { free(kq); free(M); free(priv); return -1; }
    for (int i = 0; i < R; ++i) kq[i] = b->qpt_min + ((float)i + 0.5f) * dk;
    const float cscale = 0.15f * b->b_tesla / 100.f;

    /* 1. vote: the hits split over the threads, each ORing into its own accumulator */
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num();
        uint16_t *Mt = (uint16_t *)calloc(cells, sizeof(uint16_t));
        int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
        priv[t] = Mt;
        if (Mt && col) {
#pragma omp for schedule(static)
            for (int64_t h = 0; h < n; ++h) {
                const float c = cscale * r[h], ph = phi[h];
                for (int i = 0; i < R; ++i) {   /* independent rows: vectorisable */
                    const float x = c * kq[i];
                    const float xc = fminf(fmaxf(x, -1.f), 1.f);
                    const float u = (float)P * (ph - asinf(xc) + CPU_PI) / (2.f * CPU_PI);
                    int j = (int)floorf(u) % P;
                    j += j < 0 ? P : 0;
                    col[i] = fabsf(x) <= 1.f ? j : -1;
                }
                const uint16_t bit = (uint16_t)(1u << layer[h]);
                for (int i = 0; i < R; ++i)
                    if (col[i] >= 0) Mt[(size_t)i * P + col[i]] |= bit;
            }
        }
        free(col);
#pragma omp barrier
        /* merge: the cells split over the threads, each ORing every private copy */
#pragma omp for schedule(static)
        for (int64_t q = 0; q < (int64_t)cells; ++q) {
            uint16_t v = 0;
            for (int u = 0; u < T; ++u) v |= priv[u] ? priv[u][q] : 0;
            M[q] = v;
        }
#pragma omp barrier
        free(Mt);
    }
    free(priv);
    if (M_out) memcpy(M_out, M, sizeof(uint16_t) * cells);

    /* 2. peaks: rows over the threads; per-row counts, then each row's candidates at its offset */
    int64_t *row_at = (int64_t *)calloc((size_t)R + 1, sizeof(int64_t));
    if (!row_at) { free(kq); free(M); return -1; }
    const int thr = b->threshold;
#pragma omp parallel for num_threads(T) schedule(static)
    for (int i = 0; i < R; ++i) {
        int64_t cnt = 0;
        for (int j = 0; j < P; ++j) {
            const int p = layer_count(M[(size_t)i * P + j]);
            if (p < thr) continue;
            cnt += is_peak(M, R, P, i, j, p);
        }
        row_at[i + 1] = cnt;
    }
    for (int i = 0; i < R; ++i) row_at[i + 1] += row_at[i];
    const int64_t n_cand = row_at[R];
    const int64_t kept = n_cand < cap ? n_cand : cap;
#pragma omp parallel for num_threads(T) schedule(static)
    for (int i = 0; i < R; ++i) {
        int64_t at = row_at[i];
        for (int j = 0; j < P && at < kept; ++j) {
            const int p = layer_count(M[(size_t)i * P + j]);
            if (p < thr) continue;
            if (!is_peak(M, R, P, i, j, p)) continue;
            int32_t *o = out + at * CPU_OUT_FIELDS;
            o[0] = i; o[1] = j; o[2] = M[(size_t)i * P + j];
            for (int f = 3; f < CPU_OUT_FIELDS; ++f) o[f] = 0;
            ++at;
        }
    }
    free(row_at);

    /* hits of each layer by azimuth, for the membership search */
    layer_hits lh[16];
    memset(lh, 0, sizeof(lh));
    int ok = 1;
    for (int l = 0; l < L && ok; ++l) {
        int64_t m = 0;
        for (int64_t h = 0; h < n; ++h) m += layer[h] == l;
        ukey *keys = (ukey *)malloc(sizeof(ukey) * (size_t)(m ? m : 1));
        lh[l].idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m ? m : 1));
        lh[l].u = (float *)malloc(sizeof(float) * (size_t)(m ? m : 1));
        if (!keys || !lh[l].idx || !lh[l].u) { free(keys); ok = 0; break; }
        float cmin = INFINITY, cmax = 0.f;
        int64_t k = 0;
        for (int64_t h = 0; h < n; ++h) {
            if (layer[h] != l) continue;
            keys[k].u = (float)P * (phi[h] + CPU_PI) / (2.f * CPU_PI);
            keys[k].h = h;
            const float c = cscale * r[h];
            cmin = fminf(cmin, c);
            cmax = fmaxf(cmax, c);
            ++k;
        }
        qsort(keys, (size_t)m, sizeof(ukey), key_cmp);
        for (int64_t q = 0; q < m; ++q) { lh[l].idx[q] = keys[q].h; lh[l].u[q] = keys[q].u; }
        lh[l].n = m;
        lh[l].c_min = cmin;
        lh[l].c_max = cmax;
        free(keys);
    }

    /* 3. confirm: candidates over the threads, each with its own stage-2 grid */
    const float dt = (b->cot_max - b->cot_min) / (float)b->n_cot;
    const float zscale = (float)b->n_z0 / (b->z0_max - b->z0_min);
    const int need = thr < L ? thr : L;
    if (ok) {
#pragma omp parallel num_threads(T)
        {
            uint16_t *G = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)b->n_cot * (size_t)b->n_z0);
#pragma omp for schedule(dynamic, 16)
            for (int64_t q = 0; q < kept; ++q) {
                if (!G) continue;
                int32_t *o = out + q * CPU_OUT_FIELDS;
                const int i = o[0], j = o[1];
                const float k = kq[i];
                memset(G, 0, sizeof(uint16_t) * (size_t)b->n_cot * (size_t)b->n_z0);
                int members = 0;
                for (int l = 0; l < L; ++l) {
                    if (!lh[l].n) continue;
                    /* the hits whose vote can reach column j: u within j + n_phi asin(x) / (2 pi)
                       over the layer's radius range, a bin of margin on each side */
                    const float a1 = asinf(fminf(fmaxf(lh[l].c_min * k, -1.f), 1.f));
                    const float a2 = asinf(fminf(fmaxf(lh[l].c_max * k, -1.f), 1.f));
                    const float s = (float)P / (2.f * CPU_PI);
                    const float ulo = (float)j + s * fminf(a1, a2) - 1.f, uhi = (float)j + 1.f + s * fmaxf(a1, a2) + 1.f;
                    for (int rep = -1; rep <= 1; ++rep) {   /* the window and its images a turn away */
                        const float lo = ulo + (float)(rep * P), hi = uhi + (float)(rep * P);
                        if (hi < 0.f || lo >= (float)P) continue;
                        for (int64_t e = lower(lh[l].u, lh[l].n, lo); e < lh[l].n && lh[l].u[e] < hi; ++e) {
                            const int64_t h = lh[l].idx[e];
                            const float x = cscale * r[h] * k;
                            if (!(fabsf(x) <= 1.f) || vote_col(b, phi[h], x) != j) continue;
                            ++members;
                            /* its stage-2 votes, one per cot(theta) row */
                            const float ax = fabsf(x);
                            const float sarc = ax > 0.f ? r[h] * asinf(ax) / ax : r[h];
                            const uint16_t bit = (uint16_t)(1u << l);
                            for (int m = 0; m < b->n_cot; ++m) {
                                const float t = b->cot_min + ((float)m + 0.5f) * dt;
                                const float w = zscale * (z[h] - sarc * t - b->z0_min);
                                if (w >= 0.f && w < (float)b->n_z0) G[(size_t)m * b->n_z0 + (int)w] |= bit;
                            }
                        }
                    }
                }
                int best = -1, bc = 0;
                for (int c = 0; c < b->n_cot * b->n_z0; ++c) {
                    const int p = layer_count(G[c]);
                    if (p > bc) { bc = p; best = c; }
                }
                o[3] = members;
                o[4] = best >= 0 ? best / b->n_z0 : 0;
                o[5] = best >= 0 ? best % b->n_z0 : 0;
                o[6] = best >= 0 ? G[best] : 0;
                o[7] = bc >= need;
            }
            free(G);
        }
    }
    for (int l = 0; l < L; ++l) { free(lh[l].idx); free(lh[l].u); }
    free(kq);
    free(M);
    return ok ? n_cand : -1;
}
