/*
 * FP64 CPU oracle of the Hough-transform track finder.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path; the two meet only in
 * the seeded synthetic events that both take as plain inputs.
 *
 * What it computes, in the order the method runs (Sec. 4 of Halyo et al.,
 * "First Evaluation of the CPU, GPGPU and MIC Architectures for Real Time
 * Particle Tracking based on Hough Transform at the LHC"):
 *
 *   1. vote   - every hit marks every cell of a discrete (curvature, azimuth)
 *               parameter grid that is consistent with it (Sec. 4; the
 *               A[B[i]] += 1 scatter of Sec. 8).  Curvature is q/pT, azimuth is
 *               the track direction at the beam line phi0.  A cell records
 *               either which detector layers voted for it, as a bit mask (the
 *               layer accumulator), or how many votes it received, A[B[i]] += 1
 *               literally, saturating at 65535 (the count accumulator);
 *   2. peaks  - cells with many votes that are local maxima of the grid are
 *               track candidates (Sec. 4, second step; Sec. 8).  "Many votes"
 *               is the number of layers of a mask, or the count itself;
 *   3. confirm - "more expensive computations" on each candidate (Sec. 4): the
 *               candidate's member hits vote in a second (cot theta, z0) grid.
 *
 * The paper gives these steps in prose only.  The formulas are the standard
 * helix relations for a track from the beam line in a solenoid field B [T]:
 *
 *   x     = 0.15 * B * (r / 100) * k          k = q/pT [c/GeV], r [cm]
 *   phi0  = phi - asin(x)                     valid when |x| <= 1
 *   u     = n_phi * (phi0 + pi) / (2 pi)      phi0 bin coordinate
 *   j     = floor(u) mod n_phi                (Euclidean, the axis is cyclic)
 *   s     = r * asin(|x|) / |x|               transverse arc length (s = r at x = 0)
 *   z0    = z - s * cot(theta)
 *
 * Non-prompt tracks (the paper's aim of reconstructing prompt and non-prompt
 * tracks, Sec. 2 and Sec. 4) add a third axis, the signed transverse impact
 * parameter d0: the track's closest approach to the beam line is the point
 * d0 * (-sin phi0, cos phi0), where it runs along phi0.  Its circle, of
 * curvature rho = 2 x / r (1/cm), has its centre at (d0 + 1/rho)(-sin phi0,
 * cos phi0), and a hit at (r, phi) on it satisfies
 *
 *   sin(phi - phi0) = (rho r^2 + 2 d0 + rho d0^2) / (2 r (1 + rho d0))   (= x at d0 = 0)
 *   chord           = sqrt(r^2 + d0^2 - 2 r d0 sin(phi - phi0))          closest approach to hit
 *   s               = 2 asin(|rho| chord / 2) / |rho|                    (= chord at rho = 0)
 *
 * (1 + rho d0 > 0 for the point to be the closest one; the hit is the first
 * crossing of radius r, the principal arcsine.)  With d0 bins the grid has
 * n_d0 slices of n_qpt x n_phi cells, stored one after the other ("stacked
 * rows": row m * n_qpt + i holds d0 bin m, q/pT bin i); without them
 * (n_d0 = 0) d0 is 0 and the grid is one slice.
 *
 * Each value is evaluated in IEEE double in exactly the order written here,
 * inputs promoted exactly from FP32.  A vote whose bin coordinate lies within
 * 1e-4 bin widths of a bin edge (or whose |x| lies within 1e-6 of 1) is
 * "flagged": FP32 arithmetic may legitimately put it in the neighbouring bin.
 * Build with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846
#define ORACLE_EDGE_WINDOW 1e-4
#define ORACLE_DOMAIN_WINDOW 1e-6

#define ORACLE_ACC_LAYERS 0   /* a cell holds the bit mask of the layers that voted */
#define ORACLE_ACC_COUNTS 1   /* a cell holds its number of votes, saturating at 65535 */

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ETRUNC (-2)

typedef struct {
    int32_t n_layers;
    int32_t n_qpt;
    int32_t n_phi;
    int32_t threshold;
    int32_t n_cot;
    int32_t n_z0;
    int32_t accumulator;   /* ORACLE_ACC_LAYERS or ORACLE_ACC_COUNTS */
    int32_t n_d0;          /* d0 bins over [d0_min, d0_max] cm; 0: prompt tracks, d0 = 0 */
    double b_tesla;
    double qpt_min, qpt_max;
    double cot_min, cot_max;
    double z0_min, z0_max;
    double d0_min, d0_max;
} oracle_binning;

/* A vote whose outcome is within the flag window of a decision edge. */
typedef struct {
    int64_t hit;     /* hit index in the event */
    int32_t row;     /* stacked row m * n_qpt + iq (stage 1) or icot (stage 2) */
    int32_t bin;     /* the oracle's bin on that row, -1 when the oracle cast no vote */
    int32_t alt;     /* the bin on the other side of the edge, -1 when that side casts no vote */
    int32_t layer;
    int32_t kind;    /* 1: bin edge, 2: |x| = 1 domain edge */
    int32_t cand;    /* candidate index (membership and stage 2), else -1 */
} oracle_flag;

typedef struct {
    int32_t iq, jphi;
    uint32_t mask;
    int32_t id0;     /* d0 bin (0 without a d0 axis) */
} oracle_candidate;

typedef struct {
    int32_t icot, jz0;
    uint32_t mask2;
    int32_t n_votes;   /* stage-2 votes cast (member, cot bin) pairs inside the z0 range */
} oracle_stage2_result;

static int popcount16(uint32_t m)
{
    int c = 0;
    while (m) { c += (int)(m & 1u); m >>= 1; }
    return c;
}

/* The vote weight of a cell: its number of layers, or its count. */
static int cell_value(const oracle_binning *b, uint16_t m)
{
    return b->accumulator == ORACLE_ACC_COUNTS ? (int)m : popcount16(m);
}

static int64_t floor_mod(int64_t a, int64_t n)
{
    int64_t m = a % n;
    return m < 0 ? m + n : m;
}

/* q/pT bin centre of row i. */
static double qpt_centre(const oracle_binning *b, int i)
{
    double dk = (b->qpt_max - b->qpt_min) / b->n_qpt;
    return b->qpt_min + (i + 0.5) * dk;
}

/* Sagitta argument x = r / 2R of a hit at radius r (cm) for curvature k (c/GeV). */
static double sagitta_arg(const oracle_binning *b, double r_cm, double k)
{
    return 0.15 * b->b_tesla * (r_cm / 100.0) * k;
}

/* Number of d0 slices of the grid, and the d0 bin centre of slice m (cm). */
static int n_slices(const oracle_binning *b)
{
    return b->n_d0 > 0 ? b->n_d0 : 1;
}

static double d0_centre(const oracle_binning *b, int m)
{
    if (b->n_d0 <= 0) return 0.0;
    double dd = (b->d0_max - b->d0_min) / b->n_d0;
    return b->d0_min + (m + 0.5) * dd;
}

/*
 * sin(phi - phi0) of a hit at radius r on the track of sagitta argument x and
 * impact parameter d0.  Returns 0 when 1 + rho d0 <= 0 (no such track).
 */
static int track_sin(double r, double x, double d0, double *y)
{
    if (d0 == 0.0) {
        *y = x;
        return 1;
    }
    double rho = 2.0 * x / r;
    double den = 2.0 * r * (1.0 + rho * d0);
    if (!(den > 0.0)) return 0;
    *y = (rho * r * r + 2.0 * d0 + rho * d0 * d0) / den;
    return 1;
}

/* Transverse arc length from the closest approach to the hit (r, with sin(phi - phi0) = y). */
static double track_arc(double r, double x, double d0, double y)
{
    double ax = fabs(x);
    if (d0 == 0.0) return ax > 0.0 ? r * asin(ax) / ax : r;
    double chord = sqrt(r * r + d0 * d0 - 2.0 * r * d0 * y);
    double arho = 2.0 * ax / r;
    return arho > 0.0 ? 2.0 * asin(arho * chord / 2.0) / arho : chord;
}

/* phi0 bin coordinate of the vote of a hit at azimuth phi with sin(phi - phi0) = y. */
static double phi0_coord(const oracle_binning *b, double phi, double y)
{
    double phi0 = phi - asin(y);
    return b->n_phi * (phi0 + ORACLE_PI) / (2.0 * ORACLE_PI);
}

static void push_flag(oracle_flag *flags, int64_t cap, int64_t *n, int64_t hit, int32_t row,
                      int32_t bin, int32_t alt, int32_t layer, int32_t kind, int32_t cand)
{
    if (*n < cap && flags) {
        oracle_flag *f = &flags[*n];
        f->hit = hit; f->row = row; f->bin = bin; f->alt = alt;
        f->layer = layer; f->kind = kind; f->cand = cand;
    }
    (*n)++;
}

/*
 * The vote of one hit on q/pT row i of d0 slice m.  Returns 1 and sets *j when a
 * vote is cast.  Sets *flag_kind (0, 1 or 2) and *alt, the bin on the other side
 * of the edge.
 */
static int vote_one(const oracle_binning *b, double r, double phi, int m, int i,
                    int32_t *j, int32_t *alt, int32_t *flag_kind)
{
    double x = sagitta_arg(b, r, qpt_centre(b, i));
    double y = 2.0;
    int exists = track_sin(r, x, d0_centre(b, m), &y);
    int domain = exists && fabs(fabs(y) - 1.0) < ORACLE_DOMAIN_WINDOW;
    *flag_kind = 0;
    *alt = -1;
    *j = -1;
    if (!exists || !(fabs(y) <= 1.0)) {
        if (domain) *flag_kind = 2;   /* FP32 may cast this vote */
        return 0;
    }
    double u = phi0_coord(b, phi, y);
    *j = (int32_t)floor_mod((int64_t)floor(u), b->n_phi);
    double e = nearbyint(u);
    if (fabs(u - e) < ORACLE_EDGE_WINDOW) {
        /* u >= e: the vote sits just above edge e, the other side is bin e - 1 */
        *alt = (int32_t)floor_mod(u >= e ? (int64_t)e - 1 : (int64_t)e, b->n_phi);
        *flag_kind = 1;
    }
    if (domain) *flag_kind = 2;       /* FP32 may not cast this vote */
    return 1;
}

static int check_hits(const oracle_binning *b, const uint8_t *layer, int64_t n)
{
    if (b->n_layers < 1 || b->n_layers > 16 || b->n_qpt < 1 || b->n_phi < 3)
        return ORACLE_EINVAL;
    if (b->accumulator != ORACLE_ACC_LAYERS && b->accumulator != ORACLE_ACC_COUNTS)
        return ORACLE_EINVAL;
    if (b->n_d0 < 0 || (b->n_d0 > 0 && !(b->d0_min < b->d0_max)))
        return ORACLE_EINVAL;
    for (int64_t h = 0; h < n; ++h)
        if (layer[h] >= b->n_layers) return ORACLE_EINVAL;
    return ORACLE_OK;
}

/*
 * Stage-1 vote (Sec. 4, first step).  M is n_slices x n_qpt x n_phi, row-major
 * (stacked rows), and is overwritten.  votes_by_layer[l] counts the votes cast by hits of layer l.
 * A vote ORs the hit's layer bit into its cell, or adds one to the cell's count
 * (held at 65535 once it gets there).
 */
int oracle_vote(const oracle_binning *b, const float *r, const float *phi, const uint8_t *layer,
                int64_t n, uint16_t *M, uint64_t *votes_by_layer,
                oracle_flag *flags, int64_t flag_cap, int64_t *n_flags)
{
    if (check_hits(b, layer, n) != ORACLE_OK) return ORACLE_EINVAL;
    const int64_t rows = (int64_t)n_slices(b) * b->n_qpt;
    memset(M, 0, sizeof(uint16_t) * (size_t)rows * (size_t)b->n_phi);
    for (int l = 0; l < 16; ++l) votes_by_layer[l] = 0;
    *n_flags = 0;
    for (int64_t h = 0; h < n; ++h) {
        int l = layer[h];
        for (int64_t row = 0; row < rows; ++row) {
            int m = (int)(row / b->n_qpt), i = (int)(row % b->n_qpt);
            int32_t j, alt, kind;
            int cast = vote_one(b, (double)r[h], (double)phi[h], m, i, &j, &alt, &kind);
            if (cast) {
                uint16_t *cell = &M[(size_t)row * b->n_phi + j];
                if (b->accumulator == ORACLE_ACC_COUNTS) {
                    if (*cell < 65535u) *cell = (uint16_t)(*cell + 1u);
                } else {
                    *cell |= (uint16_t)(1u << l);
                }
                votes_by_layer[l]++;
            }
            if (kind)
                push_flag(flags, flag_cap, n_flags, h, (int32_t)row, j, alt, l, kind, -1);
        }
    }
    return ORACLE_OK;
}

/*
 * Peak search (Sec. 4, second step): a cell is a candidate when its value p
 * (layer accumulator: the number of layers in its mask; count accumulator: its
 * count) reaches the threshold, no neighbour of its 3 x 3 block -- 3 x 3 x 3
 * with a d0 axis -- exceeds it, and the neighbours that precede it in raster
 * order (d0 bin, then q/pT row, then phi0 column) are strictly lower: in one
 * slice the offsets (-1,-1), (-1,0), (-1,+1), (0,-1), and with a d0 axis also
 * the whole block of the slice before.  phi0 wraps; rows and slices outside the
 * grid count as empty.  Candidates are listed in raster order.
 */
int oracle_peaks(const oracle_binning *b, const uint16_t *M, oracle_candidate *out,
                 int64_t cap, int64_t *n_out)
{
    int64_t n = 0;
    const int D = n_slices(b);
    const size_t slice = (size_t)b->n_qpt * (size_t)b->n_phi;
    for (int m = 0; m < D; ++m) {
        for (int i = 0; i < b->n_qpt; ++i) {
            for (int j = 0; j < b->n_phi; ++j) {
                int p = cell_value(b, M[m * slice + (size_t)i * b->n_phi + j]);
                if (p < b->threshold) continue;
                int is_peak = 1;
                for (int dm = -1; dm <= 1 && is_peak; ++dm) {
                    for (int di = -1; di <= 1 && is_peak; ++di) {
                        for (int dj = -1; dj <= 1; ++dj) {
                            if (dm == 0 && di == 0 && dj == 0) continue;
                            int mm = m + dm, ii = i + di;
                            int q = 0;
                            if (mm >= 0 && mm < D && ii >= 0 && ii < b->n_qpt) {
                                int jj = (int)floor_mod(j + dj, b->n_phi);
                                q = cell_value(b, M[mm * slice + (size_t)ii * b->n_phi + jj]);
                            }
                            int precedes = (dm < 0) || (dm == 0 && di < 0) || (dm == 0 && di == 0 && dj < 0);
                            if (precedes ? (q >= p) : (q > p)) { is_peak = 0; break; }
                        }
                    }
                }
                if (!is_peak) continue;
                if (n < cap) {
                    out[n].iq = i; out[n].jphi = j;
                    out[n].mask = M[m * slice + (size_t)i * b->n_phi + j]; out[n].id0 = m;
                }
                n++;
            }
        }
    }
    *n_out = n;
    return n > cap ? ORACLE_ETRUNC : ORACLE_OK;
}

static int64_t find_candidate(const oracle_candidate *c, int64_t lo, int64_t hi, int32_t j)
{
    /* candidates [lo, hi) share one row and are sorted by jphi */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (c[mid].jphi < j) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/*
 * Membership: hit h belongs to candidate (m, i, j) when its stage-1 vote on
 * q/pT row i of d0 slice m fell in bin j.  offsets has n_cand + 1 entries; members lists hit indices in
 * increasing order per candidate.  A flagged vote whose bin or alternative bin
 * is a candidate is reported with that candidate's index.
 */
int oracle_members(const oracle_binning *b, const float *r, const float *phi, const uint8_t *layer,
                   int64_t n, const oracle_candidate *c, int64_t n_cand,
                   int64_t *offsets, int64_t *members, int64_t member_cap,
                   oracle_flag *flags, int64_t flag_cap, int64_t *n_flags)
{
    if (check_hits(b, layer, n) != ORACLE_OK) return ORACLE_EINVAL;
    /* row_start[row] .. row_start[row+1]: the candidates on stacked row m * n_qpt + i */
    const int64_t rows = (int64_t)n_slices(b) * b->n_qpt;
    int64_t *row_start = (int64_t *)calloc((size_t)rows + 1, sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)n_cand + 1, sizeof(int64_t));
    if (!row_start || !fill) { free(row_start); free(fill); return ORACLE_EINVAL; }
    for (int64_t q = 0; q < n_cand; ++q) row_start[(int64_t)c[q].id0 * b->n_qpt + c[q].iq + 1]++;
    for (int64_t row = 0; row < rows; ++row) row_start[row + 1] += row_start[row];
    *n_flags = 0;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            offsets[0] = 0;
            for (int64_t q = 0; q < n_cand; ++q) offsets[q + 1] = offsets[q] + fill[q];
            memset(fill, 0, sizeof(int64_t) * (size_t)(n_cand + 1));
        }
        for (int64_t h = 0; h < n; ++h) {
            for (int64_t i = 0; i < rows; ++i) {   /* i: stacked row */
                if (row_start[i] == row_start[i + 1]) continue;
                int32_t j, alt, kind;
                int cast = vote_one(b, (double)r[h], (double)phi[h], (int)(i / b->n_qpt), (int)(i % b->n_qpt),
                                    &j, &alt, &kind);
                if (cast) {
                    int64_t q = find_candidate(c, row_start[i], row_start[i + 1], j);
                    if (q < row_start[i + 1] && c[q].jphi == j) {
                        if (pass == 1) {
                            int64_t at = offsets[q] + fill[q];
                            if (at < member_cap) members[at] = h;
                        }
                        fill[q]++;
                    }
                }
                if (pass == 1 && kind) {
                    int32_t probe[2] = { j, alt };
                    for (int e = 0; e < 2; ++e) {
                        if (probe[e] < 0) continue;
                        int64_t q = find_candidate(c, row_start[i], row_start[i + 1], probe[e]);
                        if (q < row_start[i + 1] && c[q].jphi == probe[e])
                            push_flag(flags, flag_cap, n_flags, h, (int32_t)i, j, alt, layer[h], kind, (int32_t)q);
                    }
                    if (kind == 2 && j < 0)   /* a vote the oracle did not cast: any candidate on the row */
                        for (int64_t q = row_start[i]; q < row_start[i + 1]; ++q)
                            push_flag(flags, flag_cap, n_flags, h, (int32_t)i, j, alt, layer[h], kind, (int32_t)q);
                }
            }
        }
    }
    free(row_start);
    free(fill);
    return offsets[n_cand] > member_cap ? ORACLE_ETRUNC : ORACLE_OK;
}

/*
 * Second-stage vote (the confirmation step): every member hit of a candidate
 * votes in an n_cot x n_z0 grid of (cot theta, z0) with z0 = z - s * cot theta,
 * s the transverse arc length at the candidate's curvature (and d0), from the
 * closest approach to the hit.  z0 is not cyclic:
 * votes outside [z0_min, z0_max) are not cast.  The result is the cell of most
 * layers, the lowest row-major index on ties.  With either stage-1 accumulator
 * the second grid holds layer masks.
 */
int oracle_stage2(const oracle_binning *b, const float *r, const float *z, const uint8_t *layer,
                  int64_t n, const oracle_candidate *c, int64_t n_cand,
                  const int64_t *offsets, const int64_t *members, oracle_stage2_result *out,
                  oracle_flag *flags, int64_t flag_cap, int64_t *n_flags)
{
    if (check_hits(b, layer, n) != ORACLE_OK) return ORACLE_EINVAL;
    size_t cells = (size_t)b->n_cot * (size_t)b->n_z0;
    uint16_t *M2 = (uint16_t *)malloc(sizeof(uint16_t) * cells);
    if (!M2) return ORACLE_EINVAL;
    *n_flags = 0;
    double dt = (b->cot_max - b->cot_min) / b->n_cot;
    for (int64_t q = 0; q < n_cand; ++q) {
        memset(M2, 0, sizeof(uint16_t) * cells);
        double k = qpt_centre(b, c[q].iq);
        double d0 = d0_centre(b, c[q].id0);
        int32_t votes = 0;
        for (int64_t e = offsets[q]; e < offsets[q + 1]; ++e) {
            int64_t h = members[e];
            double rr = (double)r[h];
            double x = sagitta_arg(b, rr, k);
            double y = x;
            track_sin(rr, x, d0, &y);   /* a member's track exists: its vote was cast */
            double s = track_arc(rr, x, d0, y);
            for (int m = 0; m < b->n_cot; ++m) {
                double t = b->cot_min + (m + 0.5) * dt;
                double z0 = (double)z[h] - s * t;
                double w = b->n_z0 * (z0 - b->z0_min) / (b->z0_max - b->z0_min);
                double e_w = nearbyint(w);
                int inside = (w >= 0.0 && w < (double)b->n_z0);
                int32_t bin = inside ? (int32_t)floor(w) : -1;
                if (fabs(w - e_w) < ORACLE_EDGE_WINDOW) {
                    int64_t a = w >= e_w ? (int64_t)e_w - 1 : (int64_t)e_w;
                    int32_t alt = (a >= 0 && a < b->n_z0) ? (int32_t)a : -1;
                    push_flag(flags, flag_cap, n_flags, h, m, bin, alt, layer[h], 1, (int32_t)q);
                }
                if (!inside) continue;
                M2[(size_t)m * b->n_z0 + bin] |= (uint16_t)(1u << layer[h]);
                votes++;
            }
        }
        int best = -1;
        size_t best_at = 0;
        for (size_t a = 0; a < cells; ++a) {
            int p = popcount16(M2[a]);
            if (p > best) { best = p; best_at = a; }
        }
        out[q].icot = (int32_t)(best_at / (size_t)b->n_z0);
        out[q].jz0 = (int32_t)(best_at % (size_t)b->n_z0);
        out[q].mask2 = M2[best_at];
        out[q].n_votes = votes;
    }
    free(M2);
    return ORACLE_OK;
}
