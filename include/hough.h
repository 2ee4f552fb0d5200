/*
 * hough.h -- C ABI of the GB300 Hough-transform track finder.
 *
 * The method (Halyo et al., "First Evaluation of the CPU, GPGPU and MIC
 * Architectures for Real Time Particle Tracking based on Hough Transform at
 * the LHC", Sec. 4): every hit of an event votes into a discrete grid of track
 * parameters -- curvature q/pT by azimuth phi0 at the beam line -- and local
 * maxima of the grid are the track candidates; candidates are then confirmed by
 * a second, more expensive computation (Sec. 4), here a (cot theta, z0) vote of
 * each candidate's member hits.  Each grid cell holds a 16-bit mask of the
 * detector layers that voted for it.
 *
 * Formulas (the paper gives the steps in prose; these are the helix relations
 * of a track from the beam line in a solenoid field B):
 *   x    = 0.15 * B * (r / 100) * k_i             k_i = qpt_min + (i + 1/2) dk,  r in cm
 *   phi0 = phi - asin(x)                          a vote exists when |x| <= 1
 *   j    = floor(n_phi * (phi0 + pi) / (2 pi)) mod n_phi
 *   s    = r * asin(|x|) / |x|                    transverse arc length (s = r at x = 0)
 *   z0   = z - s * t_m                            t_m = cot_min + (m + 1/2) dt
 *
 * Conventions for every entry point:
 *   - Returns HOUGH_OK (0) or a negative HOUGH_E* status; hough_last_error()
 *     gives a message for the calling thread's last failure.
 *   - `where` says where caller buffers live: HOUGH_HOST (pageable or pinned
 *     host memory) or HOUGH_DEVICE (device memory of the context's GPU).
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Calls that only enqueue work return before it runs; calls that
 *     return results to host memory synchronise the stream first.
 *   - The library owns every context and its device buffers (allocated once by
 *     hough_create, sized by hough_limits).  Caller buffers stay owned by the
 *     caller and must stay valid until the call that reads them has finished
 *     on the stream.
 *   - A context is not thread-safe: one host thread drives it at a time.
 */
#ifndef HOUGH_H
#define HOUGH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HOUGH_OK          0
#define HOUGH_EINVAL     (-1)   /* an argument is out of its documented range */
#define HOUGH_ENOMEM     (-2)   /* a device or pinned-host allocation failed */
#define HOUGH_ECUDA      (-3)   /* the CUDA runtime reported an error */
#define HOUGH_ETRUNC     (-4)   /* more results than the caller's capacity; the first cap were written */
#define HOUGH_ECAPACITY  (-5)   /* the input exceeds the limits the context was created with */
#define HOUGH_EBUSY      (-6)   /* serving: no free slot for a new event */
#define HOUGH_ETIMEDOUT  (-7)   /* a bounded wait expired */
#define HOUGH_EDEVICE    (-8)   /* a device-side check failed (see hough_stats.device_error) */
#define HOUGH_ENOTREADY  (-9)   /* the requested result has not been produced yet */

#define HOUGH_HOST   0
#define HOUGH_DEVICE 1

#define HOUGH_MAX_LAYERS 16

/* Device-side error bits reported in hough_stats.device_error. */
#define HOUGH_DEVERR_LAYER     1u   /* a hit had layer >= n_layers; it cast no vote */
#define HOUGH_DEVERR_RADIUS    2u   /* a hit had r <= 0 or a non-finite coordinate; it cast no vote */
#define HOUGH_DEVERR_CAND      4u   /* more candidates than max_candidates; the first ones were kept */
#define HOUGH_DEVERR_MEMBERS   8u   /* more member hits than max_members; the member lists were cut (stage 2 still saw every member) */
#define HOUGH_DEVERR_TIMEOUT  16u   /* an on-chip bulk copy did not complete within its bound; the accumulator is incomplete */

/* Barrel detector: number of layers and the solenoid field. */
typedef struct hough_geometry {
    int32_t n_layers;   /* 1..16; a hit's layer index must be < n_layers */
    int32_t reserved;   /* must be 0 */
    double  b_tesla;    /* field in tesla, > 0 */
} hough_geometry;

/* What a stage-1 cell holds (hough_binning.accumulator). */
#define HOUGH_ACC_LAYERS 0   /* bit l set when a hit of layer l voted for the cell */
#define HOUGH_ACC_COUNTS 1   /* the number of votes the cell received (Sec. 8: A[B[i]] += 1), saturating at 65535 */

/*
 * Accumulator axes (Sec. 4: "a discrete grid in the parameter space").
 * Stage 1: n_qpt rows of q/pT over [qpt_min, qpt_max] (c/GeV) by n_phi columns
 * of phi0 over [-pi, pi), cyclic.  A cell's value is popcount(mask) with the
 * layer accumulator, its count with the count accumulator; a cell is a
 * candidate when its value >= threshold and it is a local maximum (see
 * hough_peaks).  Stage 2: n_cot rows of cot(theta) over [cot_min, cot_max] by
 * n_z0 columns of z0 over [z0_min_cm, z0_max_cm), not cyclic; its cells hold
 * layer masks with either accumulator.
 * Limits: 1 <= n_qpt <= 65535; 64 <= n_phi <= 32768 and n_phi % 64 == 0;
 * 1 <= threshold <= 16 (layer accumulator) or <= 65535 (count accumulator);
 * 1 <= n_cot, n_z0 <= 256 and n_cot * n_z0 <= 16384;
 * qpt_min < qpt_max, cot_min < cot_max, z0_min_cm < z0_max_cm.
 * With the count accumulator HOUGH_VOTE_GATHER counts per cell the hits of the
 * two buckets its votes come from, and HOUGH_VOTE_SCATTER is the shared-memory
 * atomic scatter; both give the same counts.
 *
 * Non-prompt tracks (n_d0 > 0): a third axis of n_d0 bins of the signed
 * transverse impact parameter d0 over [d0_min_cm, d0_max_cm).  A track whose
 * closest approach to the beam line is the point d0 (-sin phi0, cos phi0),
 * where it runs along phi0, with curvature rho = 0.003 B q/pT (1/cm), puts
 * its hit at radius r where sin(phi - phi0) = (rho r^2 + 2 d0 + rho d0^2) /
 * (2 r (1 + rho d0)) (the prompt relation phi0 = phi - asin(x) at d0 = 0);
 * a vote needs 1 + rho d0 > 0 and |sin(phi - phi0)| <= 1.  The arc length of
 * stage 2 runs from the closest approach.  The grid is then n_d0 slices of
 * n_qpt x n_phi cells stored one after the other: stacked row m * n_qpt + i
 * holds d0 bin m and q/pT bin i; accumulators, candidate rows (iq) and
 * hough_get_accumulator all use stacked rows.  A cell is a candidate when it
 * is a local maximum of its 3 x 3 x 3 block (the 13 neighbours before it in
 * raster order -- slice, row, column -- strictly lower); its peak search works
 * on bands of band_rows rows of one slice, which need 3 (band_rows + 2) n_phi
 * bytes of shared memory (twice that with counts); 9 n_phi (18 n_phi) bytes
 * must fit, else HOUGH_EINVAL.
 * n_d0 = 0: prompt tracks (d0 = 0), one slice, the d0 fields ignored.
 * Limits: 0 <= n_d0 and n_d0 * n_qpt <= 65535; d0_min_cm < d0_max_cm, finite.
 */
typedef struct hough_binning {
    int32_t n_qpt, n_phi, threshold, n_cot, n_z0;
    int32_t accumulator;   /* HOUGH_ACC_LAYERS or HOUGH_ACC_COUNTS */
    double  qpt_min, qpt_max;
    double  cot_min, cot_max;
    double  z0_min_cm, z0_max_cm;
    int32_t n_d0;          /* d0 bins; 0: prompt tracks only */
    int32_t reserved;      /* must be 0 */
    double  d0_min_cm, d0_max_cm;
} hough_binning;

/* Capacities fixed at creation; every device buffer is sized from them. */
typedef struct hough_limits {
    int64_t max_hits;         /* hits per event, >= 1 */
    int32_t max_candidates;   /* stage-1 candidates kept per event, >= 1 */
    int32_t max_members;      /* member hits kept per event over all candidates, >= 1 */
} hough_limits;

/*
 * One track candidate.  (iq, jphi) is the stage-1 cell (iq the stacked row
 * m * n_qpt + i with a d0 axis), mask its value as
 * stored (the layer mask, or with the count accumulator the count); n_members
 * the hits whose stage-1 vote fell in the cell (with the count accumulator
 * equal to the count below saturation); (icot, jz0) the stage-2 maximum (most
 * layers, lowest row-major index on ties) and mask2 its layer mask.  flags:
 * bit 0 set when popcount(mask2) >= min(threshold, n_layers) (confirmed), bit 1
 * when the member list was cut by max_members.  The stage-2 fields are 0 until
 * hough_stage2 has run.
 */
typedef struct hough_candidate {
    uint32_t iq, jphi, mask, n_members;
    uint32_t icot, jz0, mask2, flags;
} hough_candidate;

/* Counters of the last processed event (filled by hough_get_stats). */
typedef struct hough_stats {
    uint64_t votes;                              /* stage-1 votes cast */
    uint64_t votes_by_layer[HOUGH_MAX_LAYERS];
    uint64_t general_votes;                      /* votes on layers whose hits do not share one radius */
    uint64_t refined_votes;                      /* of those, votes recomputed in FP64 near a bin edge */
    uint64_t stage2_votes;                       /* stage-2 votes cast */
    int64_t  n_hits;                             /* hits accepted */
    int64_t  n_candidates;                       /* candidates found (may exceed max_candidates) */
    int64_t  n_members;                          /* member hits found (may exceed max_members) */
    uint32_t device_error;                       /* HOUGH_DEVERR_* bits */
    uint32_t uniform_layers;                     /* bit l: all hits of layer l share one radius */
} hough_stats;

typedef struct hough_ctx hough_ctx;

/* Message for the calling thread's last failing call ("" if none). */
const char *hough_last_error(void);

/* Library version, "major.minor.patch". */
const char *hough_version(void);

/*
 * Create a context on CUDA device `device`: validates the arguments (HOUGH_EINVAL),
 * allocates every device buffer (HOUGH_ENOMEM) and returns it in *out.
 */
int hough_create(const hough_geometry *geometry, const hough_binning *binning,
                 const hough_limits *limits, int device, hough_ctx **out);

/* Release a context and all its buffers.  NULL is accepted.  Synchronises the device first. */
void hough_destroy(hough_ctx *ctx);

/*
 * Stage-1 vote of one event (Sec. 4, first step).  Hits are four parallel
 * arrays of n_hits entries: r (cm, > 0), phi (rad, |phi| <= 1000; it is reduced
 * modulo 2 pi), z (cm, finite), layer (< n_layers).  With HOUGH_HOST the arrays
 * are checked on the host (HOUGH_EINVAL on a bad hit) and copied, except pinned
 * arrays (cudaHostAlloc, cudaHostRegister), which the staging kernels read in
 * place over the host link: their contents must stay unchanged until the vote
 * has run on `stream`.  With HOUGH_DEVICE a bad hit is dropped on the device
 * and reported through hough_stats.device_error.  n_hits may be 0.  Replaces
 * the context's previous event.  HOUGH_ECAPACITY when n_hits > max_hits.
 * Asynchronous on `stream`.
 */
int hough_vote(hough_ctx *ctx, const float *r, const float *phi, const float *z,
               const uint8_t *layer, int64_t n_hits, int where, void *stream);

/*
 * Peak search (Sec. 4, second step) on the accumulator of the last vote: cell
 * (i, j) with value p (popcount(mask), or the count with HOUGH_ACC_COUNTS) is a
 * candidate when p >= threshold, no 3 x 3 neighbour has a larger value and the
 * neighbours at offsets (-1,-1), (-1,0), (-1,+1), (0,-1) have strictly smaller
 * values (with a d0 axis: the 3 x 3 x 3 block, see hough_binning).  phi0 wraps; rows
 * outside the grid count as empty.  Candidates are kept in raster order.
 * Asynchronous on `stream`.
 */
int hough_peaks(hough_ctx *ctx, void *stream);

/*
 * Confirmation step (Sec. 4: "more expensive computations ... to confirm"):
 * finds each candidate's member hits (hits whose stage-1 vote on the
 * candidate's row fell in its cell) and votes them into the (cot theta, z0)
 * grid; fills n_members, icot, jz0, mask2 and flags.  Asynchronous on `stream`.
 */
int hough_stage2(hough_ctx *ctx, void *stream);

/*
 * Copy the candidates of the last event (raster order) to `out` (cap entries,
 * HOUGH_HOST or HOUGH_DEVICE); *n_out receives the number found.  HOUGH_ETRUNC
 * when that exceeds cap.  Synchronises `stream`.
 */
int hough_get_candidates(hough_ctx *ctx, hough_candidate *out, int32_t cap, int32_t *n_out,
                         int where, void *stream);

/* Copy the (stacked) rows x n_phi row-major accumulator of the last vote.  Synchronises `stream`.
 * HOUGH_ENOTREADY under vote_mode HOUGH_VOTE_FUSED, which does not keep it. */
int hough_get_accumulator(hough_ctx *ctx, uint16_t *out, int where, void *stream);

/*
 * Copy the member lists of the last stage 2: offsets[n_cand + 1] (int64) and
 * hits[offsets[n_cand]] (int32 hit indices of the event, increasing within each
 * candidate).  `hit_cap` bounds `hits`; HOUGH_ETRUNC when it is too small, or when
 * the event had more member hits than max_members (HOUGH_DEVERR_MEMBERS; a cut
 * list is a subset of the candidate's members, flagged in its record), the lists
 * being copied as far as they go.  Synchronises `stream`.
 */
int hough_get_members(hough_ctx *ctx, int64_t *offsets, int32_t *hits, int64_t hit_cap,
                      int where, void *stream);

/* Counters of the last event.  Synchronises `stream`.  HOUGH_EDEVICE if device_error != 0. */
int hough_get_stats(hough_ctx *ctx, hough_stats *out, void *stream);

/*
 * Whole path on one event: hough_vote, hough_peaks, hough_stage2 and
 * hough_get_candidates in one call (hits and candidates both in `where` memory).
 * Synchronises `stream`.  With HOUGH_HOST the hits are checked on the device
 * (the predicates of hough_vote's host check); a bad hit makes the call return
 * HOUGH_EINVAL after it has synchronised, with no candidates copied.  The first
 * HOUGH_HOST call allocates the context's pinned result staging
 * (max_candidates records), kept until hough_destroy.
 */
int hough_process(hough_ctx *ctx, const float *r, const float *phi, const float *z,
                  const uint8_t *layer, int64_t n_hits, hough_candidate *out, int32_t cap,
                  int32_t *n_out, int where, void *stream);

/*
 * Kernel configuration of a context.
 *
 * vote_mode HOUGH_VOTE_GATHER (default): for every layer whose hits share one radius the
 * accumulator is computed cell by cell from the per-bucket extrema of the hits' azimuth fraction
 * (identical result, no atomics).  Each CTA of the gather kernel (gather_threads threads) owns a
 * tile of gather_rows rows x gather_cols columns and stages the slices of the bucket profile the
 * tile reads into shared memory with bulk asynchronous copies.  Layers whose hits lie at several
 * radii are added by the shared-atomic scatter kernel.
 * vote_mode HOUGH_VOTE_SCATTER: every layer by the shared-atomic scatter kernel (Sec. 6.1), each
 * CTA owning a tile of tile_qpt rows x tile_phi columns in shared memory.
 * vote_mode HOUGH_VOTE_FUSED (layer masks without a d0 axis): the gather and the peak search in
 * one kernel, a CTA (gather_threads threads) per band of band_rows full rows, which computes the
 * band's cells and those of the row above and below it into shared memory and searches the band
 * for peaks there: the accumulator is neither written to nor read back from device memory, and
 * hough_get_accumulator / hough_batch_accumulator return HOUGH_ENOTREADY.  When a layer's hits
 * lie at several radii the scatter kernel must add its votes first; the fused kernel then writes
 * the band's rows and the peak kernel runs as in the other modes.  Needs (band_rows + 2) *
 * n_phi * 2 bytes of shared memory.
 * The peak search works on bands of band_rows rows.
 *
 * With the count accumulator the gather counts its tile of gather_rows x gather_cols cells in
 * 32-bit shared counters (gather_rows * gather_cols * 4 bytes plus a staging slot of at least
 * 16 KB must fit in shared memory) and the scatter's tile holds 32-bit counters; both saturate
 * to 16 bits when the tile is written out.
 *
 * tile_phi must divide n_phi and be a multiple of 64; tile_qpt in 1..256; threads in
 * {128, 256, 512, 1024}; tile_qpt * tile_phi * 2 bytes (4 with the count accumulator) must fit
 * in shared memory; band_rows in 1..16 with (band_rows + 2) * n_phi bytes (twice that with the
 * count accumulator, three times with a d0 axis) of shared memory; gather_rows in 1..32 (0: 4);
 * gather_cols a multiple of 64 dividing n_phi (0: the largest such up to 512) with
 * n_layers * (gather_cols + 64) * 8 bytes of shared memory; gather_threads in {256, 512, 1024}
 * (0: 256).  HOUGH_EINVAL otherwise.  Every configuration gives the same results.
 */
#define HOUGH_VOTE_GATHER  0
#define HOUGH_VOTE_SCATTER 1
#define HOUGH_VOTE_FUSED   2

typedef struct hough_tiling {
    int32_t tile_qpt;
    int32_t tile_phi;
    int32_t threads;
    int32_t vote_mode;
    int32_t band_rows;
    int32_t gather_rows;
    int32_t gather_cols;
    int32_t gather_threads;
} hough_tiling;

int hough_set_tiling(hough_ctx *ctx, const hough_tiling *tiling);
int hough_get_tiling(const hough_ctx *ctx, hough_tiling *tiling);

/*
 * Device time of the last event's steps, measured with CUDA events recorded on the stream each
 * call was given (enabled by hough_enable_timing; off by default).  stage_ms: hit staging;
 * vote_ms: the vote (= gather_ms + scatter_ms); peaks_ms: peak search (= band_peaks_ms +
 * compact_ms); stage2_ms: membership and the stage-2 vote.  gather_ms covers the gather kernel
 * (with HOUGH_VOTE_FUSED, the fused vote and peak search); scatter_ms the shared-atomic kernel;
 * band_peaks_ms the standalone peak kernel; compact_ms the candidate scan.  A kernel that did not
 * run for the event (the clearing kernel when the last event left the state clean, the candidate
 * scan when stage 2 reads the band lists) reports 0.  hough_get_timing synchronises;
 * HOUGH_ENOTREADY before a timed event.
 */
typedef struct hough_timing {
    float stage_ms, vote_ms, peaks_ms, stage2_ms;
    float gather_ms, scatter_ms, band_peaks_ms, compact_ms;
    float member_ms, large_ms;   /* stage2_ms = member_ms (the confirmation kernel) + large_ms (0: no second kernel) */
    float clear_ms, count_ms, table_ms, scan_ms, sort_ms;   /* the staging kernels: stage_ms is their sum */
} hough_timing;

int hough_enable_timing(hough_ctx *ctx, int on);
int hough_get_timing(hough_ctx *ctx, hough_timing *out);

/*
 * Test of the device-side bounded wait (no GPU fault is made).  The gather vote's CTAs wait for
 * their bulk copies into shared memory with a bound of about a second; when it expires they set
 * HOUGH_DEVERR_TIMEOUT, wait once more with the full bound for the copies to land, and write
 * nothing (the accumulator is then incomplete).  first_bound < 0 makes the first bound of every
 * such wait of this context expire at once, so that a test can run that error path; 0 restores
 * the normal bound.  HOUGH_EINVAL without a context.
 */
int hough_set_copy_wait(hough_ctx *ctx, int first_bound);

/* Kernels this library has launched in the process so far (all contexts). */
uint64_t hough_kernel_launches(void);

/*
 * Throughput of 32-bit shared-memory atomicOr on device `device`, the ceiling of the vote step
 * (the vote is one shared atomic per cell update, Sec. 6.1).  pattern 0: the 32 lanes of a warp
 * hit 32 different banks; pattern 1: lanes hit words of a random permutation of a 16 KB tile
 * (the access pattern of the vote).  Runs a persistent grid of 152-multiple CTAs for about `ms`
 * milliseconds and returns lane-atomics per second in *atomics_per_s.  Synchronises the device.
 */
int hough_microbench_smem_or(int device, int pattern, double ms, double *atomics_per_s);

/*
 * Batched processing: many events of uneven size through the whole path (vote, peaks, membership,
 * stage 2) in one launch sequence, captured into a CUDA graph on the first call for a given
 * number of events and replayed afterwards.  Each event keeps its own accumulator and candidate
 * list, with the limits below applying per event (max_hits: over the whole batch); the candidate
 * records carry their member counts, but a batch keeps no member lists.
 */
typedef struct hough_batch_limits {
    int32_t max_events;       /* events per batch, >= 1 */
    int32_t max_candidates;   /* candidates kept per event, >= 1 */
    int64_t max_hits;         /* hits per batch, 1 .. 2^31 - 1 */
    int32_t max_members;      /* >= 1 (no member lists are kept in batches) */
    int32_t reserved;         /* must be 0 */
} hough_batch_limits;

typedef struct hough_batch hough_batch;

int hough_batch_create(const hough_geometry *geometry, const hough_binning *binning,
                       const hough_batch_limits *limits, int device, hough_batch **out);
void hough_batch_destroy(hough_batch *batch);

/* Kernel configuration, as hough_set_tiling; drops the captured graphs. */
int hough_batch_set_tiling(hough_batch *batch, const hough_tiling *tiling);

/*
 * Run the path on n_events events.  Hits of all events are concatenated in r, phi, z, layer
 * (as for hough_vote, in `where` memory); event e owns hits [hit_start[e], hit_start[e+1]) --
 * hit_start is a host array of n_events + 1 entries starting at 0.  With HOUGH_HOST the hits are
 * checked and copied; with HOUGH_DEVICE bad hits are dropped on the device.  Asynchronous on
 * `stream`: device-resident inputs must stay valid until the work has run.  HOUGH_ECAPACITY when
 * n_events or the hit total exceeds the limits.
 */
int hough_batch_run(hough_batch *batch, const float *r, const float *phi, const float *z,
                    const uint8_t *layer, const int64_t *hit_start, int32_t n_events, int where,
                    void *stream);

/*
 * All events' candidates of the last run, concatenated in event order into `out` (cap entries,
 * `where` memory); offsets (host, n_events + 1) receives each event's first index.  Each event's
 * list is in raster order with stage-2 fields filled.  HOUGH_ETRUNC when the total exceeds cap.
 * Synchronises `stream`.
 */
int hough_batch_candidates(hough_batch *batch, hough_candidate *out, int64_t cap, int64_t *offsets,
                           int where, void *stream);

/*
 * hough_batch_run with each step timed: the same kernels, enqueued one by one instead of as the
 * captured graph, with a CUDA event after each step; synchronises `stream` and fills in `out`
 * (hough_timing, below) the device time of the staging (stage_ms), the gather and scatter votes,
 * the peak search and candidate scan, and the confirmation (stage2_ms = member_ms).  The results
 * are those of hough_batch_run.
 */
int hough_batch_profile(hough_batch *batch, const float *r, const float *phi, const float *z,
                        const uint8_t *layer, const int64_t *hit_start, int32_t n_events, int where,
                        void *stream, hough_timing *out);

/* Counters of one event of the last run.  Synchronises `stream`. */
int hough_batch_stats(hough_batch *batch, int32_t event, hough_stats *out, void *stream);

/* The accumulator of one event of the last run.  Synchronises `stream`.  HOUGH_ENOTREADY under
 * vote_mode HOUGH_VOTE_FUSED. */
int hough_batch_accumulator(hough_batch *batch, int32_t event, uint16_t *out, int where, void *stream);

/*
 * Autotuning of a batch's kernel configuration (the paper tuned per target by hand with
 * preprocessor constants, Sec. 6.1).  hough_batch_autotune times whole batches of the given events
 * (inputs as hough_batch_run; host inputs are copied to the device once, outside the timing) for
 * a sweep of configurations -- the gather tile (rows x columns x threads), the shared-atomic
 * scatter tile of the paper's design (64..256 q/pT rows x 256..512 phi0 columns x threads), then
 * the peak band height -- each as `reps` (1..100) graph replays after one untimed replay, checks
 * that all give the same candidate total (HOUGH_EDEVICE otherwise), and applies the fastest to the
 * batch.  With a cache file (may be NULL) an entry for this GPU, SM count, axes and batch size
 * (rounded up to a power of two) is applied without timing; a new result is appended to the file
 * (one text line per entry).  Synchronises the device.
 */
typedef struct hough_tune_result {
    hough_tiling tiling;     /* the configuration applied */
    float ms;                /* its mean time per batch */
    float default_ms;        /* the default configuration's (0 when read from the cache) */
    int32_t tried;           /* configurations timed */
    int32_t from_cache;      /* 1 when the configuration came from the cache file */
} hough_tune_result;

int hough_batch_autotune(hough_batch *batch, const hough_geometry *geometry, const hough_binning *binning,
                         const float *r, const float *phi, const float *z, const uint8_t *layer,
                         const int64_t *hit_start, int32_t n_events, int where, int32_t reps,
                         const char *cache_path, hough_tune_result *out);

/* The cached configuration for these axes, this device and batch size: HOUGH_ENOTREADY when none. */
int hough_tune_lookup(const char *cache_path, const hough_geometry *geometry, const hough_binning *binning,
                      int device, int32_t n_events, hough_tiling *out);

/*
 * Served mode: a trigger-style request loop with continuous batching (the paper runs events one at
 * a time, Sec. 6-7; it has no serving loop).  Events are submitted one by one as they arrive; a
 * dispatcher thread owned by the server launches whatever has been admitted as one batch (the
 * hough_batch path: one replayed graph) as soon as fewer than max_in_flight batches are on the
 * GPU, so events that arrive while others run join the next launch, and launches of different
 * lanes overlap on the device, one stream each.  A lane is one batch's device buffers
 * (accumulators and candidate lists for max_batch_events events, allocated once and kept
 * resident) plus pinned host staging for its hits and results.  Lanes are created within
 * memory_budget; admission is bounded by them: when the filling batch is full and no lane is free,
 * a new event is refused with HOUGH_EBUSY (dead time), never queued without bound.
 *
 * Each event's result -- its candidate list in raster order with stage-2 fields, its vote count
 * and device-side error bits -- is the same as hough_process gives for that event alone.
 */
typedef struct hough_serve_config {
    int32_t lanes;             /* device batch slots: 0 = as many as memory_budget holds, at most 4; else >= 2 */
    int32_t max_in_flight;     /* batches on the GPU at once: 0 = lanes - 1; else 1 .. lanes - 1 */
    int32_t max_batch_events;  /* events per launch, >= 1 */
    int32_t max_candidates;    /* candidates kept per event, >= 1 */
    int64_t max_batch_hits;    /* hits per launch (and per event), 1 .. 2^31 - 1 */
    int32_t max_members;       /* >= 1 (served events keep no member lists) */
    int32_t reserved;          /* must be 0 */
    int64_t memory_budget;     /* device bytes all lanes may hold; 0 = no budget */
    int64_t lane_timeout_us;   /* watchdog: a launch not finished after this fails with HOUGH_ETIMEDOUT and
                                  its lane is retired; 0 = no watchdog */
} hough_serve_config;

/* Per-event result of hough_serve_poll.  Times are CLOCK_MONOTONIC nanoseconds (hough_serve_clock_ns). */
typedef struct hough_serve_result {
    uint64_t ticket;
    int64_t  arrival_ns;      /* as given to hough_serve_submit (or its submission time) */
    int64_t  submit_ns;       /* when hough_serve_submit was entered */
    int64_t  launch_ns;       /* when its batch was launched */
    int64_t  done_ns;         /* when its result reached host memory */
    int64_t  n_candidates;
    uint64_t votes;           /* stage-1 votes cast by the event */
    int32_t  status;          /* HOUGH_OK, HOUGH_EDEVICE (device_error set), HOUGH_ENOMEM, HOUGH_ETIMEDOUT, ... */
    int32_t  batch_events;    /* events that shared its launch */
    uint32_t device_error;    /* HOUGH_DEVERR_* bits */
    uint32_t reserved;
} hough_serve_result;

/* Server counters (hough_serve_get_stats). */
typedef struct hough_serve_stats {
    int64_t submitted;          /* hough_serve_submit calls with valid arguments */
    int64_t admitted;           /* events given a ticket */
    int64_t rejected_busy;      /* refused with HOUGH_EBUSY */
    int64_t rejected_invalid;   /* refused as malformed (bad layer, radius or coordinate) */
    int64_t completed;          /* events whose result reached the host */
    int64_t failed;             /* events finished with an error status */
    int64_t launches;           /* batches launched */
    int64_t launched_events;    /* events over all launches */
    int64_t max_in_flight;      /* most batches on the GPU at once */
    int64_t timeouts;           /* launches failed by the watchdog */
    int64_t alloc_failures;     /* result-buffer allocations that failed */
    int64_t retired_lanes;
    int64_t lanes;              /* lanes in service */
    int64_t in_flight;          /* batches on the GPU now */
    int64_t pending_tickets;    /* tickets not yet polled */
    int64_t device_bytes;       /* device memory held by the lanes */
} hough_serve_stats;

typedef struct hough_server hough_server;

/* Host-side fault injection for tests (no GPU fault is ever made): */
#define HOUGH_SERVE_FAULT_HOLD  1   /* launch nothing while on (a stalled dispatcher) */
#define HOUGH_SERVE_FAULT_STALL 2   /* treat every in-flight lane as never finishing while on (a stalled stream) */
#define HOUGH_SERVE_FAULT_ALLOC 3   /* the next result-buffer acquisition fails with HOUGH_ENOMEM */

/*
 * Create a server on `device`: allocates the lanes (HOUGH_ENOMEM when fewer than two, or fewer than
 * `lanes`, fit the budget), captures every batch size's graph, and starts the dispatcher thread.
 * Results live in pinned host blocks: a mapped part of max(16384, 1024 * max_batch_events)
 * candidates the pack kernel writes to, and an overflow grown to the largest batch.  A finished
 * batch's block is shared by its events until the last of them is polled (poll copies from it);
 * the pool holds at most 3 * lanes blocks, beyond which (unpolled results piling up) each event's
 * candidates are copied out of its lane's block instead.  Pinned memory is outside memory_budget.
 */
int hough_serve_create(const hough_geometry *geometry, const hough_binning *binning,
                       const hough_serve_config *config, int device, hough_server **out);

/* Stop the dispatcher, wait for the GPU work in flight, and free everything (unpolled results are dropped). */
void hough_serve_destroy(hough_server *server);

/* The server's clock: CLOCK_MONOTONIC in nanoseconds. */
int64_t hough_serve_clock_ns(void);

/*
 * Admit one event: its hits (host memory, n_hits entries; checked as hough_vote does, a malformed
 * event returns that check's status and is counted in rejected_invalid) are copied into the
 * filling batch's pinned staging before the call returns.  arrival_ns (hough_serve_clock_ns time;
 * 0 = now) is the event's arrival for latency.  *ticket identifies it for hough_serve_poll.
 * HOUGH_EBUSY when no lane can take it.  Thread-safe.
 */
int hough_serve_submit(hough_server *server, const float *r, const float *phi, const float *z,
                       const uint8_t *layer, int64_t n_hits, int64_t arrival_ns, uint64_t *ticket);

/*
 * Wait up to timeout_us (>= 0) for the event `ticket`; then copy up to cap of its candidates to
 * `out` (host), fill *result (may be NULL) and release the ticket.  Returns HOUGH_ETIMEDOUT (ticket
 * kept) if it has not finished, the event's status if that is an error, HOUGH_ETRUNC when out is
 * given and holds fewer than its candidates, else HOUGH_OK.  Thread-safe.
 */
int hough_serve_poll(hough_server *server, uint64_t ticket, hough_candidate *out, int64_t cap,
                     hough_serve_result *result, int64_t timeout_us);

/* Wait up to timeout_us until every admitted event has finished (HOUGH_ETIMEDOUT otherwise). */
int hough_serve_drain(hough_server *server, int64_t timeout_us);

int hough_serve_get_stats(hough_server *server, hough_serve_stats *out);

/* One event's hits in host memory, for hough_serve_replay. */
typedef struct hough_event_view {
    const float *r, *phi, *z;
    const uint8_t *layer;
    int64_t n_hits;
} hough_event_view;

/*
 * Trigger emulation: offer n events to the server at the given arrival times (hough_serve_clock_ns
 * time, non-decreasing).  Arrival i is event pool[i % n_pool]; `threads` submitter threads (1..64)
 * take arrivals i = t mod threads, each waiting for its arrival time before hough_serve_submit,
 * while one more thread polls every admitted event in arrival order and drops its candidates.
 * results[i] (n entries) receives arrival i's result; a refused arrival has ticket 0 and the
 * refusal (HOUGH_EBUSY) as its status.  Returns when every arrival has been offered and every
 * admitted event polled; HOUGH_ETIMEDOUT when some admitted event had no result within 60 s.
 */
int hough_serve_replay(hough_server *server, const hough_event_view *pool, int32_t n_pool,
                       const int64_t *arrival_ns, int64_t n, int32_t threads, hough_serve_result *results);

/* Switch a host-side fault (HOUGH_SERVE_FAULT_*) on (on != 0) or off. */
int hough_serve_inject(hough_server *server, int fault, int on);

/*
 * Stage-1 vote of one event with no allocation at all.  The paper has no counterpart: this exists
 * for callers that may not allocate device memory while they run -- a trigger's real-time event
 * loop, where cudaMalloc and cudaFree can synchronise the whole device and take unbounded time, or
 * a framework that has handed all device memory to its own pool -- and therefore cannot create a
 * hough_ctx.
 *
 * Runs the staging and vote kernels of hough_vote on the hits r, phi, z, layer (device pointers,
 * n_hits entries, same meaning and checks as hough_vote with HOUGH_DEVICE) and writes the
 * (stacked) rows x n_phi row-major cells -- layer masks, or counts with HOUGH_ACC_COUNTS -- to
 * `accumulator` (device, caller-owned, 16-byte aligned: the kernel writes it in 16-byte vectors;
 * another alignment returns HOUGH_EINVAL before any work).  If `device_error`
 * is not NULL it receives (device memory, asynchronously) the HOUGH_DEVERR_* bits of dropped hits.
 * The geometry and binning are read at each call; the stage-2 fields of the binning are ignored.
 *
 * Scratch: one fixed 8 MiB array in device memory, reserved on a GPU when the library's device
 * code is loaded there and held until the process exits.  With the CUDA runtime's lazy module
 * loading (its default) that happens at the first call on each device, which therefore does
 * reserve memory: make it at start-up, outside the real-time loop and before any stream capture;
 * later calls allocate nothing.  Limits: n_hits <= 131072, rows (n_qpt, times n_d0 with a d0 axis)
 * <= 1024, n_phi <= 4096; larger inputs return HOUGH_ECAPACITY before any work.  Each call looks up
 * the array's device address on the current device (no allocation), so a device reset is
 * harmless.  Every call reuses the same array and clears what must start empty, so calls
 * whose work may overlap on the GPU race: issue them on one stream or synchronise between them.
 * Asynchronous on `stream` (a cudaStream_t of the current device, NULL for the legacy stream).
 */
int hough_vote_static(const hough_geometry *geometry, const hough_binning *binning, const float *r,
                      const float *phi, const float *z, const uint8_t *layer, int64_t n_hits,
                      uint16_t *accumulator, uint32_t *device_error, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HOUGH_H */
