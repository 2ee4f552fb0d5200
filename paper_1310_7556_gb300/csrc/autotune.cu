// Autotuner of the batched path's kernel configuration (the paper tuned its kernels per target by
// hand, with preprocessor constants, Sec. 6.1; here the choice is measured on the device).
//
// The sweep times whole batches -- every kernel of the path, as the captured graph runs them --
// for each configuration of the stage-1 vote and the peak search:
//   gather vote: rows x columns of the accumulator tile per CTA, threads per CTA;
//   scatter vote (the paper's shared-atomic design, and the count accumulator's): q/pT rows x phi0
//   columns of the shared tile, threads per CTA (each thread handles one hit at a time);
//   peak search: rows per band.
// It proceeds coordinate-wise (the vote configuration with the default band height, then the band
// height with the best vote configuration), times `reps` replays of each after one untimed replay
// (which also captures the graph), and checks that every configuration yields the same candidate
// total -- every configuration computes the same result.  The fastest is applied to the batch and,
// given a cache file, appended to it under a key of the GPU, its SM count, the axes and the batch
// size, so that later processes take it without timing.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "hough_internal.cuh"

using namespace hough;

namespace {

int tfail(int code, const char *msg) { return set_last_error(code, msg); }

std::string tune_key(const hough_geometry *g, const hough_binning *bn, int device, int n_events)
{
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, device);
    int bucket = 1;
    while (bucket < n_events) bucket <<= 1;
    char buf[512];
    std::snprintf(buf, sizeof(buf),
                  "gpu=%s;sms=%d;layers=%d;b=%.9g;acc=%d;qpt=%d[%.9g,%.9g];phi=%d;thr=%d;cot=%d[%.9g,%.9g];z0=%d[%.9g,%.9g];d0=%d[%.9g,%.9g];events<=%d",
                  prop.name, prop.multiProcessorCount, g->n_layers, g->b_tesla, bn->accumulator, bn->n_qpt, bn->qpt_min, bn->qpt_max,
                  bn->n_phi, bn->threshold, bn->n_cot, bn->cot_min, bn->cot_max, bn->n_z0, bn->z0_min_cm,
                  bn->z0_max_cm, bn->n_d0, bn->n_d0 > 0 ? bn->d0_min_cm : 0.0, bn->n_d0 > 0 ? bn->d0_max_cm : 0.0, bucket);
    for (char *p = buf; *p; ++p)
        if (*p == '\t' || *p == '\n') *p = ' ';
    return buf;
}

bool read_cache(const char *path, const std::string &key, hough_tiling *out, float *ms)
{
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {   // the last entry for a key wins
        const size_t tab = line.find('\t');
        if (tab == std::string::npos || line.compare(0, tab, key) != 0 || tab != key.size()) continue;
        std::istringstream in(line.substr(tab + 1));
        hough_tiling t{};
        float m = 0.f;
        if (in >> t.tile_qpt >> t.tile_phi >> t.threads >> t.vote_mode >> t.band_rows >> t.gather_rows >>
            t.gather_cols >> t.gather_threads >> m) {
            *out = t;
            *ms = m;
            found = true;
        }
    }
    return found;
}

bool append_cache(const char *path, const std::string &key, const hough_tiling &t, float ms)
{
    std::ofstream f(path, std::ios::app);
    if (!f) return false;
    f << key << '\t' << t.tile_qpt << ' ' << t.tile_phi << ' ' << t.threads << ' ' << t.vote_mode << ' '
      << t.band_rows << ' ' << t.gather_rows << ' ' << t.gather_cols << ' ' << t.gather_threads << ' ' << ms << '\n';
    return (bool)f;
}

}  // namespace

extern "C" {

int hough_tune_lookup(const char *cache_path, const hough_geometry *geometry, const hough_binning *binning,
                      int device, int32_t n_events, hough_tiling *out)
{
    if (!cache_path || !geometry || !binning || !out || n_events < 1) return tfail(HOUGH_EINVAL, "bad arguments");
    float ms = 0.f;
    if (!read_cache(cache_path, tune_key(geometry, binning, device, n_events), out, &ms))
        return tfail(HOUGH_ENOTREADY, "no tuned configuration for these axes, device and batch size");
    return HOUGH_OK;
}

int hough_batch_autotune(hough_batch *b, const hough_geometry *geometry, const hough_binning *binning,
                         const float *r, const float *phi, const float *z, const uint8_t *layer,
                         const int64_t *hit_start, int32_t n_events, int where, int32_t reps,
                         const char *cache_path, hough_tune_result *out)
{
    if (!b || !geometry || !binning || !hit_start || !out || reps < 1 || reps > 100)
        return tfail(HOUGH_EINVAL, "bad arguments");
    if (where != HOUGH_HOST && where != HOUGH_DEVICE) return tfail(HOUGH_EINVAL, "bad where");
    std::memset(out, 0, sizeof(*out));
    int device = 0;
    cudaGetDevice(&device);
    const Axes ax = make_axes(geometry, binning);
    const std::string key = tune_key(geometry, binning, device, n_events);
    if (cache_path) {
        hough_tiling t{};
        float ms = 0.f;
        if (read_cache(cache_path, key, &t, &ms) && check_tiling_for(ax, device, &t) == HOUGH_OK) {
            int rc = hough_batch_set_tiling(b, &t);
            if (rc) return rc;
            out->tiling = t;
            out->ms = ms;
            out->from_cache = 1;
            return HOUGH_OK;
        }
    }
    // device-resident copies of host inputs, so that the timing covers the path alone
    const int64_t n = n_events > 0 ? hit_start[n_events] : 0;
    std::vector<void *> tmp;
    const float *dr = r, *dphi = phi, *dz = z;
    const uint8_t *dlayer = layer;
    auto cleanup = [&] {
        for (void *p : tmp) cudaFree(p);
    };
    if (where == HOUGH_HOST && n > 0) {
        float *a = nullptr, *bb = nullptr, *c = nullptr;
        uint8_t *d = nullptr;
        if (cudaMalloc(&a, 4 * n) || cudaMalloc(&bb, 4 * n) || cudaMalloc(&c, 4 * n) || cudaMalloc(&d, n)) {
            if (a) cudaFree(a);
            if (bb) cudaFree(bb);
            if (c) cudaFree(c);
            return tfail(HOUGH_ENOMEM, "autotune: device copies of the hits");
        }
        tmp = {a, bb, c, d};
        cudaMemcpy(a, r, 4 * n, cudaMemcpyHostToDevice);
        cudaMemcpy(bb, phi, 4 * n, cudaMemcpyHostToDevice);
        cudaMemcpy(c, z, 4 * n, cudaMemcpyHostToDevice);
        cudaMemcpy(d, layer, n, cudaMemcpyHostToDevice);
        dr = a; dphi = bb; dz = c; dlayer = d;
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) || cudaEventCreate(&e0) || cudaEventCreate(&e1)) {
        cleanup();
        return tfail(HOUGH_ECUDA, "autotune: stream or events");
    }
    std::vector<int32_t> offs(n_events + 1);
    int64_t reference_total = -1;
    int rc = HOUGH_OK;
    // time one configuration: < 0 when it is not allowed on this device, else mean ms per batch
    auto time_config = [&](const hough_tiling &t, float *ms) -> int {
        *ms = -1.f;
        if (check_tiling_for(ax, device, &t) != HOUGH_OK) return HOUGH_OK;
        int q = hough_batch_set_tiling(b, &t);
        if (q) return q;
        if ((q = batch_run(b, dr, dphi, dz, dlayer, hit_start, n_events, HOUGH_DEVICE, s, false))) return q;
        if (cudaEventRecord(e0, s)) return tfail(HOUGH_ECUDA, "autotune: event");
        for (int k = 0; k < reps; ++k)
            if ((q = batch_run(b, dr, dphi, dz, dlayer, hit_start, n_events, HOUGH_DEVICE, s, false))) return q;
        if (cudaEventRecord(e1, s)) return tfail(HOUGH_ECUDA, "autotune: event");
        if ((q = batch_enqueue_offsets(b, offs.data(), s))) return q;
        if (cudaStreamSynchronize(s)) return tfail(HOUGH_ECUDA, "autotune: a timed batch failed");
        float total = 0.f;
        cudaEventElapsedTime(&total, e0, e1);
        *ms = total / reps;
        const int64_t cands = offs[n_events];
        if (reference_total < 0) reference_total = cands;
        else if (cands != reference_total)
            return tfail(HOUGH_EDEVICE, "autotune: two configurations gave different candidate totals");
        ++out->tried;
        return HOUGH_OK;
    };
    const Tiling d0 = default_tiling_for(ax);
    hough_tiling best{};
    public_tiling(d0, &best);
    float best_ms = -1.f;
    std::vector<hough_tiling> votes;
    votes.push_back(best);   // the default first: it is the reference and the baseline
    for (int rows : {4, 8, 16, 32})
        for (int cols : {128, 256, 512, 1024})
            for (int threads : {256, 512, 1024}) {
                hough_tiling t = best;
                t.vote_mode = HOUGH_VOTE_GATHER;
                t.gather_rows = rows;
                t.gather_cols = cols;
                t.gather_threads = threads;
                if (rows * cols / 8 < threads / 2) continue;   // under half the threads would have cells
                votes.push_back(t);
            }
    for (int tq : {32, 64, 128})   // the scatter kernel's lanes take 32 rows each
        for (int tp : {128, 256, 512})
            for (int threads : {256, 512, 1024}) {
                hough_tiling t = best;
                t.vote_mode = HOUGH_VOTE_SCATTER;
                t.tile_qpt = tq;
                t.tile_phi = tp;
                t.threads = threads;
                votes.push_back(t);
            }
    for (size_t k = 0; k < votes.size() && !rc; ++k) {
        float ms;
        rc = time_config(votes[k], &ms);
        if (k == 0) out->default_ms = ms;
        if (!rc && ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
            best_ms = ms;
            best = votes[k];
        }
    }
    for (int band : {2, 4, 8}) {
        if (rc) break;
        hough_tiling t = best;
        t.band_rows = band;
        float ms;
        rc = time_config(t, &ms);
        if (!rc && ms >= 0.f && ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cleanup();
    if (rc) return rc;
    if ((rc = hough_batch_set_tiling(b, &best))) return rc;
    out->tiling = best;
    out->ms = best_ms;
    if (cache_path && !append_cache(cache_path, key, best, best_ms))
        return tfail(HOUGH_EINVAL, "autotune: the cache file could not be written");
    return HOUGH_OK;
}

}  // extern "C"
