// autotune.cu -- launch-shape autotuner (psso_autotune).
//
// The launch shape of a handle -- particles per block of the persistent
// generation kernel, and the grid of the batched pipeline's step kernels --
// never changes what a run computes (every draw is keyed by (seed, stream,
// particle, variable, generation), every fitness sum has a fixed lane order,
// and the gBest is the lowest-index arg-min), only how fast it runs.  The
// best shape depends on the row width, the swarm sizes, the function and the
// precision, so it is measured rather than modelled: each candidate gets a
// scratch handle built through the public entry points, a few warm-up
// generations, and CUDA-event timing of the requested generations on a
// private stream.  The search is a coordinate descent: particles per block
// first (persistent kernel), then blocks per SM (batched step kernels) with
// that choice fixed.  Results are cached per process.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "psso.h"
#include "psso_internal.h"

namespace {

constexpr int WARM_GENERATIONS = 3;

struct Tuned {
    int32_t threads_per_block;
    int32_t batch_blocks_per_sm;
    double best_ms;
    double default_ms;
};

std::mutex g_cache_mutex;
std::map<std::string, Tuned> g_cache;

// Everything that can change the timing of a candidate: shapes, functions,
// lattice, Eq. 2.1 thresholds (they set the fresh-draw rate) and the
// configuration, except the fields that only select where work is enqueued
// or what is logged.
std::string cache_key(const psso_problem* pr, int32_t count, const psso_config& c, int32_t gens, int device)
{
    std::ostringstream k;
    k << device << '|' << gens << '|' << c.precision << ',' << c.threads_per_block << ','
      << c.single_block_max << ',' << c.max_blocks << ',' << c.residency << ',' << c.pipeline << ','
      << c.tensor_rotation << ',' << c.batch_stream << ',' << c.batch_blocks_per_sm << '|';
    for (int32_t q = 0; q < count; ++q)
        k << pr[q].fn << ',' << pr[q].lattice << ',' << pr[q].N << ',' << pr[q].D << ',' << pr[q].Cg << ','
          << pr[q].Cp << ',' << pr[q].Cw << ';';
    return k.str();
}

// Mean ms per generation of one configuration; negative if the configuration
// is rejected (not a valid shape for these problems).  `st_out` receives the
// handle's launch counters.
psso_status time_config(const psso_problem* pr, int32_t count, psso_config c, int32_t gens, cudaStream_t s,
                        double* ms, psso_stats_t* st_out)
{
    c.stream = s;
    c.log_stride = 0;
    c.log_capacity = 0;
    psso_handle h = nullptr;
    psso_status st = psso_create_ex(pr, count, &c, &h);
    if (st != PSSO_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        st = psso_run(h, WARM_GENERATIONS);
        if (st == PSSO_OK) st = psso_sync(h);
        if (st == PSSO_OK) {
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) st = psso_run(h, gens);
            if (e == cudaSuccess && st == PSSO_OK) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess && st == PSSO_OK) st = psso_sync(h);
            float t = 0.f;
            if (e == cudaSuccess && st == PSSO_OK) e = cudaEventElapsedTime(&t, e0, e1);
            *ms = (double)t / gens;
        }
    }
    if (st == PSSO_OK && st_out) st = psso_stats(h, st_out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    psso_destroy(h);
    if (st == PSSO_OK && e != cudaSuccess) {
        psso::set_last_error(cudaGetErrorString(e));
        return PSSO_ERR_CUDA;
    }
    return st;
}

}  // namespace

extern "C" psso_status psso_autotune(const psso_problem* problems, int32_t count, const psso_config* cfg,
                                     int32_t generations, psso_config* tuned, psso_tune_report* report)
{
    if (!problems || count < 1 || !tuned) {
        psso::set_last_error("psso_autotune: need problems, count >= 1 and tuned");
        return PSSO_ERR_ARG;
    }
    if (generations < 1 || generations > 100000) {
        psso::set_last_error("psso_autotune: generations must be in [1, 100000]");
        return PSSO_ERR_ARG;
    }
    psso_config base{};
    if (cfg) base = *cfg;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        psso::set_last_error("psso_autotune: no CUDA device");
        return PSSO_ERR_CUDA;
    }
    const std::string key = cache_key(problems, count, base, generations, device);
    {
        std::lock_guard<std::mutex> lock(g_cache_mutex);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            *tuned = base;
            tuned->threads_per_block = it->second.threads_per_block;
            tuned->batch_blocks_per_sm = it->second.batch_blocks_per_sm;
            if (report) {
                std::memset(report, 0, sizeof *report);
                report->threads_per_block = it->second.threads_per_block;
                report->batch_blocks_per_sm = it->second.batch_blocks_per_sm;
                report->best_ms = it->second.best_ms;
                report->default_ms = it->second.default_ms;
            }
            return PSSO_OK;
        }
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        psso::set_last_error("psso_autotune: cudaStreamCreate failed");
        return PSSO_ERR_CUDA;
    }
    psso_config best = base;
    double best_ms = 0.0, default_ms = 0.0;
    psso_stats_t st0{};
    int32_t timed = 0;
    psso_status st = time_config(problems, count, base, generations, s, &default_ms, &st0);
    if (st == PSSO_OK) {
        ++timed;
        best_ms = default_ms;
        // Particles per block of the persistent kernel (one control warp plus
        // compute warps when a single swarm spans many blocks).
        if (st0.blocks > 0 && base.threads_per_block == 0) {
            static const int32_t tpb[] = {64, 96, 128, 160, 192, 256, 288, 320, 384, 448, 512};
            for (int32_t v : tpb) {
                if (v == st0.threads_per_block) continue;   // the default's own shape
                psso_config c = best;
                c.threads_per_block = v;
                double ms = 0.0;
                const psso_status r = time_config(problems, count, c, generations, s, &ms, nullptr);
                if (r == PSSO_ERR_ARG || r == PSSO_ERR_UNSUPPORTED) continue;   // not a shape for these rows
                if (r != PSSO_OK) { st = r; break; }
                ++timed;
                if (ms < best_ms) { best_ms = ms; best = c; }
            }
        }
        // Grid of the batched pipeline's step kernels.
        if (st == PSSO_OK && st0.batch_classes > 0 && base.batch_blocks_per_sm == 0) {
            for (int32_t v = 1; v <= 8; ++v) {
                psso_config c = best;
                c.batch_blocks_per_sm = v;
                double ms = 0.0;
                const psso_status r = time_config(problems, count, c, generations, s, &ms, nullptr);
                if (r == PSSO_ERR_ARG || r == PSSO_ERR_UNSUPPORTED) continue;
                if (r != PSSO_OK) { st = r; break; }
                ++timed;
                if (ms < best_ms) { best_ms = ms; best = c; }
            }
        }
    }
    cudaStreamDestroy(s);
    if (st != PSSO_OK) return st;
    best.stream = base.stream;
    best.log_stride = base.log_stride;
    best.log_capacity = base.log_capacity;
    *tuned = best;
    {
        std::lock_guard<std::mutex> lock(g_cache_mutex);
        g_cache[key] = Tuned{best.threads_per_block, best.batch_blocks_per_sm, best_ms, default_ms};
    }
    if (report) {
        std::memset(report, 0, sizeof *report);
        report->candidates = timed;
        report->threads_per_block = best.threads_per_block;
        report->batch_blocks_per_sm = best.batch_blocks_per_sm;
        report->best_ms = best_ms;
        report->default_ms = default_ms;
    }
    return PSSO_OK;
}
