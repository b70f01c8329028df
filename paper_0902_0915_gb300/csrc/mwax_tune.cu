// mwax_tune.cu -- autotuner for the tensor-core correlator.
//
// Picks the tuning fields of an mwax_job (MMA shape, shared-memory stages,
// L2 prefetch distance, unpack/correlate pipelining, channels per pass, time
// ranges per work item) by timing candidate configurations with CUDA events
// on the caller's own device buffers, on the caller's stream.  For a batch,
// the launch-wide fields first, then each job's time ranges per work item.  The choice can be cached in a
// text file named by the environment variable MWAX_TUNE_CACHE, one line per
// (device, shape) key; mwax_plan applies a cached choice to jobs whose
// tuning fields are all zero.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "mwax_internal.h"

namespace mwax {
namespace {

struct Cand {
  int mma_shape, stages, prefetch, pipeline, chan_group, k_split;
};

// Timed calls per candidate (after one untimed call).
constexpr int kTuneReps = 3;

std::mutex g_cache_mu;

std::string tune_key(const mwax_job &j) {
  int dev = 0;
  cudaDeviceProp prop;
  memset(&prop, 0, sizeof(prop));
  if (cudaGetDevice(&dev) == cudaSuccess) cudaGetDeviceProperties(&prop, dev);
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|sm%d|N%d|C%d|T%d|b%d|k%d", prop.name, prop.multiProcessorCount,
           j.n_inputs, j.n_chan, j.n_time, j.sample_bits, j.kind);
  for (char *c = buf; *c; ++c)
    if (*c == ' ' || *c == '\t') *c = '_';
  return buf;
}

bool cache_lookup(const std::string &key, Cand *c, double *ms) {
  const char *path = getenv("MWAX_TUNE_CACHE");
  if (!path || !*path) return false;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    char k[600];
    Cand t;
    double m = 0;
    if (sscanf(line, "%599s %d %d %d %d %d %d %lf", k, &t.mma_shape, &t.stages, &t.prefetch,
               &t.pipeline, &t.chan_group, &t.k_split, &m) == 8 &&
        key == k) {
      *c = t;  // the last matching line wins
      *ms = m;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const std::string &key, const Cand &c, double ms) {
  const char *path = getenv("MWAX_TUNE_CACHE");
  if (!path || !*path) return;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %d %d %d %.6f\n", key.c_str(), c.mma_shape, c.stages, c.prefetch,
          c.pipeline, c.chan_group, c.k_split, ms);
  fclose(f);
}

void apply(mwax_job *j, const Cand &c) {
  j->mma_shape = c.mma_shape;
  j->stages = c.stages;
  j->prefetch = c.prefetch;
  j->pipeline = c.pipeline;
  j->chan_group = c.chan_group;
  j->k_split = c.k_split;
}

// Mean device time of `reps` calls (after one warm-up), or a negative value
// if the configuration cannot run.
double time_single(const mwax_job &job, const void *volt, void *out, cudaStream_t st, int reps) {
  mwax_plan_t p = nullptr;
  if (mwax_plan(&p, &job, st) != MWAX_OK) return -1.0;
  double ms = -1.0;
  cudaEvent_t a = nullptr, b = nullptr;
  if (mwax_correlate(p, volt, job.n_inputs, job.n_chan, job.n_time, out) == MWAX_OK &&
      cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess &&
      cudaEventRecord(a, st) == cudaSuccess) {
    bool ok = true;
    for (int r = 0; r < reps && ok; ++r)
      ok = mwax_correlate(p, volt, job.n_inputs, job.n_chan, job.n_time, out) == MWAX_OK;
    float f = 0.f;
    if (ok && cudaEventRecord(b, st) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
        cudaEventElapsedTime(&f, a, b) == cudaSuccess && mwax_plan_status(p) == MWAX_OK)
      ms = f / reps;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  mwax_destroy(p);
  return ms;
}

double time_batch(const std::vector<mwax_job> &jobs, const void *const *volt, void *const *out,
                  cudaStream_t st, int reps) {
  mwax_plan_t p = nullptr;
  if (mwax_plan_batch(&p, jobs.data(), (int)jobs.size(), st) != MWAX_OK) return -1.0;
  double ms = -1.0;
  cudaEvent_t a = nullptr, b = nullptr;
  if (mwax_correlate_batch(p, volt, out) == MWAX_OK && cudaEventCreate(&a) == cudaSuccess &&
      cudaEventCreate(&b) == cudaSuccess && cudaEventRecord(a, st) == cudaSuccess) {
    bool ok = true;
    for (int r = 0; r < reps && ok; ++r) ok = mwax_correlate_batch(p, volt, out) == MWAX_OK;
    float f = 0.f;
    if (ok && cudaEventRecord(b, st) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
        cudaEventElapsedTime(&f, a, b) == cudaSuccess && mwax_plan_status(p) == MWAX_OK)
      ms = f / reps;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  mwax_destroy(p);
  return ms;
}

bool valid(const Cand &c) {
  const bool shape_ok = c.mma_shape >= 0 && c.mma_shape <= 4;
  const int max_st = correlate_tc_max_stages(c.mma_shape > 0 ? c.mma_shape - 1 : 0);
  return shape_ok && (c.stages == 0 || (c.stages >= 2 && c.stages <= max_st)) && c.k_split >= 0 &&
         c.k_split <= 8;
}

bool all_auto(const mwax_job &j) {
  return j.mma_shape == 0 && j.stages == 0 && j.prefetch == 0 && j.pipeline == 0 &&
         j.chan_group == 0 && j.k_split == 0;
}

}  // namespace

// Used by mwax_plan: fill the tuning fields of an all-auto job from the cache.
void apply_tune_cache(mwax_job *j) {
  if (!all_auto(*j) || j->engine != MWAX_ENGINE_TENSOR) return;
  Cand c;
  double ms;
  // a cached choice that this build cannot run (e.g. more stages than the
  // shape allows) is ignored
  if (cache_lookup(tune_key(*j), &c, &ms) && valid(c)) apply(j, c);
}

}  // namespace mwax

using namespace mwax;

extern "C" {

mwax_status mwax_autotune(mwax_job *job, const void *voltages, void *out, cudaStream_t stream,
                          mwax_tune_report *report) {
  mwax::NvtxRange nvtx_("mwax_autotune");
  if (!job || !voltages || !out) return MWAX_ERR_INVALID_ARG;
  mwax_tune_report rep;
  memset(&rep, 0, sizeof(rep));
  if (job->engine != MWAX_ENGINE_TENSOR) {
    if (report) *report = rep;
    return MWAX_OK;
  }
  const std::string key = tune_key(*job);
  Cand best;
  double best_ms = 0;
  if (cache_lookup(key, &best, &best_ms) && valid(best)) {
    apply(job, best);
    rep.from_cache = 1;
    rep.best_ms = best_ms;
    if (report) *report = rep;
    return MWAX_OK;
  }
  mwax_job base = *job;
  apply(&base, Cand{0, 0, 0, 0, 0, 0});
  // Candidate 0 is the plan's own default (every field automatic: the pair
  // mode where the integration is one exact segment, the checked single
  // segment for longer 8-bit exact jobs, else the narrow shape), so the
  // report's default_ms is that plan's time and a tuned choice can only
  // replace it by being measurably faster.  An explicit pair request
  // (mma_shape 3) on a job longer than one exact segment plans as the
  // checked single segment; explicit flush segments are not candidates.
  // Pair-mode candidates with time ranges per item fail to plan (and are
  // skipped) where the job cannot take them (FP16 kind, too few time blocks),
  // and so do the fused pair mode's (mma_shape 4) outside 4-bit exact jobs of
  // whole 16-input sample rows.
  const std::vector<Cand> cands = {
      {0, 0, 0, 0, 0, 0},  {3, 0, -1, 1, 0, 1}, {3, 0, -1, 1, 0, 2}, {3, 0, -1, 1, 0, 4},
      {3, 0, -1, 1, 0, 8}, {4, 0, -1, 1, 0, 1}, {4, 0, -1, 1, 0, 2}, {4, 0, -1, 1, 0, 4},
      {1, 2, -1, 1, 0, 0}, {1, 2, 8, 1, 0, 0},  {2, 4, -1, 1, 0, 0}, {2, 3, -1, 1, 0, 0},
      {1, 2, -1, 2, 0, 0}, {3, 0, -1, 2, 0, 1},
  };
  best_ms = -1.0;
  for (const Cand &c : cands) {
    mwax_job j = base;
    apply(&j, c);
    const double ms = time_single(j, voltages, out, stream, kTuneReps);
    // earlier (simpler) candidates win ties: a later one must be >1% faster
    if (ms > 0 && (best_ms < 0 || ms < 0.99 * best_ms)) {
      best_ms = ms;
      best = c;
    }
    if (&c == &cands[0]) rep.default_ms = ms;
    rep.candidates++;
  }
  if (best_ms < 0) return MWAX_ERR_UNSUPPORTED;
  apply(job, best);
  rep.best_ms = best_ms;
  cache_store(key, best, best_ms);
  if (report) *report = rep;
  return MWAX_OK;
}

mwax_status mwax_autotune_batch(mwax_job *jobs, int n_jobs, const void *const *voltages,
                                void *const *out, cudaStream_t stream, mwax_tune_report *report) {
  mwax::NvtxRange nvtx_("mwax_autotune_batch");
  if (!jobs || n_jobs < 1 || !voltages || !out) return MWAX_ERR_INVALID_ARG;
  mwax_tune_report rep;
  memset(&rep, 0, sizeof(rep));
  std::vector<mwax_job> base(jobs, jobs + n_jobs);
  // candidate 0: the batch plan's own default (all fields automatic); the
  // fused pair mode (4) fails to plan, and is skipped, unless every job allows it
  const std::vector<Cand> cands = {{0, 0, 0, 0, 0, 0}, {3, 0, -1, 0, 0, 0}, {4, 0, -1, 0, 0, 0},
                                   {1, 2, -1, 0, 0, 0}, {1, 2, 8, 0, 0, 0},  {2, 4, -1, 0, 0, 0},
                                   {2, 3, -1, 0, 0, 0}};
  Cand best{0, 0, 0, 0, 0, 0};
  double best_ms = -1.0;
  for (const Cand &c : cands) {
    std::vector<mwax_job> js = base;
    for (auto &j : js) {
      j.mma_shape = c.mma_shape;
      j.stages = c.stages;
      j.prefetch = c.prefetch;
    }
    const double ms = time_batch(js, voltages, out, stream, kTuneReps);
    if (ms > 0 && (best_ms < 0 || ms < 0.99 * best_ms)) {
      best_ms = ms;
      best = c;
    }
    if (&c == &cands[0]) rep.default_ms = ms;
    rep.candidates++;
  }
  if (best_ms < 0) return MWAX_ERR_UNSUPPORTED;
  for (int k = 0; k < n_jobs; ++k) {
    jobs[k].mma_shape = best.mma_shape;
    jobs[k].stages = best.stages;
    jobs[k].prefetch = best.prefetch;
    jobs[k].k_split = 0;
  }
  // then each job's time ranges per work item, one job at a time with the
  // others fixed (the automatic choice first; a split must be >1% faster)
  for (int k = 0; k < n_jobs; ++k) {
    for (const int ks : {1, 2, 4, 8}) {
      std::vector<mwax_job> js(jobs, jobs + n_jobs);
      js[k].k_split = ks;
      const double ms = time_batch(js, voltages, out, stream, kTuneReps);
      rep.candidates++;
      if (ms > 0 && ms < 0.99 * best_ms) {
        best_ms = ms;
        jobs[k].k_split = ks;
      }
    }
  }
  rep.best_ms = best_ms;
  if (report) *report = rep;
  return MWAX_OK;
}

}  // extern "C"
