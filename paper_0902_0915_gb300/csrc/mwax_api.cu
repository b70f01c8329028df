// mwax_api.cu -- plans, argument checks and the C entry points of libmwax.
//
// A plan fixes the shape of one or more correlation jobs, checks the int32
// bound, picks the tiling (samples per operand block, FP32 segment length,
// channel groups), allocates the operand scratch and the device status
// word, and launches the kernels on its stream:
//   tensor engine: per channel group, unpack (k_unpack.cu) then one
//                  persistent tcgen05 launch (k_correlate.cu);
//   plain engine:  one CUDA-core launch per channel (k_plain.cu).
// Batch plans run every job's unpack and then ONE persistent correlate
// launch over all jobs' work items, captured in a CUDA graph on first use.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "mwax_internal.h"

namespace mwax {
namespace {

constexpr int64_t kExactWindow = int64_t(1) << 24;  // integers exact in FP32
constexpr int64_t kDefaultScratchBudget = int64_t(8) << 30;
constexpr unsigned long long kDefaultTimeoutNs = 2000000000ull;  // 2 s per wait
constexpr int kMaxSplit = 8;  // time ranges per pair-mode work item

struct JobState {
  mwax_job job;
  int n_tiles = 0, n_pairs = 0, spb = 0, kb = 0, flush_blocks = 1, chan_group = 1;
  int k_split = 1;  // pair mode: time ranges per work item (resolved at plan time)
  int64_t n_bl = 0;
  int64_t op_chan_bytes = 0;  // operand bytes of one channel
  int64_t in_chan_bytes = 0;  // packed input bytes of one channel
  int64_t out_chan_bytes = 0;
  uint8_t *op = nullptr;  // batch plans: operand buffer for all channels of this job
};

}  // namespace
}  // namespace mwax

struct mwax_plan_s {
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  bool batch = false;
  int engine = MWAX_ENGINE_TENSOR;
  int sample_bits = 4;
  int kind = MWAX_KIND_EXACT;
  int stages = 2;
  int prefetch = 0;
  int mode = 0;  // correlate kernel: 0 narrow, 1 wide, 2 pair, 3 fused pair (mma_shape - 1)
  int withhold_seg = -1;
  int unpack_sms = 0;  // overlapped pipeline: SMs given to the persistent unpack (0: co-resident)
  unsigned long long timeout_ns = mwax::kDefaultTimeoutNs;
  std::vector<mwax::JobState> jobs;
  uint8_t *scratch = nullptr;  // single-job plans: operand buffer for one channel group
  uint8_t *scratch2 = nullptr;  // second buffer when unpack and correlate overlap
  int64_t scratch_bytes = 0;
  // overlapped pipeline: unpack of group g+1 (aux stream) runs beside the
  // persistent correlate of group g (plan stream)
  bool overlap = false;
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_start = nullptr, ev_unpacked[2] = {nullptr, nullptr}, ev_freed[2] = {nullptr, nullptr};
  int32_t *status = nullptr;
  // pair mode: device work lists; single-job plans hold the list of a full
  // channel group followed by that of the ragged last group, batch plans the
  // list of their one launch
  int4 *items = nullptr;
  int64_t n_items_full = 0, n_items_last = 0;
  // checked single segment (8-bit exact jobs longer than one exact segment):
  // the pair-mode pass accumulates each item in one FP32 segment, a check
  // lists the channels whose largest auto-correlation reached 2^24 (bad[0] =
  // count, bad[1..] = channels) and a narrow launch recomputes just those with
  // flush_blocks segments
  bool checked = false;
  int32_t *bad = nullptr;
  // [0]: channels recomputed since the caller last read the count; [1]: in
  // the current call (copied to recomp_host at the end of each call)
  unsigned long long *recomputed = nullptr;
  // adaptivity: after a call in which more than a quarter of the channels
  // had to be recomputed, the next kNarrowCalls calls run the narrow shape
  // directly, then the pair pass is tried again
  unsigned long long *recomp_host = nullptr;  // pinned
  cudaEvent_t ev_recomp = nullptr;
  bool recomp_pending = false;
  int narrow_calls_left = 0;
  // batch graphs: every job's unpack, then the one persistent correlate launch
  cudaGraphExec_t graph = nullptr, graph2 = nullptr;
  std::vector<const void *> graph_in;
  std::vector<void *> graph_out;
  // host path
  cudaStream_t h2d = nullptr, d2h = nullptr;
  uint8_t *stage_in[2] = {nullptr, nullptr};
  uint8_t *stage_out[2] = {nullptr, nullptr};
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr},
              ev_out[2] = {nullptr, nullptr};
  int64_t stage_in_bytes = 0, stage_out_bytes = 0;
  // kernel timing (events on the launching stream)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec {
    int kind;  // 0 unpack, 1 correlate, 2 host-to-device copy, 3 device-to-host copy
    cudaEvent_t start, stop;
    int64_t bytes;
  };
  std::vector<Rec> recs;

};

namespace mwax {
namespace {

// Device allocation of plan buffers.  Test hook: with MWAX_TEST_FAIL_ALLOC set
// to a non-zero value, plan allocations report cudaErrorMemoryAllocation
// without allocating (read on every call), so the OOM paths can be tested
// without exhausting a device.
cudaError_t plan_alloc(void **ptr, size_t bytes) {
  const char *f = getenv("MWAX_TEST_FAIL_ALLOC");
  if (f && *f && strcmp(f, "0") != 0) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(ptr, bytes);
}

mwax_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MWAX_OK;
  if (e == cudaErrorMemoryAllocation) return MWAX_ERR_OOM;
  return MWAX_ERR_CUDA;
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

mwax_status check_job(const mwax_job &j) {
  if (j.n_inputs < 1 || j.n_chan < 1 || j.n_time < 1) return MWAX_ERR_INVALID_ARG;
  if (j.sample_bits != 4 && j.sample_bits != 8) return MWAX_ERR_INVALID_ARG;
  if (j.kind != MWAX_KIND_EXACT && j.kind != MWAX_KIND_FP16) return MWAX_ERR_INVALID_ARG;
  if (j.engine != MWAX_ENGINE_TENSOR && j.engine != MWAX_ENGINE_PLAIN) return MWAX_ERR_INVALID_ARG;
  if (j.flush_blocks < 0 || j.chan_group < 0) return MWAX_ERR_INVALID_ARG;
  if (j.mma_shape < 0 || j.mma_shape > 4) return MWAX_ERR_INVALID_ARG;
  if (j.pipeline < 0 || j.pipeline > 2) return MWAX_ERR_INVALID_ARG;
  if (j.stages < 0 || j.stages == 1 ||
      j.stages > correlate_tc_max_stages(j.mma_shape > 0 ? j.mma_shape - 1 : 0))
    return MWAX_ERR_INVALID_ARG;
  if (j.prefetch < -1 || j.prefetch > 64) return MWAX_ERR_INVALID_ARG;
  if (j.timeout_ms < 0 || j.test_fault < 0 || j.unpack_sms < 0) return MWAX_ERR_INVALID_ARG;
  if (j.k_split < 0 || j.k_split > kMaxSplit) return MWAX_ERR_INVALID_ARG;
  if (j.kind == MWAX_KIND_FP16 && (j.sample_bits != 8 || j.engine != MWAX_ENGINE_TENSOR))
    return MWAX_ERR_UNSUPPORTED;
  if (j.n_inputs > 65536) return MWAX_ERR_UNSUPPORTED;
  if (j.kind == MWAX_KIND_EXACT && (int64_t)j.n_time > mwax_max_n_time(j.sample_bits))
    return MWAX_ERR_OVERFLOW_BOUND;
  return MWAX_OK;
}

void derive(JobState &s) {
  const mwax_job &j = s.job;
  s.n_tiles = (j.n_inputs + kTile - 1) / kTile;
  s.n_pairs = s.n_tiles * (s.n_tiles + 1) / 2;
  s.spb = samples_per_block(j.sample_bits);
  s.kb = (j.n_time + s.spb - 1) / s.spb;
  const int64_t m = sample_max(j.sample_bits);
  // largest segment whose partial sums provably stay inside the exact window
  const int64_t per_block = (int64_t)s.spb * 2 * m * m;
  int64_t f = kExactWindow / per_block;
  if (j.kind == MWAX_KIND_FP16) f = s.kb;
  if (j.flush_blocks > 0) f = j.flush_blocks;
  s.flush_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(f, s.kb));
  s.n_bl = (int64_t)j.n_inputs * (j.n_inputs + 1) / 2;
  s.op_chan_bytes = (int64_t)s.n_tiles * kTile * s.kb * kRowBytes;
  s.in_chan_bytes = (int64_t)j.n_time * j.n_inputs * bytes_per_sample(j.sample_bits);
  s.out_chan_bytes = s.n_bl * 8;
  int64_t g = j.chan_group > 0 ? j.chan_group : kDefaultScratchBudget / s.op_chan_bytes;
  s.chan_group = (int)std::max<int64_t>(1, std::min<int64_t>(g, j.n_chan));
}

mwax_status init_device(mwax_plan_s *p, cudaStream_t stream) {
  if (cudaGetDevice(&p->device) != cudaSuccess) return MWAX_ERR_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, p->device) != cudaSuccess) return MWAX_ERR_CUDA;
  if (prop.major != 10 || prop.minor != 3) return MWAX_ERR_UNSUPPORTED;
  p->sm_count = prop.multiProcessorCount;
  p->stream = stream;
  if (const char *e = getenv("MWAX_TIMEOUT_MS")) {
    long v = atol(e);
    if (v > 0) p->timeout_ns = (unsigned long long)v * 1000000ull;
  }
  cudaError_t e = cudaMalloc(&p->status, sizeof(int32_t));
  if (e != cudaSuccess) return cuda_status(e);
  return cuda_status(cudaMemsetAsync(p->status, 0, sizeof(int32_t), stream));
}

// Event pair around one launch when timing is on.
struct TimedLaunch {
  mwax_plan_s *p;
  int kind, start = -1;
  cudaStream_t st;
  TimedLaunch(mwax_plan_s *plan, int k, cudaStream_t s) : p(plan), kind(k), st(s) {
    if (!p->timing) return;
    start = next_event();
    if (start >= 0) cudaEventRecord(p->ev_pool[start], st);
  }
  int next_event() {
    const int used = (int)p->recs.size() * 2 + (start >= 0 ? 1 : 0);
    while ((int)p->ev_pool.size() <= used) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      p->ev_pool.push_back(e);
    }
    return used;
  }
  void done(int64_t bytes = 0) {
    if (start < 0) return;
    const int stop = next_event();
    if (stop < 0) return;
    cudaEventRecord(p->ev_pool[stop], st);
    p->recs.push_back({kind, p->ev_pool[start], p->ev_pool[stop], bytes});
    start = -1;
  }
};

TcJob tc_job(const JobState &s, const uint8_t *op, void *out_c0, int nc) {
  TcJob tj;
  tj.op = op;
  tj.out = out_c0;
  tj.n_inputs = s.job.n_inputs;
  tj.n_tiles = s.n_tiles;
  tj.n_pairs = s.n_pairs;
  tj.kb = s.kb;
  tj.flush_blocks = s.flush_blocks;
  tj.n_chan = nc;
  tj.n_time = s.job.n_time;
  tj.n_bl = s.n_bl;
  tj.k_split = s.k_split;
  return tj;
}

// The time ranges per pair-mode work item of a job: the job's own k_split,
// checked, or automatic -- 1 unless the launch's items (base_items) fill at
// most half the SMs, then the largest k <= 8 with base_items * k <= SMs and
// k <= time blocks / 2.  -1: a k_split the job cannot take.
int resolve_split(const mwax_job &job, int mode, int kb, int64_t base_items, int sm_count) {
  const bool can = (mode == 2 || mode == 3) && job.kind == MWAX_KIND_EXACT;
  if (job.k_split > 0) {
    if (job.k_split == 1) return 1;
    return can && 2 * job.k_split <= kb ? job.k_split : -1;
  }
  if (!can || base_items < 1 || base_items * 2 > sm_count) return 1;
  int k = (int)std::min<int64_t>(kMaxSplit, sm_count / base_items);
  k = std::min(k, kb / 2);
  return std::max(k, 1);
}

// Fused pair mode chosen automatically up to this many 128-input tiles: each
// operand tile is converted once per work item that reads it (about n_tiles /
// 2 + 1 times per channel and time block), against one write and one read of
// the unpacked operands through HBM without the fusion.
constexpr int kFusedAutoTiles = 2;

// Kernel mode for a job's mma_shape (0 = auto: the fused pair mode for small
// 4-bit exact arrays that allow it (fused_ok, at most kFusedAutoTiles tiles),
// else the pair mode where every job integrates in one exact segment, else
// narrow); -1 when an explicit pair or fused pair request cannot be served.
int choose_mode(int mma_shape, const std::vector<TcJob> &tj, bool fused_ok) {
  const bool pair_ok = pair_mode_supported(tj.data(), (int)tj.size());
  if (mma_shape == 4) return pair_ok && fused_ok ? 3 : -1;
  if (mma_shape == 3) return pair_ok ? 2 : -1;
  if (mma_shape == 1 || mma_shape == 2) return mma_shape - 1;
  bool small = true;
  for (const TcJob &j : tj) small = small && j.n_tiles <= kFusedAutoTiles;
  if (pair_ok && fused_ok && small) return 3;
  return pair_ok ? 2 : 0;
}

bool pair_like(int mode) { return mode == 2 || mode == 3; }

// Build the pair-mode work lists (a and, if non-empty, b after it) and copy
// them to a device buffer owned by the plan.
cudaError_t upload_items(mwax_plan_s *p, const std::vector<TcJob> &a, const std::vector<TcJob> &b) {
  std::vector<int4> la, lb;
  build_pair_items(a.data(), (int)a.size(), la);
  if (!b.empty()) build_pair_items(b.data(), (int)b.size(), lb);
  p->n_items_full = (int64_t)la.size();
  p->n_items_last = (int64_t)lb.size();
  la.insert(la.end(), lb.begin(), lb.end());
  if (la.empty()) return cudaSuccess;
  cudaError_t e = plan_alloc(reinterpret_cast<void **>(&p->items), la.size() * sizeof(int4));
  if (e == cudaSuccess)
    e = cudaMemcpy(p->items, la.data(), la.size() * sizeof(int4), cudaMemcpyHostToDevice);
  return e;
}

TcLaunch launch_cfg(const mwax_plan_s *p) {
  TcLaunch c;
  c.sample_bits = p->sample_bits;
  c.kind = p->kind;
  // with the overlapped pipeline the correlate leaves unpack_sms SMs to the unpack
  c.grid = p->overlap ? p->sm_count - p->unpack_sms : p->sm_count;
  c.stages = p->stages;
  c.prefetch = p->prefetch;
  c.mode = p->mode;
  c.withhold_seg = p->withhold_seg;
  c.status = p->status;
  c.timeout_ns = p->timeout_ns;
  return c;
}

// Unpack variant: automatic = the TMA tile kernel (5) for shapes that allow it
// (and whose sample buffer starts on a 16-byte boundary, which TMA needs),
// else the full-line kernel (4-bit) or the shared-memory transpose; the
// environment variable MWAX_UNPACK = 1 (shared-memory transpose) or 2
// (full-line) forces a fallback, for comparisons.
bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int unpack_choice(const JobState &s, const void *volt) {
  static const int env = [] {
    const char *e = getenv("MWAX_UNPACK");
    return e ? atoi(e) : 0;
  }();
  const bool aligned = (reinterpret_cast<uintptr_t>(volt) & 15u) == 0;
  const bool tile_ok = unpack_tile_supported(s.job.sample_bits, s.job.n_inputs) && aligned;
  if (env == 1 || env == 2) return env;
  return tile_ok ? 5 : 0;
}

// small-footprint unpack: CTAs per SM when it runs alone
constexpr int kTileCtasPerSm = 6;

mwax_status unpack_group(mwax_plan_s *p, const JobState &s, const uint8_t *volt, int64_t c0, int nc,
                         uint8_t *op, int ctas, cudaStream_t st) {
  TimedLaunch tu(p, 0, st);
  cudaError_t e;
  const int v = unpack_choice(s, volt);
  if (p->overlap && p->unpack_sms == 0)  // one tile CTA beside the correlate on every SM
    e = launch_unpack_tile(volt, s.job.sample_bits, s.job.n_inputs, s.job.n_time, s.n_tiles, s.kb,
                           c0, nc, op, p->sm_count, p->status, p->timeout_ns, st);
  else if (ctas > 0)  // overlapped on `ctas` SMs set aside
    e = launch_unpack_persistent(volt, s.job.sample_bits, s.job.n_inputs, s.job.n_time, s.n_tiles,
                                 s.kb, c0, nc, op, ctas, st);
  else if (v == 5)
    e = launch_unpack_tile(volt, s.job.sample_bits, s.job.n_inputs, s.job.n_time, s.n_tiles, s.kb,
                           c0, nc, op, p->sm_count * kTileCtasPerSm, p->status, p->timeout_ns, st);
  else
    e = launch_unpack(volt, s.job.sample_bits, s.job.n_inputs, s.job.n_time, s.n_tiles, s.kb, c0,
                      nc, op, v, st);
  tu.done();
  return cuda_status(e);
}

constexpr int kNarrowCalls = 8;

// Start of a call of a checked plan: true = pair pass + check, false = this
// call runs the narrow shape (see mwax_plan_s::narrow_calls_left).
bool checked_call_uses_pair(mwax_plan_s *p) {
  if (p->recomp_pending && cudaEventQuery(p->ev_recomp) == cudaSuccess) {
    p->recomp_pending = false;
    if (*p->recomp_host * 4 > (unsigned long long)p->jobs[0].job.n_chan)
      p->narrow_calls_left = kNarrowCalls;
  }
  if (p->narrow_calls_left > 0) {
    --p->narrow_calls_left;
    return false;
  }
  return true;
}

// End of a call of a checked plan that ran the pair pass: publish this
// call's recompute count to the host without blocking.
cudaError_t checked_call_done(mwax_plan_s *p, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(p->recomp_host, p->recomputed + 1, sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->recomputed + 1, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaEventRecord(p->ev_recomp, st);
  if (e == cudaSuccess) p->recomp_pending = true;
  return e;
}

mwax_status correlate_group(mwax_plan_s *p, const JobState &s, const uint8_t *op, int nc,
                            void *out_c0, cudaStream_t st, bool use_pair = true) {
  TcJob tj = tc_job(s, op, out_c0, nc);
  TcLaunch cfg = launch_cfg(p);
  if (p->mode == 2 && !use_pair) {  // a checked plan's narrow call (never fused)
    cfg.mode = 0;
    cfg.stages = correlate_tc_max_stages(0);
    TimedLaunch tn(p, 1, st);
    cudaError_t e = launch_correlate_tc(&tj, 1, cfg, st);
    tn.done();
    return cuda_status(e);
  }
  if (pair_like(p->mode)) {
    const bool full = nc == s.chan_group;
    cfg.items = full ? p->items : p->items + p->n_items_full;
    cfg.n_items = full ? p->n_items_full : p->n_items_last;
    if (p->checked) tj.flush_blocks = s.kb;  // one optimistic segment per item
  }
  TimedLaunch tc(p, 1, st);
  cudaError_t e = cudaSuccess;
  if (pair_like(p->mode) && s.k_split > 1)  // the time ranges' partial sums are added into it
    e = cudaMemsetAsync(out_c0, 0, (size_t)(nc * s.out_chan_bytes), st);
  if (e == cudaSuccess) e = launch_correlate_tc(&tj, 1, cfg, st);
  if (e == cudaSuccess && p->checked) {
    e = launch_exact_check(reinterpret_cast<const int32_t *>(out_c0), s.n_bl, s.job.n_inputs, nc,
                           p->bad, p->recomputed, st);
    if (e == cudaSuccess) {
      // the flagged channels again, narrow shape, exact segments (an empty
      // list makes every CTA return at once)
      TcJob fj = tc_job(s, op, out_c0, nc);
      TcLaunch fc = launch_cfg(p);
      fc.mode = 0;
      fc.stages = correlate_tc_max_stages(0);
      fc.withhold_seg = -1;
      fc.chan_map = p->bad + 1;
      fc.n_chan_dev = p->bad;
      e = launch_correlate_tc(&fj, 1, fc, st);
    }
  }
  tc.done();
  return cuda_status(e);
}

// Channels [c0, c0+nc) of a single-job tensor plan, one after the other on
// `st`: unpack into the scratch, then one persistent correlate launch (the
// fused pair mode reads the packed samples itself: the launch only).
mwax_status run_group(mwax_plan_s *p, const JobState &s, const uint8_t *volt, int64_t c0, int nc,
                      void *out_c0, cudaStream_t st, bool use_pair = true) {
  if (p->mode == 3) return correlate_group(p, s, volt + c0 * s.in_chan_bytes, nc, out_c0, st, use_pair);
  mwax_status r = unpack_group(p, s, volt, c0, nc, p->scratch, 0, st);
  if (r != MWAX_OK) return r;
  return correlate_group(p, s, p->scratch, nc, out_c0, st, use_pair);
}

mwax_status correlate_device(mwax_plan_s *p, const uint8_t *volt, void *out, cudaStream_t st) {
  const JobState &s = p->jobs[0];
  if (p->engine == MWAX_ENGINE_PLAIN) {
    for (int c = 0; c < s.job.n_chan; ++c) {
      TimedLaunch tl(p, 1, st);
      cudaError_t e = launch_plain_channel(volt + (int64_t)c * s.in_chan_bytes, s.job.sample_bits,
                                           s.job.n_inputs, s.job.n_time,
                                           reinterpret_cast<int32_t *>(out) + (int64_t)c * s.n_bl * 2,
                                           p->sm_count, st);
      tl.done();
      if (e != cudaSuccess) return cuda_status(e);
    }
    return MWAX_OK;
  }
  uint8_t *out8 = reinterpret_cast<uint8_t *>(out);
  const bool use_pair = !p->checked || checked_call_uses_pair(p);
  if (!p->overlap) {
    for (int64_t c0 = 0; c0 < s.job.n_chan; c0 += s.chan_group) {
      const int nc = (int)std::min<int64_t>(s.chan_group, s.job.n_chan - c0);
      mwax_status r = run_group(p, s, volt, c0, nc, out8 + c0 * s.out_chan_bytes, st, use_pair);
      if (r != MWAX_OK) return r;
    }
    return p->checked && use_pair ? cuda_status(checked_call_done(p, st)) : MWAX_OK;
  }
  // Overlapped: the unpack of group g+1 runs on the aux stream into the other
  // scratch buffer while group g correlates: either one small unpack CTA per
  // SM beside the persistent correlate CTA (unpack_sms == 0; it uses the DRAM
  // bandwidth the correlate leaves idle), or a persistent unpack on
  // unpack_sms SMs with the correlate on the rest.
  uint8_t *buf[2] = {p->scratch, p->scratch2};
  cudaError_t e = cudaEventRecord(p->ev_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->aux, p->ev_start, 0);
  if (e != cudaSuccess) return cuda_status(e);
  int64_t g = 0;
  for (int64_t c0 = 0; c0 < s.job.n_chan; c0 += s.chan_group, ++g) {
    const int k = (int)(g & 1);
    const int nc = (int)std::min<int64_t>(s.chan_group, s.job.n_chan - c0);
    if (g >= 2 && (e = cudaStreamWaitEvent(p->aux, p->ev_freed[k], 0)) != cudaSuccess)
      return cuda_status(e);
    mwax_status r = unpack_group(p, s, volt, c0, nc, buf[k], p->unpack_sms, p->aux);
    if (r != MWAX_OK) return r;
    if ((e = cudaEventRecord(p->ev_unpacked[k], p->aux)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaStreamWaitEvent(st, p->ev_unpacked[k], 0)) != cudaSuccess) return cuda_status(e);
    r = correlate_group(p, s, buf[k], nc, out8 + c0 * s.out_chan_bytes, st, use_pair);
    if (r != MWAX_OK) return r;
    if ((e = cudaEventRecord(p->ev_freed[k], st)) != cudaSuccess) return cuda_status(e);
  }
  return p->checked && use_pair ? cuda_status(checked_call_done(p, st)) : MWAX_OK;
}

void free_plan(mwax_plan_s *p) {
  if (!p) return;
  if (p->graph) cudaGraphExecDestroy(p->graph);
  if (p->graph2) cudaGraphExecDestroy(p->graph2);
  for (auto &s : p->jobs)
    if (s.op) cudaFree(s.op);
  if (p->scratch) cudaFree(p->scratch);
  if (p->scratch2) cudaFree(p->scratch2);
  if (p->status) cudaFree(p->status);
  if (p->items) cudaFree(p->items);
  if (p->bad) cudaFree(p->bad);
  if (p->recomputed) cudaFree(p->recomputed);
  if (p->recomp_host) cudaFreeHost(p->recomp_host);
  if (p->ev_recomp) cudaEventDestroy(p->ev_recomp);
  if (p->aux) cudaStreamDestroy(p->aux);
  if (p->ev_start) cudaEventDestroy(p->ev_start);
  for (int k = 0; k < 2; ++k) {
    if (p->stage_in[k]) cudaFree(p->stage_in[k]);
    if (p->stage_out[k]) cudaFree(p->stage_out[k]);
    if (p->ev_in[k]) cudaEventDestroy(p->ev_in[k]);
    if (p->ev_comp[k]) cudaEventDestroy(p->ev_comp[k]);
    if (p->ev_out[k]) cudaEventDestroy(p->ev_out[k]);
    if (p->ev_unpacked[k]) cudaEventDestroy(p->ev_unpacked[k]);
    if (p->ev_freed[k]) cudaEventDestroy(p->ev_freed[k]);
  }
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);

  if (p->h2d) cudaStreamDestroy(p->h2d);
  if (p->d2h) cudaStreamDestroy(p->d2h);
  delete p;
}

}  // namespace
}  // namespace mwax

using namespace mwax;

extern "C" {

const char *mwax_status_string(mwax_status s) {
  switch (s) {
    case MWAX_OK: return "ok";
    case MWAX_ERR_INVALID_ARG: return "invalid argument";
    case MWAX_ERR_SHAPE_MISMATCH: return "shape differs from the plan";
    case MWAX_ERR_OVERFLOW_BOUND: return "n_time * 2 * max^2 exceeds the int32 range";
    case MWAX_ERR_UNSUPPORTED: return "unsupported device or option";
    case MWAX_ERR_OOM: return "device allocation failed";
    case MWAX_ERR_CUDA: return "CUDA runtime error";
    case MWAX_ERR_TIMEOUT: return "a bounded device wait timed out";
  }
  return "unknown status";
}

int64_t mwax_n_baselines(int n_inputs) {
  if (n_inputs < 0) return -1;
  return (int64_t)n_inputs * (n_inputs + 1) / 2;
}

int64_t mwax_baseline_index(int i, int j) {
  if (j < 0 || i < j) return -1;
  return (int64_t)i * (i + 1) / 2 + j;
}

mwax_status mwax_baseline_pair(int64_t b, int *i, int *j) {
  if (b < 0 || !i || !j) return MWAX_ERR_INVALID_ARG;
  // largest i with i(i+1)/2 <= b, by bisection on exact integers
  int64_t lo = 0, hi = 3037000499LL;  // hi(hi+1)/2 fits int64
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo + 1) / 2;
    if (mid * (mid + 1) / 2 <= b) lo = mid;
    else hi = mid - 1;
  }
  if (lo > 2147483647LL) return MWAX_ERR_INVALID_ARG;
  *i = (int)lo;
  *j = (int)(b - lo * (lo + 1) / 2);
  return MWAX_OK;
}

int64_t mwax_max_n_time(int sample_bits) {
  if (sample_bits != 4 && sample_bits != 8) return -1;
  const int64_t m = sample_max(sample_bits);
  return (int64_t)2147483647 / (2 * m * m);
}

mwax_status mwax_plan(mwax_plan_t *plan, const mwax_job *job, cudaStream_t stream) {
  NvtxRange nvtx_("mwax_plan");
  if (!plan) return MWAX_ERR_INVALID_ARG;
  *plan = nullptr;
  if (!job) return MWAX_ERR_INVALID_ARG;
  mwax_status r = check_job(*job);
  if (r != MWAX_OK) return r;
  mwax_plan_s *p = new (std::nothrow) mwax_plan_s();
  if (!p) return MWAX_ERR_OOM;
  r = init_device(p, stream);
  if (r != MWAX_OK) {
    free_plan(p);
    return r;
  }
  mwax_job tuned = *job;
  apply_tune_cache(&tuned);
  job = &tuned;
  JobState s;
  s.job = *job;
  derive(s);
  p->jobs.push_back(s);
  p->engine = job->engine;
  p->sample_bits = job->sample_bits;
  p->kind = job->kind;
  if (job->prefetch != 0) p->prefetch = job->prefetch < 0 ? 0 : job->prefetch;
  if (job->timeout_ms > 0) p->timeout_ns = (unsigned long long)job->timeout_ms * 1000000ull;
  p->withhold_seg = job->test_fault - 1;
  if (p->engine == MWAX_ENGINE_TENSOR) {
    std::vector<TcJob> full = {tc_job(s, nullptr, nullptr, s.chan_group)};
    // exact jobs longer than one exact segment, shape and segments left to the
    // plan: one checked optimistic segment per pair-mode item
    p->checked = job->kind == MWAX_KIND_EXACT && job->flush_blocks == 0 &&
                 (job->mma_shape == 0 || job->mma_shape == 3) && s.flush_blocks < s.kb &&
                 s.n_tiles <= 255;
    if (p->checked) full[0].flush_blocks = s.kb;
    const bool fused_ok = !p->checked && fused_pair_supported(full.data(), 1, job->sample_bits, job->kind);
    p->mode = choose_mode(job->mma_shape, full, fused_ok);
    if (p->mode < 0) {
      free_plan(p);
      return MWAX_ERR_UNSUPPORTED;
    }
    // time ranges per pair-mode item, from the items of one channel group
    std::vector<int4> base;
    if (pair_like(p->mode)) build_pair_items(full.data(), 1, base);
    const int split = resolve_split(*job, p->mode, s.kb, (int64_t)base.size(), p->sm_count);
    if (split < 0) {
      free_plan(p);
      return MWAX_ERR_UNSUPPORTED;
    }
    s.k_split = p->jobs[0].k_split = full[0].k_split = split;
    p->stages = job->stages > 0 ? job->stages : correlate_tc_max_stages(p->mode);
    if (p->stages > correlate_tc_max_stages(p->mode)) {
      free_plan(p);
      return MWAX_ERR_INVALID_ARG;
    }
    const int64_t one = p->mode == 3 ? 0 : s.op_chan_bytes * s.chan_group;  // fused: no operands
    const bool even = s.job.sample_bits == 8 ? s.job.n_inputs % 2 == 0 : true;
    // unpack_sms 0: the small unpack CTA runs beside the correlate on every SM
    // where the shape allows it, else 20 SMs are set aside for the unpack
    // (pair mode fills the shared memory: no room for a co-resident unpack CTA)
    p->unpack_sms = job->unpack_sms > 0 ? job->unpack_sms
                    : unpack_tile_supported(s.job.sample_bits, s.job.n_inputs) && p->mode != 2
                        ? 0
                        : 20;
    p->overlap = job->pipeline == 2 && s.chan_group < s.job.n_chan && even &&
                 p->unpack_sms < p->sm_count && p->mode != 3;
    p->scratch_bytes = one * (p->overlap ? 2 : 1);
    cudaError_t e = cudaSuccess;
    if (one > 0) {
      e = plan_alloc(reinterpret_cast<void **>(&p->scratch), (size_t)one);
      if (e == cudaSuccess) e = cudaMemsetAsync(p->scratch, 0, (size_t)one, stream);
    }
    if (e == cudaSuccess && p->overlap) {
      e = plan_alloc(reinterpret_cast<void **>(&p->scratch2), (size_t)one);
      if (e == cudaSuccess) e = cudaMemsetAsync(p->scratch2, 0, (size_t)one, stream);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming);
      for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&p->ev_unpacked[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_freed[k], cudaEventDisableTiming);
      }
    }
    if (e == cudaSuccess && pair_like(p->mode)) {
      const int last = (int)(s.job.n_chan % s.chan_group);
      std::vector<TcJob> tail;
      if (last) {
        tail.push_back(tc_job(s, nullptr, nullptr, last));
        tail[0].flush_blocks = full[0].flush_blocks;
      }
      e = upload_items(p, full, tail);
    }
    if (e == cudaSuccess && p->checked) {
      e = plan_alloc(reinterpret_cast<void **>(&p->bad), (size_t)(s.chan_group + 1) * sizeof(int32_t));
      if (e == cudaSuccess)
        e = plan_alloc(reinterpret_cast<void **>(&p->recomputed), 2 * sizeof(unsigned long long));
      if (e == cudaSuccess)
        e = cudaMemsetAsync(p->recomputed, 0, 2 * sizeof(unsigned long long), stream);
      if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void **>(&p->recomp_host), sizeof(unsigned long long),
                          cudaHostAllocDefault);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_recomp, cudaEventDisableTiming);
      if (e == cudaSuccess) e = correlate_tc_prepare(p->sample_bits, p->kind, correlate_tc_max_stages(0), 0);
    }
    if (e == cudaSuccess) e = correlate_tc_prepare(p->sample_bits, p->kind, p->stages, p->mode);
    if (e != cudaSuccess) {
      free_plan(p);
      return cuda_status(e);
    }
  }
  *plan = p;
  return MWAX_OK;
}

mwax_status mwax_plan_batch(mwax_plan_t *plan, const mwax_job *jobs, int n_jobs,
                            cudaStream_t stream) {
  NvtxRange nvtx_("mwax_plan_batch");
  if (!plan) return MWAX_ERR_INVALID_ARG;
  *plan = nullptr;
  if (!jobs || n_jobs < 1 || n_jobs > MWAX_MAX_JOBS) return MWAX_ERR_INVALID_ARG;
  for (int k = 0; k < n_jobs; ++k) {
    mwax_status r = check_job(jobs[k]);
    if (r != MWAX_OK) return r;
    if (jobs[k].engine != MWAX_ENGINE_TENSOR) return MWAX_ERR_UNSUPPORTED;
    if (jobs[k].sample_bits != jobs[0].sample_bits || jobs[k].kind != jobs[0].kind)
      return MWAX_ERR_UNSUPPORTED;  // one kernel instantiation per launch
  }
  mwax_plan_s *p = new (std::nothrow) mwax_plan_s();
  if (!p) return MWAX_ERR_OOM;
  mwax_status r = init_device(p, stream);
  if (r != MWAX_OK) {
    free_plan(p);
    return r;
  }
  p->batch = true;
  p->sample_bits = jobs[0].sample_bits;
  p->kind = jobs[0].kind;
  if (jobs[0].prefetch != 0) p->prefetch = jobs[0].prefetch < 0 ? 0 : jobs[0].prefetch;
  for (int k = 0; k < n_jobs; ++k) {
    JobState s;
    s.job = jobs[k];
    derive(s);
    p->jobs.push_back(s);
  }
  std::vector<TcJob> tj;
  for (const JobState &s : p->jobs) tj.push_back(tc_job(s, nullptr, nullptr, s.job.n_chan));
  // the fused pair mode where every job allows it (the correlate then reads
  // each job's voltages itself: no unpack graph, no operand buffers)
  const bool fused_ok = fused_pair_supported(tj.data(), n_jobs, jobs[0].sample_bits, jobs[0].kind);
  p->mode = choose_mode(jobs[0].mma_shape, tj, fused_ok);
  if (p->mode < 0) {
    free_plan(p);
    return MWAX_ERR_UNSUPPORTED;
  }
  for (int k = 0; k < n_jobs && p->mode != 3; ++k) {
    JobState &s = p->jobs[k];
    cudaError_t e = plan_alloc(reinterpret_cast<void **>(&s.op), (size_t)(s.op_chan_bytes * s.job.n_chan));
    if (e == cudaSuccess)
      e = cudaMemsetAsync(s.op, 0, (size_t)(s.op_chan_bytes * s.job.n_chan), stream);
    p->scratch_bytes += s.op_chan_bytes * s.job.n_chan;
    tj[k].op = s.op;
    if (e != cudaSuccess) {
      free_plan(p);
      return cuda_status(e);
    }
  }
  // each job's time ranges per pair-mode item, from the launch's items
  std::vector<int4> base;
  if (pair_like(p->mode)) build_pair_items(tj.data(), (int)tj.size(), base);
  for (int k = 0; k < n_jobs; ++k) {
    const int split = resolve_split(jobs[k], p->mode, p->jobs[k].kb, (int64_t)base.size(), p->sm_count);
    if (split < 0) {
      free_plan(p);
      return MWAX_ERR_UNSUPPORTED;
    }
    p->jobs[k].k_split = tj[k].k_split = split;
  }
  p->stages = jobs[0].stages > 0 ? jobs[0].stages : correlate_tc_max_stages(p->mode);
  cudaError_t e = p->stages <= correlate_tc_max_stages(p->mode) ? cudaSuccess : cudaErrorInvalidValue;
  if (e == cudaSuccess && pair_like(p->mode)) e = upload_items(p, tj, {});
  if (e == cudaSuccess) e = correlate_tc_prepare(p->sample_bits, p->kind, p->stages, p->mode);
  if (e != cudaSuccess) {
    free_plan(p);
    return e == cudaErrorInvalidValue ? MWAX_ERR_INVALID_ARG : cuda_status(e);
  }
  *plan = p;
  return MWAX_OK;
}

mwax_status mwax_destroy(mwax_plan_t plan) {
  if (!plan) return MWAX_OK;
  const cudaError_t e = cudaStreamSynchronize(plan->stream);
  free_plan(plan);
  return cuda_status(e);
}

mwax_status mwax_plan_get_info(mwax_plan_t plan, mwax_plan_info *info) {
  if (!plan || !info) return MWAX_ERR_INVALID_ARG;
  memset(info, 0, sizeof(*info));
  const JobState &s = plan->jobs[0];
  info->n_jobs = (int32_t)plan->jobs.size();
  info->engine = plan->engine;
  info->samples_per_block = s.spb;
  info->flush_blocks = s.flush_blocks;
  info->chan_group = plan->batch ? s.job.n_chan : s.chan_group;
  info->grid = plan->sm_count;
  info->stages = plan->stages;
  info->mma_shape = plan->mode + 1;
  info->checked_segment = plan->checked ? 1 : 0;
  info->k_split = 1;
  for (const auto &j : plan->jobs) info->k_split = std::max(info->k_split, j.k_split);
  info->pipeline = plan->overlap ? 2 : 1;
  info->prefetch = plan->prefetch;
  info->scratch_bytes = plan->scratch_bytes + plan->stage_in_bytes * 2 + plan->stage_out_bytes * 2;
  int64_t items = 0;
  if (pair_like(plan->mode) && plan->batch) {
    items = plan->n_items_full;
  } else if (pair_like(plan->mode)) {
    items = (s.job.n_chan / s.chan_group) * plan->n_items_full + plan->n_items_last;
  } else {
    for (const auto &j : plan->jobs) items += (int64_t)j.job.n_chan * j.n_pairs;
  }
  info->work_items = items;
  return MWAX_OK;
}

mwax_status mwax_plan_status(mwax_plan_t plan) {
  if (!plan) return MWAX_ERR_INVALID_ARG;
  int32_t v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, plan->status, sizeof(v), cudaMemcpyDeviceToHost, plan->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(plan->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(plan->status, 0, sizeof(int32_t), plan->stream);
  if (e != cudaSuccess) return cuda_status(e);
  return (mwax_status)v;
}

mwax_status mwax_plan_recomputed_channels(mwax_plan_t plan, int64_t *n_channels) {
  if (!plan || !n_channels) return MWAX_ERR_INVALID_ARG;
  *n_channels = 0;
  if (!plan->recomputed) return MWAX_OK;
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, plan->recomputed, sizeof(v), cudaMemcpyDeviceToHost, plan->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(plan->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(plan->recomputed, 0, sizeof(v), plan->stream);
  if (e != cudaSuccess) return cuda_status(e);
  *n_channels = (int64_t)v;
  return MWAX_OK;
}

mwax_status mwax_correlate(mwax_plan_t plan, const void *voltages, int n_inputs, int n_chan,
                           int n_time, void *out) {
  NvtxRange nvtx_("mwax_correlate");
  if (!plan || plan->batch) return MWAX_ERR_INVALID_ARG;
  const JobState &s = plan->jobs[0];
  if (n_inputs != s.job.n_inputs || n_chan != s.job.n_chan || n_time != s.job.n_time)
    return MWAX_ERR_SHAPE_MISMATCH;
  if (!is_device_ptr(voltages) || !is_device_ptr(out)) return MWAX_ERR_INVALID_ARG;
  if (!aligned16(voltages) || !aligned16(out)) return MWAX_ERR_INVALID_ARG;
  return correlate_device(plan, reinterpret_cast<const uint8_t *>(voltages), out, plan->stream);
}

mwax_status mwax_correlate_batch(mwax_plan_t plan, const void *const *voltages, void *const *out) {
  NvtxRange nvtx_("mwax_correlate_batch");
  if (!plan || !plan->batch || !voltages || !out) return MWAX_ERR_INVALID_ARG;
  const int nj = (int)plan->jobs.size();
  for (int k = 0; k < nj; ++k)
    if (!is_device_ptr(voltages[k]) || !is_device_ptr(out[k]) || !aligned16(voltages[k]) ||
        !aligned16(out[k]))
      return MWAX_ERR_INVALID_ARG;
  const bool fused = plan->mode == 3;  // no unpack graph: the correlate reads the voltages
  bool same = (fused || plan->graph != nullptr) && plan->graph2 != nullptr;
  for (int k = 0; k < nj && same; ++k)
    same = plan->graph_in[k] == voltages[k] && plan->graph_out[k] == out[k];
  if (!same) {
    for (cudaGraphExec_t *ge : {&plan->graph, &plan->graph2})
      if (*ge) {
        cudaGraphExecDestroy(*ge);
        *ge = nullptr;
      }
    std::vector<TcJob> tj(nj);
    for (int k = 0; k < nj; ++k)
      tj[k] = tc_job(plan->jobs[k],
                     fused ? reinterpret_cast<const uint8_t *>(voltages[k]) : plan->jobs[k].op, out[k],
                     plan->jobs[k].job.n_chan);
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_status(e);
    // graph 1: every job's unpack (none in the fused pair mode); graph 2: one
    // persistent launch over all items
    for (int part = fused ? 1 : 0; part < 2 && e == cudaSuccess; ++part) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (part == 0) {
        for (int k = 0; k < nj && e == cudaSuccess; ++k) {
          const JobState &s = plan->jobs[k];
          const uint8_t *v = reinterpret_cast<const uint8_t *>(voltages[k]);
          const int uv = unpack_choice(s, v);
          if (uv == 5)
            e = launch_unpack_tile(v, s.job.sample_bits, s.job.n_inputs, s.job.n_time, s.n_tiles,
                                   s.kb, 0, s.job.n_chan, s.op, plan->sm_count * kTileCtasPerSm,
                                   plan->status, plan->timeout_ns, cs);
          else
            e = launch_unpack(v, s.job.sample_bits, s.job.n_inputs, s.job.n_time, s.n_tiles, s.kb, 0,
                              s.job.n_chan, s.op, 0, cs);
        }
      } else if (e == cudaSuccess) {
        // jobs whose items are cut into time ranges add into a zeroed output
        for (int k = 0; k < nj && e == cudaSuccess; ++k)
          if (plan->jobs[k].k_split > 1)
            e = cudaMemsetAsync(out[k], 0, (size_t)(plan->jobs[k].job.n_chan * plan->jobs[k].out_chan_bytes), cs);
        TcLaunch cfg = launch_cfg(plan);
        cfg.items = plan->items;
        cfg.n_items = plan->n_items_full;
        if (e == cudaSuccess) e = launch_correlate_tc(tj.data(), nj, cfg, cs);
      }
      cudaError_t e2 = cudaStreamEndCapture(cs, &g);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(part == 0 ? &plan->graph : &plan->graph2, g, 0);
      if (g) cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      for (cudaGraphExec_t *ge : {&plan->graph, &plan->graph2})
        if (*ge) {
          cudaGraphExecDestroy(*ge);
          *ge = nullptr;
        }
      return cuda_status(e);
    }
    plan->graph_in.assign(voltages, voltages + nj);
    plan->graph_out.assign(out, out + nj);
  }
  cudaError_t e = cudaSuccess;
  if (!fused) {
    TimedLaunch tu(plan, 0, plan->stream);
    e = cudaGraphLaunch(plan->graph, plan->stream);
    tu.done();
    if (e != cudaSuccess) return cuda_status(e);
  }
  TimedLaunch tc(plan, 1, plan->stream);
  e = cudaGraphLaunch(plan->graph2, plan->stream);
  tc.done();
  return cuda_status(e);
}

mwax_status mwax_plan_set_timing(mwax_plan_t plan, int enable) {
  if (!plan) return MWAX_ERR_INVALID_ARG;
  plan->timing = enable != 0;
  return MWAX_OK;
}

mwax_status mwax_plan_get_timing(mwax_plan_t plan, mwax_timing *t) {
  if (!plan || !t) return MWAX_ERR_INVALID_ARG;
  memset(t, 0, sizeof(*t));
  cudaError_t e = cudaStreamSynchronize(plan->stream);
  if (e != cudaSuccess) return cuda_status(e);
  for (const auto &r : plan->recs) {
    float ms = 0.f;
    e = cudaEventSynchronize(r.stop);  // copy events live on the copy streams
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.start, r.stop);
    if (e != cudaSuccess) return cuda_status(e);
    if (r.kind == 0) {
      t->unpack_ms += ms;
      t->unpack_launches += 1;
    } else if (r.kind == 1) {
      t->correlate_ms += ms;
      t->correlate_launches += 1;
    } else if (r.kind == 2) {
      t->h2d_ms += ms;
      t->h2d_bytes += r.bytes;
      t->h2d_copies += 1;
    } else {
      t->d2h_ms += ms;
      t->d2h_bytes += r.bytes;
      t->d2h_copies += 1;
    }
  }
  plan->recs.clear();
  return MWAX_OK;
}

mwax_status mwax_correlate_host(mwax_plan_t plan, const void *voltages_host, int n_inputs,
                                int n_chan, int n_time, void *out_host) {
  NvtxRange nvtx_("mwax_correlate_host");
  if (!plan || plan->batch || !voltages_host || !out_host) return MWAX_ERR_INVALID_ARG;
  JobState &s = plan->jobs[0];
  if (n_inputs != s.job.n_inputs || n_chan != s.job.n_chan || n_time != s.job.n_time)
    return MWAX_ERR_SHAPE_MISMATCH;
  const int G = s.chan_group;
  cudaError_t e = cudaSuccess;
  if (!plan->h2d) {
    plan->stage_in_bytes = s.in_chan_bytes * G;
    plan->stage_out_bytes = s.out_chan_bytes * G;
    e = cudaStreamCreateWithFlags(&plan->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&plan->d2h, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaMalloc(&plan->stage_in[k], (size_t)plan->stage_in_bytes);
      if (e == cudaSuccess) e = cudaMalloc(&plan->stage_out[k], (size_t)plan->stage_out_bytes);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->ev_in[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->ev_comp[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->ev_out[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_status(e);
  }
  const uint8_t *hin = reinterpret_cast<const uint8_t *>(voltages_host);
  uint8_t *hout = reinterpret_cast<uint8_t *>(out_host);
  const bool use_pair = !plan->checked || checked_call_uses_pair(plan);
  // the copy streams must not start before earlier work on the plan's stream
  e = cudaEventRecord(plan->ev_comp[0], plan->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->h2d, plan->ev_comp[0], 0);
  int64_t gi = 0;
  for (int64_t c0 = 0; c0 < n_chan && e == cudaSuccess; c0 += G, ++gi) {
    const int k = (int)(gi & 1);
    const int nc = (int)std::min<int64_t>(G, n_chan - c0);
    // input stage k is free once the compute of group gi-2 finished
    if (gi >= 2) e = cudaStreamWaitEvent(plan->h2d, plan->ev_comp[k], 0);
    if (e == cudaSuccess) {
      TimedLaunch tc_in(plan, 2, plan->h2d);
      e = cudaMemcpyAsync(plan->stage_in[k], hin + c0 * s.in_chan_bytes, nc * s.in_chan_bytes,
                          cudaMemcpyHostToDevice, plan->h2d);
      tc_in.done(nc * s.in_chan_bytes);
    }
    if (e == cudaSuccess) e = cudaEventRecord(plan->ev_in[k], plan->h2d);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->stream, plan->ev_in[k], 0);
    // output stage k is free once its copy-out of group gi-2 finished
    if (e == cudaSuccess && gi >= 2) e = cudaStreamWaitEvent(plan->stream, plan->ev_out[k], 0);
    if (e != cudaSuccess) break;
    mwax_status r;
    if (plan->engine == MWAX_ENGINE_PLAIN) {
      r = MWAX_OK;
      for (int c = 0; c < nc && r == MWAX_OK; ++c)
        r = cuda_status(launch_plain_channel(
            plan->stage_in[k] + (int64_t)c * s.in_chan_bytes, s.job.sample_bits, s.job.n_inputs,
            s.job.n_time, reinterpret_cast<int32_t *>(plan->stage_out[k]) + (int64_t)c * s.n_bl * 2,
            plan->sm_count, plan->stream));
    } else {
      r = run_group(plan, s, plan->stage_in[k], 0, nc, plan->stage_out[k], plan->stream, use_pair);
    }
    if (r != MWAX_OK) return r;
    e = cudaEventRecord(plan->ev_comp[k], plan->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->d2h, plan->ev_comp[k], 0);
    if (e == cudaSuccess) {
      TimedLaunch tc_out(plan, 3, plan->d2h);
      e = cudaMemcpyAsync(hout + c0 * s.out_chan_bytes, plan->stage_out[k], nc * s.out_chan_bytes,
                          cudaMemcpyDeviceToHost, plan->d2h);
      tc_out.done(nc * s.out_chan_bytes);
    }
    if (e == cudaSuccess) e = cudaEventRecord(plan->ev_out[k], plan->d2h);
  }
  if (e == cudaSuccess && plan->checked && use_pair) e = checked_call_done(plan, plan->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(plan->d2h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(plan->stream);
  return cuda_status(e);
}

}  // extern "C"
