// mwax_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "mwax.h"

#include <nvtx3/nvToolsExt.h>

namespace mwax {
// NVTX range over one library call (visible in profilers; a no-op otherwise).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace mwax

namespace mwax {

// Tensor-core tiling: a tile is 128 inputs (the MMA M and N extent) of one
// block of S time samples, 128 rows of 128 bytes (one 128-byte swizzle row
// each): for 8-bit samples a row per input, S re then S im values; for 4-bit
// samples a row per sample and plane (S re rows, then S im rows), each row the
// tile's 128 inputs.
constexpr int kTile = 128;
constexpr int kRowBytes = 128;

inline int samples_per_block(int sample_bits) { return sample_bits == 4 ? 64 : 32; }
inline int bytes_per_sample(int sample_bits) { return sample_bits == 4 ? 1 : 2; }
inline int sample_max(int sample_bits) { return sample_bits == 4 ? 7 : 127; }

// ---- plain CUDA-core correlator (one launch per channel) ------------------
// sm_count sizes the launch: a channel with few tile pairs has its
// integration cut into ranges (the output is zeroed first, on s).
cudaError_t launch_plain_channel(const uint8_t *volt_chan, int sample_bits, int n_inputs,
                                 int n_time, int32_t *out_chan, int sm_count, cudaStream_t s);

// ---- unpack: packed samples -> tensor-core operand tiles -------------------
// volt: [n_chan_total][T][N] packed.  op, 8-bit samples (K-major):
// [n_chan][kb][n_tiles*128][128 B]; 4-bit samples (MN-major):
// [n_chan][kb][2 planes x 64 samples][n_tiles*128 bytes].  Same size per
// channel either way.  variant (8-bit): 0 = automatic, 1 = shared-memory
// transpose, 2 = full-line; 4-bit samples have one form (the streaming kernel).
cudaError_t launch_unpack(const uint8_t *volt, int sample_bits, int n_inputs, int n_time,
                          int n_tiles, int kb, int64_t chan0, int n_chan, uint8_t *op,
                          int variant, cudaStream_t s);

// Persistent unpack on `ctas` CTAs that cannot share an SM with a correlate
// CTA (used when the unpack of the next channel group runs beside the
// correlation of the current one on disjoint SMs).  Needs even N (8-bit).
cudaError_t launch_unpack_persistent(const uint8_t *volt, int sample_bits, int n_inputs,
                                     int n_time, int n_tiles, int kb, int64_t chan0, int n_chan,
                                     uint8_t *op, int ctas, cudaStream_t s);

// Small-footprint unpack.  8-bit samples with n_inputs even: the tile kernel
// (one 128-input tile x one time block per task, ~25 KB of shared memory:
// several CTAs per SM when it runs alone, one beside a resident correlate CTA
// when it overlaps; TMA store of the operand tile; the raw box by 2D TMA where
// the sample rows are whole 16-byte units, else loaded by the threads).
// 4-bit samples, any n_inputs: the streaming kernel (no shared memory) on
// ctas / 2 CTAs of 256 threads.
bool unpack_tile_supported(int sample_bits, int n_inputs);
cudaError_t launch_unpack_tile(const uint8_t *volt, int sample_bits, int n_inputs, int n_time,
                               int n_tiles, int kb, int64_t chan0, int n_chan, uint8_t *op,
                               int ctas, int32_t *status, unsigned long long timeout_ns,
                               cudaStream_t s);
// ---- tensor-core correlator -------------------------------------------------
#define MWAX_MAX_JOBS 8

struct TcJob {
  const uint8_t *op;  // operand tiles of n_chan channels (layout: see launch_unpack); fused
                      // pair mode: the packed samples [n_chan][n_time][n_inputs] themselves
  void *out;          // visibilities of the first of these n_chan channels
  int32_t n_inputs, n_tiles, n_pairs, kb, flush_blocks, n_chan;
  int32_t n_time = 0;  // samples per integration (read by the fused pair mode)
  int64_t n_bl;
  // pair mode: time ranges per work item (1: whole integration; > 1: each
  // range's partial sums are added into the zeroed output with int32 atomics)
  int32_t k_split = 1;
};

struct TcLaunch {
  int sample_bits;
  int kind;  // mwax_kind
  int grid;
  int stages;
  int prefetch;  // K-blocks of L2 prefetch ahead of the TMA loads (0 = none; narrow only)
  int mode;      // 0: narrow (N=128 MMAs), 1: wide (N=256 with B' built in shared
                 // memory), 2: pair (two tile pairs per work item, see items), 3: fused
                 // pair (pair mode reading packed 4-bit samples, no unpack pass)
  int withhold_seg;  // test hook (-1: off): see mwax_job.test_fault
  int32_t *status;
  unsigned long long timeout_ns;
  const int4 *items = nullptr;  // mode 2: device work list from build_pair_items
  int64_t n_items = 0;
  // modes 0/1, one job: correlate only the channels chan_map[0 .. *n_chan_dev)
  // (device memory, written by an earlier launch on the stream)
  const int32_t *chan_map = nullptr;
  const int32_t *n_chan_dev = nullptr;
};

// Encodes one TMA descriptor per job and launches the persistent kernel over
// the work items: in modes 0 and 1 the concatenated (job, channel, tile pair)
// items, job by job, channel-major; in mode 2 the given work list.
cudaError_t launch_correlate_tc(const TcJob *jobs, int n_jobs, const TcLaunch &cfg,
                                cudaStream_t s);
int correlate_tc_smem_bytes(int stages, int mode);
int correlate_tc_max_stages(int mode);
cudaError_t correlate_tc_prepare(int sample_bits, int kind, int stages, int mode);

// Pair mode needs every job's integration in one exact segment (kb <=
// flush_blocks), at most 255 tiles, kb < 2^28 and 1 <= k_split <= min(kb, 8).
bool pair_mode_supported(const TcJob *jobs, int n_jobs);
// The fused pair mode also needs 4-bit exact samples, n_inputs a multiple of
// 16 (whole 16-byte sample rows) and sample buffers on 16-byte boundaries.
bool fused_pair_supported(const TcJob *jobs, int n_jobs, int sample_bits, int kind);
// The pair-mode work list of one launch over `jobs` (16 bytes per item).
void build_pair_items(const TcJob *jobs, int n_jobs, std::vector<int4> &items);

// After a pass that accumulated each item in one FP32 segment: append to
// bad[1..] (count in bad[0], reset here) every channel of out[0 .. n_chan)
// whose largest auto-correlation reached 2^24, so its result may be inexact,
// and add their number to recomputed[0] and recomputed[1].
cudaError_t launch_exact_check(const int32_t *out, int64_t n_bl, int n_inputs, int n_chan,
                               int32_t *bad, unsigned long long *recomputed, cudaStream_t s);

// Fill the tuning fields of an all-auto job from the MWAX_TUNE_CACHE file.
void apply_tune_cache(mwax_job *job);

}  // namespace mwax
