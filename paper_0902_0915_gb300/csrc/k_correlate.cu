// k_correlate.cu -- tensor-core X-engine correlator for sm_103a (tcgen05).
//
// Computes, for every fine channel and every 128x128 tile pair (I >= J) of
// the input triangle (paper Sec. 2: all antenna pairs cross-correlated per
// channel, then integrated over the dump),
//     Re V_ij = sum_t xr_i xr_j + xi_i xi_j
//     Im V_ij = sum_t xi_i xr_j - xr_i xi_j
// as a dense rank-T Hermitian update on the 5th-generation tensor cores.
//
// Operands come from k_unpack.cu as 128 x 128-byte tiles of exact small
// floats, one per 128 inputs and block of S time samples, each holding two K
// slices of re and two of im (one MMA consumes one slice):
//   8-bit samples (binary16, S = 32), K-major: a row per input,
//       [re x 32 | im x 32]; slice s of re is bytes 32s .. 32s+31 of every
//       row, of im bytes 64 + 32s ..;
//   4-bit samples (E4M3, S = 64), MN-major: rows 0..63 hold the re codes of
//       the tile's 128 inputs at samples 0..63, rows 64..127 the im codes;
//       slice s of re is rows 32s .. 32s+31, of im rows 64 + 32s ...
// Per block the MMA warp issues eight M=128 N=128 MMAs:
//     D_re += re_A[s] . re_B[s] + im_A[s] . im_B[s]     s = 0, 1
//     D_im += im_A[s] . re_B[s]                         (xi_i xr_j)
//     D_im -= re_A[s] . im_B[s]                         (xr_i xi_j; negate-B bit)
// Every product of two sample values is an exact integer and every partial
// sum stays an integer below 2^24 for `flush_blocks` blocks, so the FP32
// accumulator in tensor memory is exact; at the end of each such segment
// the epilogue warps convert it (round-to-nearest, exact) to int32 and add
// it to int32 register totals.  The plan bounds T so the totals fit int32.
//
// Roles (one persistent CTA per SM, 10 warps):
//   warp 0      single-thread TMA producer: tiles A_I and A_J of the next
//               K blocks into a ring of shared-memory stages (three blocks per
//               stage for the narrow shape; A_J skipped on diagonal tiles)
//   warp 1      tensor-memory allocator and single-thread MMA issuer (one
//               full-barrier wait and one commit per stage)
//   warps 2..9  epilogue: tcgen05.ld of the FP32 accumulator, int32 flush,
//               packed lower-triangle store (the integration dump)
// Two 256-column accumulators (re 128 | im 128) are double-buffered in the
// 512 tensor-memory columns so the epilogue of one segment overlaps the
// MMAs of the next.
//
// Pair mode (jobs whose whole integration is one exact segment: 4-bit
// samples up to 171,136 time samples, and the FP16 variant): a work item
// holds two tile pairs, usually (I, J) and (I, J+1) of one channel, so one
// M=128 N=256 MMA against the consecutive shared-memory tiles [A_J | A_J+1]
// produces both; the A tile is loaded once for the two pairs and the tensor
// pipe runs 136-cycle instructions, which hide the issuing thread's barrier
// waits.  The 512 columns then hold one item (Re of both pairs in [0, 256),
// Im in [256, 512)); the epilogue converts it once and stores it through a
// per-warp shared-memory transpose, so every store instruction writes whole
// 128-byte row segments.
//
// Every mbarrier wait is bounded by a %globaltimer deadline; on expiry the
// kernel records MWAX_ERR_TIMEOUT in the plan's status word, stops issuing,
// waits (bounded) for its own copies and MMAs in flight, frees its tensor
// memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include "mwax_internal.h"
#include "mwax_nib4.h"

namespace mwax {
namespace {

constexpr int kTileBytes = kTile * kRowBytes;  // 16 KB

// Three MMA shapes (MODE).  0, narrow: eight M=128 N=128 MMAs per block (Re
// and Im separately, negate-B bit for the minus sign).  1, wide: four M=128
// N=256 MMAs per block against B = [A_J ; B'_J], B'_J = [-im_j | re_j] built
// in shared memory by two extra warps.  2, pair: work items of two tile
// pairs (see the header), up to three tiles per block.
// A shared-memory stage holds `kps` consecutive K blocks behind one pair of
// full/empty barriers.  An mbarrier wait costs the single issuing thread
// about as much as two N=128 MMA issues, and every stage boundary leaves a
// bubble in the tensor pipe, so the narrow shape takes three blocks (24
// MMAs) per wait and per commit: two stages of 96 KB.
// 3, fused pair: the pair mode for 4-bit samples with the unpack folded in:
// the eight epilogue warps also convert: they read the packed samples from
// global memory and write the E4M3 operand tiles into the stages themselves
// (no operand buffer in HBM, no unpack pass), and drain each item's
// accumulator after its last stage.
constexpr int kModeNarrow = 0, kModeWide = 1, kModePair = 2, kModePairFused = 3;
constexpr int kEpiStageBytes = 32 * 128;  // pair mode: one warp's 32 rows x 16 (re, im) words

template <int MODE>
struct Shape {
  static constexpr bool pair = MODE == kModePair || MODE == kModePairFused;
  static constexpr int warps = MODE == kModeWide ? 12 : 10;
  // warps 2 .. 2+conv_warps-1: B' builders (wide only)
  static constexpr int conv_warps = MODE == kModeWide ? 2 : 0;
  static constexpr int epi0 = 2 + conv_warps;  // 8 epilogue warps from here to the last
  static constexpr int epi_warps = warps - epi0;
  // fused pair mode: the epilogue warps convert the samples (full-barrier arrivals per stage)
  static constexpr int fill_arrivals = MODE == kModePairFused ? epi_warps : 1;
  static constexpr int kps = MODE == kModeWide ? 1 : pair ? 2 : 3;  // K blocks per stage
  static constexpr int block_bytes = (MODE == kModeNarrow ? 2 : 3) * kTileBytes;  // tiles of one block
  static constexpr int stage_bytes = kps * block_bytes;
  static constexpr int max_stages = MODE == kModeWide ? 4 : 2;
  static constexpr int epi_bytes = pair ? epi_warps * kEpiStageBytes : 0;
};
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccCols = 256;  // re 128 | im 128
constexpr int kMaxJobs = MWAX_MAX_JOBS;

// One job of a (possibly batched) launch.
struct KJob {
  void *out;           // visibilities of the job's first channel in this launch
  int64_t item_begin;  // first work item of this job
  int64_t n_bl;        // N(N+1)/2
  int32_t n_inputs, n_tiles, n_pairs, kb, flush_blocks;
  int32_t n_time;       // fused pair mode: samples per integration
  const uint8_t *volt;  // fused pair mode: packed samples of the launch's first channel
};

struct KParams {
  KJob job[kMaxJobs];
  int32_t *status;
  const int4 *items;  // pair mode: the work list (n_items entries)
  // narrow mode, one job: when n_chan_dev is set, the launch covers the
  // *n_chan_dev channels chan_map[0..) (count and list written on the device)
  const int32_t *chan_map;
  const int32_t *n_chan_dev;
  int64_t n_items;
  unsigned long long timeout_ns;
  int32_t n_jobs, stages, prefetch;
  int32_t withhold_seg;  // test hook: segment whose accumulator release the epilogue withholds (-1: none)
};

struct KMaps {
  CUtensorMap m[kMaxJobs];
};

// ---- PTX wrappers --------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with parity `parity` to complete.  Returns false
// on timeout, or when another role has raised the abort flag.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int *abort_flag,
                                          unsigned long long timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (abort_flag && *abort_flag) return false;
    if (globaltimer() - t0 > timeout_ns) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Fire-and-forget L2 prefetch of one box of the tensor (no completion tracking).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

// Shared-memory matrix descriptor, MN-major, 128-byte swizzle: atoms of 8 K
// rows x 128 bytes of MN (1024 bytes, stride byte offset) and the next
// 128-input tile along MN kTileBytes on (leading byte offset; used when B
// spans two tiles, N = 256).
__device__ __forceinline__ uint64_t sw128_mn_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(kTileBytes >> 4) << 16;  // leading byte offset: next MN atom
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: next 8 K rows
  d |= (uint64_t)1 << 46;                  // version
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}

// Operand tile of each sample width: its descriptor and the descriptor
// offsets (16-byte units) of the K slices re 0, re 1, im 0, im 1.
template <int BITS>
struct Op;
template <>
struct Op<8> {  // binary16, K-major
  static constexpr bool mn = false;
  static constexpr uint64_t re0 = 0, re1 = 2, im0 = 4, im1 = 6;
  static __device__ __forceinline__ uint64_t desc(uint32_t addr) { return sw128_desc(addr); }
};
template <>
struct Op<4> {  // E4M3, MN-major
  static constexpr bool mn = true;
  static constexpr uint64_t re0 = 0, re1 = 256, im0 = 512, im1 = 768;
  static __device__ __forceinline__ uint64_t desc(uint32_t addr) { return sw128_mn_desc(addr); }
};

// Instruction descriptor: FP32 accumulate, A/B type code 0 (F16 for
// kind::f16, E4M3 for kind::f8f6f4), optional negation of B, K-major (8-bit
// samples) or MN-major (4-bit samples) A and B, M = 128, N = n.
template <int BITS>
__host__ __device__ constexpr uint32_t make_idesc(bool negate_b, int n) {
  return (1u << 4) | ((negate_b ? 1u : 0u) << 14) | ((Op<BITS>::mn ? 1u : 0u) << 15) |
         ((Op<BITS>::mn ? 1u : 0u) << 16) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kTile >> 4) << 24);
}

// TMA coordinates of a tile: (x, y) of K block 0 and the row step per K block.
//   8-bit: [chan][kb][row][128 B] viewed as rows of 128 bytes; tile I of
//          channel c, block b at row (c * KB + b) * n_rows + 128 I;
//   4-bit: [chan][kb][128 rows][n_rows bytes]; x = 128 I, row (c * KB + b) * 128.
template <int BITS>
struct TileAt {
  int x, y, step;
  __device__ __forceinline__ TileAt(int c, int tile, int KB, int n_rows) {
    if constexpr (Op<BITS>::mn) {
      x = tile * kTile;
      y = c * KB * kTile;
      step = kTile;
    } else {
      x = 0;
      y = c * KB * n_rows + tile * kTile;
      step = n_rows;
    }
  }
};

template <int BITS>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  if constexpr (BITS == 8) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// tile pair p -> (I, J), p = I(I+1)/2 + J, I >= J
__device__ __forceinline__ void pair_of(int p, int &I, int &J) {
  int i = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  while (i * (i + 1) / 2 > p) --i;
  I = i;
  J = p - i * (i + 1) / 2;
}

// Work item -> (job, channel, I, J).  Items are numbered job by job.
struct Item {
  int job, c, I, J;
};
__device__ __forceinline__ Item decode_item(const KParams &p, int64_t item) {
  int j = 0;
  while (j + 1 < p.n_jobs && item >= p.job[j + 1].item_begin) ++j;
  const int64_t local = item - p.job[j].item_begin;
  Item it;
  it.job = j;
  const int cl = (int)(local / p.job[j].n_pairs);
  it.c = p.chan_map ? __ldg(p.chan_map + cl) : cl;
  pair_of((int)(local % p.job[j].n_pairs), it.I, it.J);
  return it;
}

// Items of a narrow/wide launch (read once per thread; with a device-side
// channel count the launch was sized for the largest count).
__device__ __forceinline__ int64_t launch_items(const KParams &p) {
  if (!p.n_chan_dev) return p.n_items;
  return (int64_t)*reinterpret_cast<const volatile int32_t *>(p.n_chan_dev) * p.job[0].n_pairs;
}

// Named barrier `id` over `threads` threads (whole warps); waiting warps sleep.
__device__ __forceinline__ void named_bar_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

__device__ __forceinline__ void raise_timeout(volatile int *abort_flag, int32_t *status) {
  *abort_flag = 1;
  atomicExch(status, (int32_t)MWAX_ERR_TIMEOUT);
}

// Lane 0 waits; the result is broadcast so the warp takes one branch.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned long long timeout_ns, int lane) {
  int ok = 1;
  if (lane == 0) ok = mbar_wait(bar, parity, abort_flag, timeout_ns) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// ---- pair-mode work items -------------------------------------------------
// One int4 per item: x = channel of the first pair, y = channel of the second
// (both relative to the launch's first channel), z = job | type << 8 |
// I0 << 16 | J0 << 24, w = I1 | J1 << 8 | split << 16 | n_split << 24: the
// item covers time blocks [split KB / n_split, (split + 1) KB / n_split)
// (n_split 1: the whole integration, results stored; n_split > 1: the
// partial sums are added into the zeroed output with int32 atomics).
//   kItemShared:  (I0, J0) and (I0, J1 = J0 + 1 <= I0) of channel x; tiles
//                 [A_J0 | A_J1 | A_I0] (two tiles, [A_J0 | A_I0], when J1 = I0)
//   kItemTwoDiag: (I0, I0) of channel x and (I1, I1) of channel y; [A_I0 | A_I1]
//   kItemOne:     (I0, J0) of channel x alone; [A_I0 | A_J0] ([A_I0] if diagonal)
enum : uint32_t { kItemOne = 0, kItemShared = 1, kItemTwoDiag = 2 };

struct PairItem {
  int job, type, c0, c1, I0, J0, I1, J1, split, n_split;
};

__device__ __forceinline__ PairItem decode_pair_item(const int4 d) {
  const uint32_t z = (uint32_t)d.z, w = (uint32_t)d.w;
  PairItem it;
  it.c0 = d.x;
  it.c1 = d.y;
  it.job = (int)(z & 0xFFu);
  it.type = (int)((z >> 8) & 0xFFu);
  it.I0 = (int)((z >> 16) & 0xFFu);
  it.J0 = (int)(z >> 24);
  it.I1 = (int)(w & 0xFFu);
  it.J1 = (int)((w >> 8) & 0xFFu);
  it.split = (int)((w >> 16) & 0xFFu);
  it.n_split = (int)(w >> 24);
  return it;
}

// Time blocks [k0, k1) of an item of a job with KB blocks.
__device__ __forceinline__ void item_blocks(const PairItem &it, int KB, int &k0, int &k1) {
  // 32-bit products: exact for n_split <= 8 and KB < 2^28 (pair_mode_supported)
  k0 = (int)((uint32_t)(it.split * KB) / (uint32_t)it.n_split);
  k1 = (int)((uint32_t)((it.split + 1) * KB) / (uint32_t)it.n_split);
}

// Pair-mode epilogue: each lane writes column j (lane & 15) of 16 of the 32
// staged rows i0 + r (r = 2 r2 + lane / 16) of one half-block, lower triangle
// only; ADD: add into the output with int32 atomics (one time range of several)
// instead of storing.
template <bool ADD>
__device__ __forceinline__ void store_rows(const uint8_t *stg, uint32_t *out, int lane, int i0,
                                           int j, int n) {
  const int col = lane & 15;
#pragma unroll
  for (int r2 = 0; r2 < 16; ++r2) {
    const int r = 2 * r2 + (lane >> 4);
    const uint2 val = *reinterpret_cast<const uint2 *>(stg + r * 128 + ((col ^ (r & 15)) << 3));
    const int i = i0 + r;
    if (i < n && j <= i) {
      uint32_t *dst = out + 2 * ((int64_t)i * (i + 1) / 2 + j);
      if constexpr (ADD) {
        atomicAdd(reinterpret_cast<int *>(dst), (int)val.x);
        atomicAdd(reinterpret_cast<int *>(dst) + 1, (int)val.y);
      } else {
        *reinterpret_cast<uint2 *>(dst) = val;
      }
    }
  }
}

// The eight MMAs of one K block: N = 128 (one tile pair) or 256 (B spans two
// tiles: two pairs sharing A).
template <int BITS, int N>
__device__ __forceinline__ void block_mmas(uint32_t d_re, uint32_t d_im, uint64_t da, uint64_t db,
                                           uint32_t acc0) {
  using O = Op<BITS>;
  constexpr uint32_t id = make_idesc<BITS>(false, N), idn = make_idesc<BITS>(true, N);
  tc_mma<BITS>(d_re, da + O::re0, db + O::re0, id, acc0);
  tc_mma<BITS>(d_re, da + O::re1, db + O::re1, id, 1u);
  tc_mma<BITS>(d_re, da + O::im0, db + O::im0, id, 1u);
  tc_mma<BITS>(d_re, da + O::im1, db + O::im1, id, 1u);
  tc_mma<BITS>(d_im, da + O::im0, db + O::re0, id, acc0);
  tc_mma<BITS>(d_im, da + O::im1, db + O::re1, id, 1u);
  tc_mma<BITS>(d_im, da + O::re0, db + O::im0, idn, 1u);
  tc_mma<BITS>(d_im, da + O::re1, db + O::im1, idn, 1u);
}

// The eight M=128 N=128 MMAs of one K block of one tile pair.
template <int BITS>
__device__ __forceinline__ void narrow_block(uint32_t d_re, uint32_t d_im, uint64_t da, uint64_t db,
                                             uint32_t acc0) {
  block_mmas<BITS, kTile>(d_re, d_im, da, db, acc0);
}

// Fused pair mode: one converter thread's share of tile I of channel c, time
// block kb (64 samples): the packed samples of kConvUnits (sample, 16-input)
// units (unit u = sample u / 8, inputs 16 (u % 8) ..; thread ct takes units
// ct + 256 m), loaded first (fused_load), then written as E4M3 codes
// (fused_store), re plane at row t and im plane at row 64 + t of the tile,
// each 16-byte chunk at its 128-byte swizzle position.  Samples past T and
// inputs past N read as zero (N is a multiple of 16).
__device__ __forceinline__ uint4 ld_stream16(const uint8_t *p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

#ifndef MWAX_FUSED_PREFETCH
#define MWAX_FUSED_PREFETCH 3  // fused pair mode: stages of L2 prefetch ahead of the converters (0: none)
#endif
constexpr int kFusedPrefetch = MWAX_FUSED_PREFETCH;
constexpr int kConvThreads = 256;                  // fused pair mode: the 8 epilogue warps
constexpr int kConvUnits = 64 * 8 / kConvThreads;  // (sample, 16 inputs) units per thread per tile

struct FusedTile {
  const uint8_t *row0;  // sample 0 of the block, input 128 I, channel c (never dereferenced as is)
  int t_left;           // samples of the block that exist (T - 64 kb, may be <= 0)
  int in_left;          // inputs of the tile that exist (N - 128 I)
};

__device__ __forceinline__ void fused_load(const FusedTile &f, int N, int ct, uint4 (&w)[kConvUnits]) {
#pragma unroll
  for (int m = 0; m < kConvUnits; ++m) {
    const int u = ct + kConvThreads * m;
    const int t = u >> 3, x = (u & 7) << 4;
    w[m] = t < f.t_left && x < f.in_left ? ld_stream16(f.row0 + (int64_t)t * N + x) : make_uint4(0, 0, 0, 0);
  }
}

__device__ __forceinline__ void fused_store(uint8_t *tile, int ct, const uint4 (&w)[kConvUnits]) {
#pragma unroll
  for (int m = 0; m < kConvUnits; ++m) {
    const int u = ct + kConvThreads * m;
    const int t = u >> 3, ch = u & 7;
    const int off = t * kRowBytes + ((ch ^ (t & 7)) << 4);
    const uint4 v = w[m];
    *reinterpret_cast<uint4 *>(tile + off) =
        make_uint4(nib4_to_e4m3_f16(v.x), nib4_to_e4m3_f16(v.y), nib4_to_e4m3_f16(v.z), nib4_to_e4m3_f16(v.w));
    *reinterpret_cast<uint4 *>(tile + 64 * kRowBytes + off) =
        make_uint4(nib4_to_e4m3_f16(v.x >> 4), nib4_to_e4m3_f16(v.y >> 4), nib4_to_e4m3_f16(v.z >> 4), nib4_to_e4m3_f16(v.w >> 4));
  }
}

// Pair-mode epilogue of one work item (warp (q, h) of the eight epilogue
// warps): wait for the accumulator (one thread; the result goes through a
// two-entry flag so all eight warps take the same branch), convert, release
// the accumulator, store the item's lower-triangle visibilities.  false: a
// wait ran out (every warp stops).
template <int KIND>
__device__ __forceinline__ bool drain_item(const KParams &p, const PairItem &it, uint32_t n_it,
                                           uint32_t tfull, uint32_t tempty, uint32_t tmem_base,
                                           uint8_t *stg, volatile int *abort_flag,
                                           volatile int *epi_flag, int warp, int lane, int epi0) {
  const unsigned long long tmo = p.timeout_ns;
  const int q = warp & 3;
  const int h = (warp - epi0) >> 2;
  const KJob &jb = p.job[it.job];
  if (warp == epi0 && lane == 0) {
    const bool got = mbar_wait(tfull, n_it & 1u, abort_flag, tmo);
    if (!got) raise_timeout(abort_flag, p.status);
    epi_flag[n_it & 1u] = got ? 1 : 0;
  }
  named_bar_sync(1, 8 * 32);
  if (!epi_flag[n_it & 1u]) return false;
  tc_fence_after();
  const bool has = h == 0 || it.type != kItemOne;
  int c, I, J;
  if (it.type == kItemShared) {
    c = it.c0;
    I = it.I0;
    J = h ? it.J1 : it.J0;
  } else if (it.type == kItemTwoDiag) {
    c = h ? it.c1 : it.c0;
    I = h ? it.I1 : it.I0;
    J = I;
  } else {
    c = it.c0;
    I = it.I0;
    J = it.J0;
  }
  const uint32_t trow = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * kTile);
  uint32_t *out = reinterpret_cast<uint32_t *>(jb.out) + (int64_t)c * jb.n_bl * 2;
  const int n = jb.n_inputs;
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    uint32_t vre[32], vim[32];
    if (has) {
      tc_ld32(trow + 32 * cc, vre);
      tc_ld32(trow + 2 * kTile + 32 * cc, vim);
      tc_wait_ld();
    }
    if (cc == 3) {
      // every column of this warp is in registers: release the accumulator
      // (test hook: withholding one release makes the MMA warp's bounded
      // wait run out -> MWAX_ERR_TIMEOUT, clean exit)
      tc_fence_before();
      __syncwarp();
      if (lane == 0 && (int)n_it != p.withhold_seg) mbar_arrive(tempty);
    }
    if (!has) continue;
    if constexpr (KIND == MWAX_KIND_EXACT) {
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        vre[k] = (uint32_t)__float2int_rn(__uint_as_float(vre[k]));
        vim[k] = (uint32_t)__float2int_rn(__uint_as_float(vim[k]));
      }
    }
#pragma unroll
    for (int half = 0; half < 2; ++half) {
#pragma unroll
      for (int k = 0; k < 16; ++k)
        *reinterpret_cast<uint2 *>(stg + lane * 128 + ((k ^ (lane & 15)) << 3)) =
            make_uint2(vre[16 * half + k], vim[16 * half + k]);
      __syncwarp();
      const int j = J * kTile + 32 * cc + 16 * half + (lane & 15);
      const int i0 = I * kTile + q * 32;
      if (it.n_split > 1)  // one time range of several: exact integer adds
        store_rows<true>(stg, out, lane, i0, j, n);
      else
        store_rows<false>(stg, out, lane, i0, j, n);
      __syncwarp();
    }
  }
  return true;
}

// The same as a separate call (fused pair mode: the converters' state stays
// out of the epilogue's register allocation).
template <int KIND>
__device__ __noinline__ bool drain_item_call(const KParams &p, const PairItem &it, uint32_t n_it,
                                             uint32_t tfull, uint32_t tempty, uint32_t tmem_base,
                                             uint8_t *stg, volatile int *abort_flag,
                                             volatile int *epi_flag, int warp, int lane, int epi0) {
  return drain_item<KIND>(p, it, n_it, tfull, tempty, tmem_base, stg, abort_flag, epi_flag, warp,
                          lane, epi0);
}

// The roles in pair mode.  Warp 0: TMA producer (idle in the fused pair
// mode), warp 1: MMA issuer, warps 2..9: epilogue (in the fused pair mode
// also the sample converters).  Barriers as in the kernel: full[0..S)
// empty[S..2S) tfull[3S] tempty[3S+2] drain[3S+4] (one accumulator buffer:
// index 0 only).
template <int BITS, int KIND, bool FUSED>
__device__ __forceinline__ void pair_roles(const KMaps &maps, const KParams &p, uint8_t *smem,
                                           uint32_t smem_base, uint8_t *epi_smem, uint32_t bar0,
                                           uint32_t tmem_base, volatile int *abort_flag,
                                           volatile int *epi_flag, volatile int *conv_done,
                                           int warp, int lane) {
  using Sh = Shape<FUSED ? kModePairFused : kModePair>;
  constexpr int kStageBytes = Sh::stage_bytes;
  const int S = p.stages;
  const unsigned long long tmo = p.timeout_ns;
  auto full = [&](int s) { return bar0 + 8u * (uint32_t)s; };
  auto empty = [&](int s) { return bar0 + 8u * (uint32_t)(S + s); };
  const uint32_t tfull = bar0 + 8u * (uint32_t)(3 * S);
  const uint32_t tempty = bar0 + 8u * (uint32_t)(3 * S + 2);
  const uint32_t drain = bar0 + 8u * (uint32_t)(3 * S + 4);

  if (warp == 0) {
    // ---------------- TMA producer (one thread) ----------------
    if (!FUSED && lane == 0) {
      for (int j = 0; j < p.n_jobs; ++j)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.m[j]))
                     : "memory");
      int stage = 0;
      uint32_t phase = 0;
      int64_t issued = 0;
      bool ok = true;
      for (int64_t item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        const PairItem it = decode_pair_item(__ldg(p.items + item));
        const KJob &jb = p.job[it.job];
        const CUtensorMap *map = &maps.m[it.job];
        const int n_rows = jb.n_tiles * kTile;
        // each tile of the item at K block 0, in shared-memory order
        TileAt<BITS> ts[3] = {TileAt<BITS>(0, 0, 0, 0), TileAt<BITS>(0, 0, 0, 0),
                              TileAt<BITS>(0, 0, 0, 0)};
        int nt;
        if (it.type == kItemShared) {
          ts[0] = TileAt<BITS>(it.c0, it.J0, jb.kb, n_rows);
          ts[1] = TileAt<BITS>(it.c0, it.J1, jb.kb, n_rows);  // A_I itself when J1 == I0
          ts[2] = TileAt<BITS>(it.c0, it.I0, jb.kb, n_rows);
          nt = it.J1 == it.I0 ? 2 : 3;
        } else if (it.type == kItemTwoDiag) {
          ts[0] = TileAt<BITS>(it.c0, it.I0, jb.kb, n_rows);
          ts[1] = TileAt<BITS>(it.c1, it.I1, jb.kb, n_rows);
          nt = 2;
        } else {
          ts[0] = TileAt<BITS>(it.c0, it.I0, jb.kb, n_rows);
          ts[1] = TileAt<BITS>(it.c0, it.J0, jb.kb, n_rows);
          nt = it.I0 == it.J0 ? 1 : 2;
        }
        const uint32_t blk_bytes = (uint32_t)nt * kTileBytes;
        int k0, k1;
        item_blocks(it, jb.kb, k0, k1);
        for (int kb = k0; kb < k1; kb += Sh::kps) {
          const int nb = min(Sh::kps, k1 - kb);
          if (!mbar_wait(empty(stage), phase ^ 1u, abort_flag, tmo)) {
            raise_timeout(abort_flag, p.status);
            ok = false;
            break;
          }
          const uint32_t a = smem_base + (uint32_t)stage * kStageBytes;
          mbar_arrive_expect_tx(full(stage), (uint32_t)nb * blk_bytes);
          for (int j = 0; j < nb; ++j)
            for (int t = 0; t < nt; ++t)
              tma_load_2d(a + (uint32_t)(j * Sh::block_bytes + t * kTileBytes), map, ts[t].x,
                          ts[t].y + (kb + j) * ts[t].step, full(stage));
          ++issued;
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // wait (bounded) until every copy this thread issued has landed
      int st = stage;
      uint32_t ph = phase;
      for (int64_t k = 0; k < issued && k < S; ++k) {
        if (--st < 0) {
          st = S - 1;
          ph ^= 1u;
        }
        mbar_wait(full(st), ph, nullptr, tmo);
      }
    }
    if (FUSED && kFusedPrefetch > 0 && lane == 0) {
      // ------------ fused pair mode: L2 prefetch of the packed samples ------------
      // The sample rows of each stage's channels, kFusedPrefetch stages ahead
      // of the converters (paced by their count of filled stages, conv_done;
      // a hint only: no result is read), so that their loads hit L2.
      int64_t g = 0;  // stages of this CTA so far
      bool ok = true;
      for (int64_t item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        const PairItem it = decode_pair_item(__ldg(p.items + item));
        const KJob &jb = p.job[it.job];
        const int N = jb.n_inputs, T = jb.n_time;
        const int cb = it.type == kItemTwoDiag ? it.c1 : it.c0;
        int k0, k1;
        item_blocks(it, jb.kb, k0, k1);
        for (int kb = k0; kb < k1; kb += Sh::kps, ++g) {
          if (*conv_done < g - kFusedPrefetch) {
            const uint64_t t0 = globaltimer();
            while (*conv_done < g - kFusedPrefetch) {
              if (*abort_flag || globaltimer() - t0 > tmo) {
                ok = false;
                break;
              }
              __nanosleep(128);
            }
            if (!ok) break;
          }
          const int r0 = kb * 64, r1 = min((kb + Sh::kps) * 64, T);
          if (r1 <= r0) continue;
          const uint32_t bytes = (uint32_t)(r1 - r0) * (uint32_t)N;
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                           jb.volt + ((int64_t)it.c0 * T + r0) * N),
                       "r"(bytes)
                       : "memory");
          if (cb != it.c0)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                             jb.volt + ((int64_t)cb * T + r0) * N),
                         "r"(bytes)
                         : "memory");
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer (one thread) ----------------
    if (lane == 0) {
      const uint32_t d_re = tmem_base, d_im = tmem_base + 2 * kTile;
      int stage = 0;
      uint32_t phase = 0, n_it = 0;
      bool ok = true;
      for (int64_t item = blockIdx.x; item < p.n_items && ok; item += gridDim.x) {
        const PairItem it = decode_pair_item(__ldg(p.items + item));
        int k0, k1;
        item_blocks(it, p.job[it.job].kb, k0, k1);
        // the accumulator is free once the epilogue has read the previous item
        if (!mbar_wait(tempty, (n_it & 1u) ^ 1u, abort_flag, tmo)) {
          raise_timeout(abort_flag, p.status);
          break;
        }
        tc_fence_after();
        const uint32_t a_off = it.J1 == it.I0 ? kTileBytes : 2 * kTileBytes;  // A_I of a shared item
        for (int kb = k0; kb < k1; kb += Sh::kps) {
          const int nb = min(Sh::kps, k1 - kb);
          if (!mbar_wait(full(stage), phase, abort_flag, tmo)) {
            raise_timeout(abort_flag, p.status);
            ok = false;
            break;
          }
          tc_fence_after();
          for (int j = 0; j < nb; ++j) {
            const uint32_t a = smem_base + (uint32_t)stage * kStageBytes + (uint32_t)(j * Sh::block_bytes);
            const uint32_t acc0 = kb + j == k0 ? 0u : 1u;
            if (it.type == kItemShared) {
              // B = [A_J0 ; A_J1]: columns 0..127 give pair (I, J0), 128..255 pair (I, J1)
              const uint64_t da = Op<BITS>::desc(a + a_off), db = Op<BITS>::desc(a);
              block_mmas<BITS, 2 * kTile>(d_re, d_im, da, db, acc0);
            } else if (it.type == kItemTwoDiag) {
              const uint64_t d0 = Op<BITS>::desc(a), d1 = Op<BITS>::desc(a + kTileBytes);
              narrow_block<BITS>(d_re, d_im, d0, d0, acc0);
              narrow_block<BITS>(d_re + kTile, d_im + kTile, d1, d1, acc0);
            } else {
              const uint64_t da = Op<BITS>::desc(a);
              const uint64_t db = it.I0 == it.J0 ? da : Op<BITS>::desc(a + kTileBytes);
              narrow_block<BITS>(d_re, d_im, da, db, acc0);
            }
          }
          if (kb + nb == k1) tc_commit(tfull);
          tc_commit(empty(stage));
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        ++n_it;
      }
      // no MMA may be in flight when tensor memory is freed
      tc_commit(drain);
      mbar_wait(drain, 0, nullptr, tmo);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: convert + integration dump ----------------
    // Warp (q, h): tensor-memory lanes 32q.. (rows of the tile) of pair h.
    // Each 32-column chunk goes through this warp's shared-memory buffer, 16
    // columns at a time: lane r writes row r (16 (re, im) words, XOR-swizzled
    // so the 16 lanes of a phase hit distinct banks), then each store
    // instruction writes rows r and r+1 as two contiguous 128-byte runs.
    // One thread waits for the accumulator; the result goes through a
    // two-entry flag so all eight warps take the same branch (false: stop).
    uint8_t *stg = epi_smem + (warp - Sh::epi0) * kEpiStageBytes;
    auto drain = [&](const PairItem &it, uint32_t n_it) -> bool {
      if constexpr (FUSED)
        return drain_item_call<KIND>(p, it, n_it, tfull, tempty, tmem_base, stg, abort_flag,
                                     epi_flag, warp, lane, Sh::epi0);
      else
        return drain_item<KIND>(p, it, n_it, tfull, tempty, tmem_base, stg, abort_flag, epi_flag,
                                warp, lane, Sh::epi0);
    };
    uint32_t n_it = 0;
    if constexpr (!FUSED) {
      for (int64_t item = blockIdx.x; item < p.n_items; item += gridDim.x) {
        if (!drain(decode_pair_item(__ldg(p.items + item)), n_it)) break;
        ++n_it;
      }
    } else {
      // Fused pair mode: first every stage of the item (the same items and
      // blocks as the MMA issuer; each stage written by all eight warps and
      // released with one arrival per warp after a proxy fence, since the
      // tensor core reads generic-proxy stores), then the item's drain.  A
      // warp whose wait for a free stage runs out skips the rest of the item
      // and still joins the drain, where the shared flag ends every warp.
      const int ct = (int)threadIdx.x - 32 * Sh::epi0;
      int stage = 0;
      uint32_t phase = 0;
      int64_t filled = 0;  // stages of this CTA filled so far
      for (int64_t item = blockIdx.x; item < p.n_items; item += gridDim.x) {
        const PairItem it = decode_pair_item(__ldg(p.items + item));
        const KJob &jb = p.job[it.job];
        const int N = jb.n_inputs, T = jb.n_time;
        // the item's tiles in shared-memory order (as the producer loads them)
        int tc[3] = {it.c0, it.c0, it.c0}, ti[3] = {0, 0, 0};
        int nt;
        if (it.type == kItemShared) {
          ti[0] = it.J0;
          ti[1] = it.J1;
          ti[2] = it.I0;
          nt = it.J1 == it.I0 ? 2 : 3;
        } else if (it.type == kItemTwoDiag) {
          ti[0] = it.I0;
          tc[1] = it.c1;
          ti[1] = it.I1;
          nt = 2;
        } else {
          ti[0] = it.I0;
          ti[1] = it.J0;
          nt = it.I0 == it.J0 ? 1 : 2;
        }
        int k0, k1;
        item_blocks(it, jb.kb, k0, k1);
        for (int kb = k0; kb < k1; kb += Sh::kps) {
          const int nb = min(Sh::kps, k1 - kb);
          if (!warp_wait(empty(stage), phase ^ 1u, abort_flag, tmo, lane)) {
            if (lane == 0) raise_timeout(abort_flag, p.status);
            break;
          }
          uint8_t *st_base = smem + (size_t)stage * kStageBytes;
          // every load of the stage first (one memory latency per stage), then
          // the conversions and shared-memory stores
          uint4 w[Sh::kps][3][kConvUnits];
#pragma unroll
          for (int j = 0; j < Sh::kps; ++j) {
            const int s0 = (kb + j) * 64;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
              if (j < nb && t < nt) {
                FusedTile f;
                f.row0 = jb.volt + ((int64_t)tc[t] * T + s0) * N + ti[t] * kTile;
                f.t_left = T - s0;
                f.in_left = N - ti[t] * kTile;
                fused_load(f, N, ct, w[j][t]);
              }
            }
          }
#pragma unroll
          for (int j = 0; j < Sh::kps; ++j)
#pragma unroll
            for (int t = 0; t < 3; ++t)
              if (j < nb && t < nt) fused_store(st_base + j * Sh::block_bytes + t * kTileBytes, ct, w[j][t]);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(full(stage));
          ++filled;
          if (warp == Sh::epi0 && lane == 0) *conv_done = (int)filled;  // paces the L2 prefetch
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!drain(it, n_it)) break;
        ++n_it;
      }
    }
  }
}

template <int BITS, int KIND, int MODE>
__global__ void __launch_bounds__(Shape<MODE>::warps * 32, 1)
    correlate_tc_kernel(const __grid_constant__ KMaps maps, const __grid_constant__ KParams p) {
  using Sh = Shape<MODE>;
  constexpr bool WIDE = MODE == kModeWide;
  constexpr bool PAIR = Sh::pair;
  constexpr bool FUSED = MODE == kModePairFused;
  constexpr int kStageBytes = Sh::stage_bytes;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~static_cast<uintptr_t>(1023));
  const int S = p.stages;
  uint8_t *epi_smem = smem + (size_t)S * kStageBytes;  // pair mode: per-warp store staging
  uint64_t *bars = reinterpret_cast<uint64_t *>(epi_smem + Sh::epi_bytes);
  // full[0..S) empty[S..2S) bfull[2S..3S) tfull[3S..3S+2) tempty[3S+2..3S+4) drain[3S+4]
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 3 * S + 5);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  // [0..1]: result of the epilogue's accumulator wait; [2]: fused pair mode's filled-stage count
  volatile int *epi_flag = abort_flag + 1;
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto empty = [&](int s) { return smem_u32(bars + S + s); };
  auto bfull = [&](int s) { return smem_u32(bars + 2 * S + s); };
  auto tfull = [&](int b) { return smem_u32(bars + 3 * S + b); };
  auto tempty = [&](int b) { return smem_u32(bars + 3 * S + 2 + b); };
  const uint32_t drain = smem_u32(bars + 3 * S + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long tmo = p.timeout_ns;
  const uint32_t smem_base = smem_u32(smem);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), Sh::fill_arrivals);  // the TMA producer, or the converting warps
      mbar_init(empty(s), 1);
      mbar_init(bfull(s), Sh::conv_warps > 0 ? Sh::conv_warps : 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), Sh::epi_warps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    epi_flag[2] = 0;  // fused pair mode: stages the converters have filled
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int64_t n_items = launch_items(p);

  if constexpr (PAIR) {
    pair_roles<BITS, KIND, FUSED>(maps, p, smem, smem_base, epi_smem, smem_u32(bars), tmem_base,
                                  abort_flag, epi_flag, epi_flag + 2, warp, lane);
  } else if (warp == 0) {
    // ---------------- TMA producer (one thread) ----------------
    if (lane == 0) {
      for (int j = 0; j < p.n_jobs; ++j)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.m[j]))
                     : "memory");
      // stage / phase advance incrementally: no division in the per-stage path
      int stage = 0;
      uint32_t phase = 0;
      int64_t issued = 0;
      bool ok = true;
      for (int64_t item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
        const Item it = decode_item(p, item);
        const KJob &jb = p.job[it.job];
        const CUtensorMap *map = &maps.m[it.job];
        // operand rows: [chan][kb][row][128 B]; block kb of tile I starts at row
        // (c * KB + kb) * n_rows + I * 128
        const int n_rows = jb.n_tiles * kTile;
        const TileAt<BITS> tA(it.c, it.I, jb.kb, n_rows), tB(it.c, it.J, jb.kb, n_rows);
        const bool diag = it.I == it.J;
        const uint32_t blk_bytes = diag ? kTileBytes : 2 * kTileBytes;  // TMA bytes per block
        // warm L2 for the first blocks of the item; later blocks are prefetched
        // `prefetch` blocks ahead of their TMA load (first-touch misses go to DRAM)
        const int pf = p.prefetch;
        for (int kb = 0; kb < pf && kb < jb.kb; ++kb) {
          tma_prefetch_2d(map, tA.x, tA.y + kb * tA.step);
          if (!diag) tma_prefetch_2d(map, tB.x, tB.y + kb * tB.step);
        }
        for (int kb = 0; kb < jb.kb; kb += Sh::kps) {
          const int nb = min(Sh::kps, jb.kb - kb);
          if (pf > 0)
            for (int j = 0; j < nb && kb + j + pf < jb.kb; ++j) {
              tma_prefetch_2d(map, tA.x, tA.y + (kb + j + pf) * tA.step);
              if (!diag) tma_prefetch_2d(map, tB.x, tB.y + (kb + j + pf) * tB.step);
            }
          if (!mbar_wait(empty(stage), phase ^ 1u, abort_flag, tmo)) {
            raise_timeout(abort_flag, p.status);
            ok = false;
            break;
          }
          const uint32_t a = smem_base + (uint32_t)stage * kStageBytes;
          mbar_arrive_expect_tx(full(stage), (uint32_t)nb * blk_bytes);
          for (int j = 0; j < nb; ++j) {
            const uint32_t aj = a + (uint32_t)(j * Sh::block_bytes);
            tma_load_2d(aj, map, tA.x, tA.y + (kb + j) * tA.step, full(stage));
            if (!diag) tma_load_2d(aj + kTileBytes, map, tB.x, tB.y + (kb + j) * tB.step, full(stage));
          }
          ++issued;
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // wait (bounded) until every copy this thread issued has landed
      int st = stage;
      uint32_t ph = phase;
      for (int64_t k = 0; k < issued && k < S; ++k) {
        if (--st < 0) {
          st = S - 1;
          ph ^= 1u;
        }
        mbar_wait(full(st), ph, nullptr, tmo);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer (one thread) ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc<BITS>(false, WIDE ? 2 * kTile : kTile);
      int stage = 0;
      uint32_t phase = 0;
      uint32_t seg = 0;
      bool ok = true;
      for (int64_t item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
        const Item it = decode_item(p, item);
        const KJob &jb = p.job[it.job];
        const int F = jb.flush_blocks, KB = jb.kb;
        const bool diag = it.I == it.J;
        int in_seg = 0;  // blocks already accumulated in the current segment
        for (int kb = 0; kb < KB; kb += Sh::kps) {
          const int nb = min(Sh::kps, KB - kb);
          if (!mbar_wait(full(stage), phase, abort_flag, tmo) ||
              (WIDE && !mbar_wait(bfull(stage), phase, abort_flag, tmo))) {
            raise_timeout(abort_flag, p.status);
            ok = false;
            break;
          }
          tc_fence_after();
          for (int j = 0; j < nb; ++j) {
            const bool seg_start = in_seg == 0;
            const uint32_t buf = seg & 1u;
            if (seg_start) {
              if (!mbar_wait(tempty(buf), ((seg >> 1) & 1u) ^ 1u, abort_flag, tmo)) {
                raise_timeout(abort_flag, p.status);
                ok = false;
                break;
              }
              tc_fence_after();
            }
            const uint32_t a = smem_base + (uint32_t)stage * kStageBytes + (uint32_t)(j * Sh::block_bytes);
            // descriptors of the 32-byte K slices: start address advances by 2 units of 16 B
            const uint64_t da = Op<BITS>::desc(a);
            const uint64_t db = diag ? da : Op<BITS>::desc(a + kTileBytes);
            const uint32_t d_re = tmem_base + buf * kAccCols;
            const uint32_t acc0 = seg_start ? 0u : 1u;
            if constexpr (WIDE) {
              // B = [A_J ; B'_J], B'_J holding -im_J in place of re_J and re_J in
              // place of im_J: columns 0..127 give Re, 128..255 give Im
              using O = Op<BITS>;
              tc_mma<BITS>(d_re, da + O::re0, db + O::re0, idesc, acc0);
              tc_mma<BITS>(d_re, da + O::re1, db + O::re1, idesc, 1u);
              tc_mma<BITS>(d_re, da + O::im0, db + O::im0, idesc, 1u);
              tc_mma<BITS>(d_re, da + O::im1, db + O::im1, idesc, 1u);
            } else {
              narrow_block<BITS>(d_re, d_re + kTile, da, db, acc0);
            }
            if (++in_seg == F || kb + j == KB - 1) {
              tc_commit(tfull(buf));
              ++seg;
              in_seg = 0;
            }
          }
          if (!ok) break;
          tc_commit(empty(stage));
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // no MMA may be in flight when tensor memory is freed
      tc_commit(drain);
      mbar_wait(drain, 0, nullptr, tmo);
    }
    __syncwarp();
  } else if (WIDE && warp < Sh::epi0) {
    // ---------------- B' builder (wide shape) ----------------
    // B'_J holds -im_J where A_J holds re_J and re_J where it holds im_J.
    // 8-bit (K-major): B' row r = [-im_j | re_j]: 16-byte chunk c of the
    //   (128-byte swizzled) row is chunk c ^ 4 of the A_J row, negated for c < 4.
    // 4-bit (MN-major): B' row r is A_J row (r + 64) mod 128 (the other plane,
    //   same swizzle phase since r and r + 64 agree mod 8), negated for r < 64.
    // Thread t copies chunk c = t & 7 of rows (t >> 3) + 8m, m = 0..15; all 16
    // loads are issued before the stores.
    constexpr uint32_t neg = BITS == 8 ? 0x80008000u : 0x80808080u;  // packed sign bits
    const int ct = (warp - 2) * 32 + lane;                           // 0 .. 63
    const int c = ct & 7, r0 = ct >> 3, sw = r0 & 7;
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
      const Item it = decode_item(p, item);
      const KJob &jb = p.job[it.job];
      const bool diag = it.I == it.J;
      for (int kb = 0; kb < jb.kb; ++kb) {
        if (!warp_wait(full(stage), phase, abort_flag, tmo, lane)) {
          if (lane == 0) raise_timeout(abort_flag, p.status);
          ok = false;
          break;
        }
        const uint8_t *src = smem + (size_t)stage * kStageBytes + (diag ? 0 : kTileBytes);
        uint8_t *dst = smem + (size_t)stage * kStageBytes + (diag ? kTileBytes : 2 * kTileBytes);
        uint4 v[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          const int r = r0 + 8 * m;
          const int so = Op<BITS>::mn ? ((r + 64) & 127) * kRowBytes + (c << 4)
                                      : r * kRowBytes + (((c ^ 4) ^ sw) << 4);
          v[m] = *reinterpret_cast<const uint4 *>(src + so);
        }
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          const int r = r0 + 8 * m;
          const uint32_t flip = (Op<BITS>::mn ? r < 64 : c < 4) ? neg : 0u;
          const int doff = Op<BITS>::mn ? r * kRowBytes + (c << 4) : r * kRowBytes + ((c ^ sw) << 4);
          uint4 w = v[m];
          w.x ^= flip;
          w.y ^= flip;
          w.z ^= flip;
          w.w ^= flip;
          *reinterpret_cast<uint4 *>(dst + doff) = w;
        }
        // generic-proxy writes -> visible to the tensor core's async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(bfull(stage));
        if (++stage == S) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
  } else {
    // ---------------- epilogue: flush + integration dump ----------------
    const int q = warp & 3;               // tensor-memory lane quadrant of this warp
    const int h = (warp - Sh::epi0) >> 2;  // column half: local columns [64h, 64h + 64)
    uint32_t seg = 0;
    bool ok = true;
    for (int64_t item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
      const Item it = decode_item(p, item);
      const KJob &jb = p.job[it.job];
      const int F = jb.flush_blocks;
      const int n_seg = (jb.kb + F - 1) / F;
      uint32_t tot[128];  // [0,64): re of columns 64h+k, [64,128): im
#pragma unroll
      for (int k = 0; k < 128; ++k) tot[k] = 0u;
      for (int sidx = 0; sidx < n_seg; ++sidx) {
        const uint32_t buf = seg & 1u;
        // one thread polls the accumulator barrier; the other epilogue warps
        // sleep on a named barrier instead of spinning (their issue slots are
        // shared with the MMA and producer warps).  The result goes through a
        // two-entry flag so every epilogue warp takes the same branch.
        if (warp == Sh::epi0 && lane == 0) {
          const bool got = mbar_wait(tfull(buf), (seg >> 1) & 1u, abort_flag, tmo);
          if (!got) raise_timeout(abort_flag, p.status);
          epi_flag[seg & 1u] = got ? 1 : 0;
        }
        named_bar_sync(1, 8 * 32);
        if (!epi_flag[seg & 1u]) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t trow = tmem_base + ((uint32_t)(q * 32) << 16) + buf * kAccCols;
#pragma unroll
        for (int chunk = 0; chunk < 4; ++chunk) {
          const uint32_t col = chunk < 2 ? (uint32_t)(64 * h + 32 * chunk)
                                         : (uint32_t)(kTile + 64 * h + 32 * (chunk - 2));
          uint32_t v[32];
          tc_ld32(trow + col, v);
          tc_wait_ld();
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            if constexpr (KIND == MWAX_KIND_EXACT) {
              const int x = __float2int_rn(__uint_as_float(v[k]));
              tot[chunk * 32 + k] = (uint32_t)((int)tot[chunk * 32 + k] + x);
            } else {
              tot[chunk * 32 + k] = v[k];
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        // (test hook: withholding one release makes the MMA warp's bounded
        // wait for that accumulator run out -> MWAX_ERR_TIMEOUT, clean exit)
        if (lane == 0 && (int)seg != p.withhold_seg) mbar_arrive(tempty(buf));
        ++seg;
      }
      if (!ok) break;
      // packed lower-triangle store: row i, columns j in [J*128 + 64h, +64), j <= i
      const int i = it.I * kTile + q * 32 + lane;
      if (i < jb.n_inputs) {
        const int64_t rowb = (int64_t)i * (i + 1) / 2;
        uint32_t *out = reinterpret_cast<uint32_t *>(jb.out) + (int64_t)it.c * jb.n_bl * 2;
#pragma unroll
        for (int k = 0; k < 64; ++k) {
          const int j = it.J * kTile + 64 * h + k;
          if (j < jb.n_inputs && j <= i) {
            const uint2 val = make_uint2(tot[k], tot[64 + k]);
            *reinterpret_cast<uint2 *>(out + 2 * (rowb + j)) = val;
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// ---- exactness check of a one-segment pass ---------------------------------
// Every product term of a pair (i, j) is bounded by |x_i(t)| |x_j(t)|, so by
// Cauchy-Schwarz every partial sum the tensor core forms for that pair, in any
// order, is at most sqrt(E_i E_j) <= max(E_i, E_j) with E_i = sum_t |x_i(t)|^2
// = Re V_ii.  A channel whose largest auto-correlation stayed below 2^24 was
// therefore accumulated exactly in FP32.  Otherwise the FP32 auto sum, a sum
// of non-negative terms, cannot have ended below 2^24 either (rounding is
// monotonic and 2^24 is representable), so the test below catches every
// channel that left the exact window.  One CTA per channel; flagged channels
// are appended to bad[1..] (count in bad[0]).
__global__ void __launch_bounds__(256) exact_check_kernel(const int32_t *out, int64_t n_bl,
                                                          int n_inputs, int32_t *bad,
                                                          unsigned long long *recomputed) {
  // recomputed[0]: running total for the caller, recomputed[1]: this call
  const int c = blockIdx.x;
  const int32_t *o = out + (int64_t)c * n_bl * 2;
  uint32_t m = 0;
  for (int i = threadIdx.x; i < n_inputs; i += blockDim.x)
    m = max(m, (uint32_t)__ldg(o + 2 * ((int64_t)i * (i + 1) / 2 + i)));  // negative -> huge
  m = __reduce_max_sync(0xffffffffu, m);
  __shared__ uint32_t wmax[8];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, wmax[w]);
    if (m >= (1u << 24)) {
      bad[1 + atomicAdd(bad, 1)] = c;
      atomicAdd(recomputed, 1ull);
      atomicAdd(recomputed + 1, 1ull);
    }
  }
}

// ---- host side ------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

template <int BITS, int KIND, int MODE>
cudaError_t set_smem_attr(int bytes) {
  return cudaFuncSetAttribute(correlate_tc_kernel<BITS, KIND, MODE>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int MODE>
cudaError_t prepare_shape(int sample_bits, int kind, int bytes) {
  if (sample_bits == 4) return set_smem_attr<4, MWAX_KIND_EXACT, MODE>(bytes);
  if (kind == MWAX_KIND_FP16) return set_smem_attr<8, MWAX_KIND_FP16, MODE>(bytes);
  return set_smem_attr<8, MWAX_KIND_EXACT, MODE>(bytes);
}

template <int MODE>
void launch_shape(int sample_bits, int kind, int grid, int smem, cudaStream_t s, const KMaps &maps,
                  const KParams &kp) {
  const int threads = Shape<MODE>::warps * 32;
  if (sample_bits == 4)
    correlate_tc_kernel<4, MWAX_KIND_EXACT, MODE><<<grid, threads, smem, s>>>(maps, kp);
  else if (kind == MWAX_KIND_FP16)
    correlate_tc_kernel<8, MWAX_KIND_FP16, MODE><<<grid, threads, smem, s>>>(maps, kp);
  else
    correlate_tc_kernel<8, MWAX_KIND_EXACT, MODE><<<grid, threads, smem, s>>>(maps, kp);
}

int4 encode_item(int job, uint32_t type, int c0, int c1, int I0, int J0, int I1, int J1,
                 int split = 0, int n_split = 1) {
  const uint32_t z = (uint32_t)job | type << 8 | (uint32_t)I0 << 16 | (uint32_t)J0 << 24;
  const uint32_t w = (uint32_t)I1 | (uint32_t)J1 << 8 | (uint32_t)split << 16 | (uint32_t)n_split << 24;
  return make_int4(c0, c1, (int)z, (int)w);
}

}  // namespace

int correlate_tc_max_stages(int mode) {
  return mode == kModeWide ? Shape<kModeWide>::max_stages
         : mode == kModePair ? Shape<kModePair>::max_stages
         : mode == kModePairFused ? Shape<kModePairFused>::max_stages
                                  : Shape<kModeNarrow>::max_stages;
}

int correlate_tc_smem_bytes(int stages, int mode) {
  const int stage_bytes = mode == kModeWide ? Shape<kModeWide>::stage_bytes
                          : mode == kModePair ? Shape<kModePair>::stage_bytes
                          : mode == kModePairFused ? Shape<kModePairFused>::stage_bytes
                                                   : Shape<kModeNarrow>::stage_bytes;
  const int epi_bytes = mode == kModePair ? Shape<kModePair>::epi_bytes
                        : mode == kModePairFused ? Shape<kModePairFused>::epi_bytes
                                                 : 0;
  return 1024 + stages * stage_bytes + epi_bytes + (3 * stages + 5) * 8 + 32;
}

cudaError_t correlate_tc_prepare(int sample_bits, int kind, int stages, int mode) {
  const int bytes = correlate_tc_smem_bytes(stages, mode);
  if (mode == kModeWide) return prepare_shape<kModeWide>(sample_bits, kind, bytes);
  if (mode == kModePair) return prepare_shape<kModePair>(sample_bits, kind, bytes);
  if (mode == kModePairFused)
    return sample_bits == 4 && kind == MWAX_KIND_EXACT
               ? set_smem_attr<4, MWAX_KIND_EXACT, kModePairFused>(bytes)
               : cudaErrorInvalidValue;
  return prepare_shape<kModeNarrow>(sample_bits, kind, bytes);
}

cudaError_t launch_exact_check(const int32_t *out, int64_t n_bl, int n_inputs, int n_chan,
                               int32_t *bad, unsigned long long *recomputed, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int32_t), s);
  if (e != cudaSuccess || n_chan <= 0) return e;
  exact_check_kernel<<<n_chan, 256, 0, s>>>(out, n_bl, n_inputs, bad, recomputed);
  return cudaGetLastError();
}

bool pair_mode_supported(const TcJob *jobs, int n_jobs) {
  for (int j = 0; j < n_jobs; ++j)
    if (jobs[j].kb > jobs[j].flush_blocks || jobs[j].n_tiles > 255 || jobs[j].k_split < 1 ||
        jobs[j].k_split > jobs[j].kb || jobs[j].k_split > 8 || jobs[j].kb >= (1 << 28))
      return false;
  return n_jobs >= 1 && n_jobs <= kMaxJobs;
}

bool fused_pair_supported(const TcJob *jobs, int n_jobs, int sample_bits, int kind) {
  if (sample_bits != 4 || kind != MWAX_KIND_EXACT) return false;
  for (int j = 0; j < n_jobs; ++j)
    if (jobs[j].n_inputs % 16 != 0 || jobs[j].n_time < 1 ||
        (jobs[j].op && (reinterpret_cast<uintptr_t>(jobs[j].op) & 15u) != 0))
      return false;
  return true;
}

// Channel by channel, row I of the tile triangle gives the shared items
// (I; J, J+1) for J = 0, 2, ... while J+1 <= I, and, when I+1 is odd, its
// diagonal pair (I, I) is left over; consecutive leftovers (in the same or the
// next channel of the job) form a two-diagonal item, and a last unmatched one
// a single item.  Items of one channel are adjacent, so the CTAs working on a
// channel at the same time share its operand tiles in L2.  A job with
// k_split > 1 gives every item k_split times, one per time range.
void build_pair_items(const TcJob *jobs, int n_jobs, std::vector<int4> &items) {
  items.clear();
  for (int jn = 0; jn < n_jobs; ++jn) {
    const TcJob &job = jobs[jn];
    const int S = job.k_split;
    auto push = [&](uint32_t type, int c0, int c1, int I0, int J0, int I1, int J1) {
      for (int sp = 0; sp < S; ++sp)
        items.push_back(encode_item(jn, type, c0, c1, I0, J0, I1, J1, sp, S));
    };
    bool pending = false;
    int pc = 0, pI = 0;
    for (int c = 0; c < job.n_chan; ++c)
      for (int I = 0; I < job.n_tiles; ++I) {
        for (int J = 0; J + 1 <= I; J += 2) push(kItemShared, c, c, I, J, I, J + 1);
        if ((I + 1) % 2 == 1) {
          if (pending) {
            push(kItemTwoDiag, pc, c, pI, pI, I, I);
            pending = false;
          } else {
            pending = true;
            pc = c;
            pI = I;
          }
        }
      }
    if (pending) push(kItemOne, pc, pc, pI, pI, 0, 0);
  }
}

}  // namespace mwax

extern "C" int64_t mwax_pair_work_list(int n_tiles, int n_chan, int32_t *items, int64_t capacity) {
  if (n_tiles < 1 || n_tiles > 255 || n_chan < 1 || capacity < 0 || (capacity > 0 && !items))
    return -1;
  mwax::TcJob job{};
  job.n_tiles = n_tiles;
  job.n_chan = n_chan;
  std::vector<int4> list;
  mwax::build_pair_items(&job, 1, list);
  const int64_t n = (int64_t)list.size();
  for (int64_t k = 0; k < n && k < capacity; ++k) {
    const uint32_t z = (uint32_t)list[k].z, w = (uint32_t)list[k].w;
    int32_t *o = items + 7 * k;
    o[0] = (int32_t)((z >> 8) & 0xFFu);  // type
    o[1] = list[k].x;                    // c0
    o[2] = (int32_t)((z >> 16) & 0xFFu);  // I0
    o[3] = (int32_t)(z >> 24);           // J0
    o[4] = list[k].y;                    // c1
    o[5] = (int32_t)(w & 0xFFu);          // I1
    o[6] = (int32_t)((w >> 8) & 0xFFu);   // J1
  }
  return n;
}

namespace mwax {

cudaError_t launch_correlate_tc(const TcJob *jobs, int n_jobs, const TcLaunch &cfg,
                                cudaStream_t s) {
  if (n_jobs < 1 || n_jobs > kMaxJobs) return cudaErrorInvalidValue;
  if (cfg.mode < kModeNarrow || cfg.mode > kModePairFused) return cudaErrorInvalidValue;
  if (cfg.stages < 2 || cfg.stages > correlate_tc_max_stages(cfg.mode)) return cudaErrorInvalidValue;
  const bool pair = cfg.mode == kModePair || cfg.mode == kModePairFused;
  const bool fused = cfg.mode == kModePairFused;
  if (pair && (!pair_mode_supported(jobs, n_jobs) || !cfg.items || cfg.n_items < 0))
    return cudaErrorInvalidValue;
  if (fused && !fused_pair_supported(jobs, n_jobs, cfg.sample_bits, cfg.kind))
    return cudaErrorInvalidValue;
  if ((cfg.chan_map || cfg.n_chan_dev) &&
      (pair || n_jobs != 1 || !cfg.chan_map || !cfg.n_chan_dev))
    return cudaErrorInvalidValue;
  PFN_cuTensorMapEncodeTiled_v12000 encode = fused ? nullptr : get_encode_fn();
  if (!fused && !encode) return cudaErrorNotSupported;
  KMaps maps;
  KParams kp;
  memset(&maps, 0, sizeof(maps));
  memset(&kp, 0, sizeof(kp));
  int64_t items = 0;
  for (int j = 0; j < n_jobs; ++j) {
    const TcJob &job = jobs[j];
    if (job.flush_blocks < 1 || job.kb < 1 || job.n_tiles < 1) return cudaErrorInvalidValue;
    if (fused && !job.op) return cudaErrorInvalidValue;
    KJob &kj = kp.job[j];
    kj.out = job.out;
    kj.item_begin = items;
    kj.n_bl = job.n_bl;
    kj.n_inputs = job.n_inputs;
    kj.n_tiles = job.n_tiles;
    kj.n_pairs = job.n_pairs;
    kj.kb = job.kb;
    kj.flush_blocks = job.flush_blocks;
    kj.n_time = job.n_time;
    kj.volt = fused ? job.op : nullptr;  // the fused pair mode reads the packed samples
    items += (int64_t)job.n_chan * job.n_pairs;
    if (fused) continue;  // no operand tiles, no tensor map
    // 8-bit: [chan][kb][row][128 B] viewed as rows of 128 bytes;
    // 4-bit: [chan][kb][128 rows][n_rows bytes]; the box is one 16 KB tile
    const cuuint64_t n_rows = (cuuint64_t)job.n_tiles * kTile;
    const bool mn = cfg.sample_bits == 4;
    const cuuint64_t rows = (cuuint64_t)job.n_chan * job.kb * (mn ? (cuuint64_t)kTile : n_rows);
    if (rows > 0x7FFFFFFFull) return cudaErrorInvalidValue;  // TMA row coordinate is int32
    cuuint64_t dims[2] = {mn ? n_rows : (cuuint64_t)kRowBytes, rows};
    cuuint64_t strides[1] = {mn ? n_rows : (cuuint64_t)kRowBytes};
    cuuint32_t box[2] = {(cuuint32_t)kRowBytes, (cuuint32_t)kTile};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&maps.m[j], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                        const_cast<uint8_t *>(job.op), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  if (pair) {
    kp.items = cfg.items;
    items = cfg.n_items;
  }
  kp.chan_map = cfg.chan_map;  // (items stays the bound for all n_chan channels)
  kp.n_chan_dev = cfg.n_chan_dev;
  kp.status = cfg.status;
  kp.n_items = items;
  kp.timeout_ns = cfg.timeout_ns;
  kp.n_jobs = n_jobs;
  kp.stages = cfg.stages;
  kp.prefetch = cfg.prefetch;
  kp.withhold_seg = cfg.withhold_seg;
  if (items <= 0) return cudaSuccess;
  const int grid = (int)(items < cfg.grid ? items : cfg.grid);
  const int smem = correlate_tc_smem_bytes(cfg.stages, cfg.mode);
  if (cfg.mode == kModeWide)
    launch_shape<kModeWide>(cfg.sample_bits, cfg.kind, grid, smem, s, maps, kp);
  else if (cfg.mode == kModePair)
    launch_shape<kModePair>(cfg.sample_bits, cfg.kind, grid, smem, s, maps, kp);
  else if (fused)
    correlate_tc_kernel<4, MWAX_KIND_EXACT, kModePairFused>
        <<<grid, Shape<kModePairFused>::warps * 32, smem, s>>>(maps, kp);
  else
    launch_shape<kModeNarrow>(cfg.sample_bits, cfg.kind, grid, smem, s, maps, kp);
  return cudaGetLastError();
}

}  // namespace mwax
