// k_unpack.cu -- packed complex samples -> tensor-core operand tiles.
//
// Input  volt[chan][t][input]: 4+4-bit (one byte, low nibble re) or 8+8-bit
//        (re byte, im byte) two's-complement samples.
// Output, per channel and block of S time samples, the operand tiles the
//        correlator's MMAs read, holding the samples as exact small floats:
//   8-bit samples (S = 32, IEEE binary16, exact for |v| <= 2048), K-major:
//        op[chan][kb][row][128 B], one 128-byte row per input (rows >= N
//        zero up to a multiple of the 128-input tile), contiguous across
//        inputs, holding [ re(t0) .. re(t0+31) | im(t0) .. im(t0+31) ]: one
//        row of a 128-byte-swizzled K-major shared-memory tile, 16 KB per
//        tile and time block.  The transpose goes through shared memory.
//   4-bit samples (S = 64, FP8 E4M3, exact for |v| <= 16), MN-major:
//        op[chan][kb][plane][s][n_rows] bytes, n_rows = 128 x tiles: row
//        (plane 0, s) holds the re codes of every input at sample 64 kb + s
//        (inputs contiguous, the order they arrive in), row (plane 1, s) the
//        im codes.  One tile of one time block is a 128 x 128-byte box (rows:
//        64 re, then 64 im samples; columns: the tile's 128 inputs), the
//        MN-major 128-byte-swizzled tile the MMAs read.  No transpose is
//        needed: a register-only streaming kernel converts each byte's two
//        nibbles in place.
// Time samples past T and inputs past N are zero (the plan zeroes its
// operand buffers once; these positions are never written): zeros add
// nothing to any product.
//
// HBM-bound: loads and stores are 16-byte vectors where the row lengths allow.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "mwax_internal.h"
#include "mwax_nib4.h"

namespace mwax {
namespace {

constexpr int kRowsPerCta = 64;
constexpr int kStride = kRowBytes + 16;  // shared row stride (keeps 16-byte alignment)

// 8-bit samples, shared-memory transpose (fallback for shapes the tile and
// line kernels do not take).
__global__ void __launch_bounds__(256) unpack8_kernel(const uint8_t *__restrict__ volt,
                                                      uint8_t *__restrict__ op, int N, int T,
                                                      int n_rows, int kb, int64_t chan0) {
  constexpr int S = 32;
  __shared__ __align__(16) uint8_t sblk[kRowsPerCta][kStride];

  const int tb = blockIdx.y;        // time block
  const int r0 = blockIdx.x * kRowsPerCta;
  const int c = blockIdx.z;         // channel within the group
  const int tid = threadIdx.x;
  const int64_t chan = chan0 + c;

  for (int k = tid; k < S * kRowsPerCta; k += 256) {
    const int t = k / kRowsPerCta, l = k % kRowsPerCta;
    const int i = r0 + l, tg = tb * S + t;
    const bool valid = i < N && tg < T;
    short2 v = make_short2(0, 0);
    if (valid) {
      const char2 sv = reinterpret_cast<const char2 *>(volt)[(chan * T + tg) * (int64_t)N + i];
      v = make_short2(sv.x, sv.y);
    }
    const __half hr = __short2half_rn(v.x), hi = __short2half_rn(v.y);
    *reinterpret_cast<__half *>(&sblk[l][2 * t]) = hr;
    *reinterpret_cast<__half *>(&sblk[l][2 * (S + t)]) = hi;
  }
  __syncthreads();
  for (int k = tid; k < kRowsPerCta * 8; k += 256) {
    const int row = k >> 3, piece = k & 7;
    const int i = r0 + row;
    if (i >= n_rows) continue;
    const uint4 v = *reinterpret_cast<const uint4 *>(&sblk[row][piece * 16]);
    uint8_t *dst = op + (((int64_t)c * kb + tb) * n_rows + i) * kRowBytes + piece * 16;
    *reinterpret_cast<uint4 *>(dst) = v;
  }
}

// ---- full-line path (8-bit) -------------------------------------------------------
// Each thread converts two inputs x one 32-sample block (two full 128-byte
// rows), so every store covers complete 128-byte lines, while every warp load
// is one contiguous line (consecutive threads take consecutive inputs at the
// same time sample).  Requires N even for aligned 4-byte loads.

// int8 in the low byte of each 16-bit lane -> binary16: 0x6400 | (v ^ 0x80)
// encodes 1024 + v + 128 exactly; subtracting 1152 leaves v.
__device__ __forceinline__ uint32_t s8pair_to_h2(uint32_t lanes) {
  const uint32_t t = ((lanes & 0x00FF00FFu) ^ 0x00800080u) | 0x64006400u;
  __half2 h = *reinterpret_cast<const __half2 *>(&t);
  const __half2 bias = __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480));
  h = __hsub2(h, bias);
  return *reinterpret_cast<uint32_t *>(&h);
}

// Inputs i0, i0+1 of time block tb of channel c (of the group starting at chan0).
__device__ __forceinline__ void unpack8_task(const uint8_t *__restrict__ volt,
                                             uint8_t *__restrict__ op, int N, int T, int n_rows,
                                             int kb, int64_t chan0, int c, int tb, int i0) {
  const int64_t chan = chan0 + c;
  uint32_t w[32];  // (re_a, im_a, re_b, im_b) at t = tb*32 + r
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int t = tb * 32 + r;
    w[r] = (i0 < N && t < T)
               ? __ldg(reinterpret_cast<const uint32_t *>(volt + ((chan * T + t) * (int64_t)N + i0) * 2))
               : 0u;
  }
  uint8_t *row_a = op + (((int64_t)c * kb + tb) * n_rows + i0) * kRowBytes;
  uint8_t *row_b = row_a + kRowBytes;
#pragma unroll
  for (int q = 0; q < 4; ++q) {  // 16-byte chunk q: samples 8q .. 8q+7
    uint32_t ra[4], ia[4], rb[4], ib[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t x = w[8 * q + 2 * k], y = w[8 * q + 2 * k + 1];
      ra[k] = s8pair_to_h2(__byte_perm(x, y, 0x4400));
      ia[k] = s8pair_to_h2(__byte_perm(x, y, 0x5511));
      rb[k] = s8pair_to_h2(__byte_perm(x, y, 0x6622));
      ib[k] = s8pair_to_h2(__byte_perm(x, y, 0x7733));
    }
    *reinterpret_cast<uint4 *>(row_a + 16 * q) = make_uint4(ra[0], ra[1], ra[2], ra[3]);
    *reinterpret_cast<uint4 *>(row_a + 64 + 16 * q) = make_uint4(ia[0], ia[1], ia[2], ia[3]);
    *reinterpret_cast<uint4 *>(row_b + 16 * q) = make_uint4(rb[0], rb[1], rb[2], rb[3]);
    *reinterpret_cast<uint4 *>(row_b + 64 + 16 * q) = make_uint4(ib[0], ib[1], ib[2], ib[3]);
  }
}

__global__ void __launch_bounds__(128) unpack8_line_kernel(const uint8_t *__restrict__ volt,
                                                           uint8_t *__restrict__ op, int N, int T,
                                                           int n_rows, int kb, int64_t chan0) {
  const int i0 = 2 * (blockIdx.x * 128 + threadIdx.x);
  if (i0 >= n_rows) return;
  unpack8_task(volt, op, N, T, n_rows, kb, chan0, blockIdx.z, blockIdx.y, i0);
}

// Persistent form: a few CTAs loop over all tasks (input pair fastest).  Its
// dynamic shared-memory request (unused) keeps it off SMs that hold a
// correlate CTA, so the two kernels run side by side on disjoint SMs.
__global__ void __launch_bounds__(512) unpack8_persist_kernel(const uint8_t *__restrict__ volt,
                                                              uint8_t *__restrict__ op, int N,
                                                              int T, int n_rows, int kb,
                                                              int64_t chan0, int n_chan) {
  const int pairs = n_rows / 2;
  const int64_t tasks = (int64_t)n_chan * kb * pairs;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < tasks;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int ip = (int)(k % pairs);
    const int64_t r = k / pairs;
    unpack8_task(volt, op, N, T, n_rows, kb, chan0, (int)(r / kb), (int)(r % kb), 2 * ip);
  }
}

// ---- 4-bit samples: MN-major streaming unpack --------------------------------------
// One thread takes VEC consecutive inputs (16, 4 or 1 bytes of samples, as N
// allows aligned loads) of one (channel, sample) row at a time and writes
// their re codes to the re plane and their im codes to the im plane of the
// row's time block: a pure element-wise conversion, coalesced on both sides.
// Threads of a CTA cover whole rows (rows per CTA step = 256 / (N / VEC)) or,
// for long rows, stride along one row; the (channel, sample) position
// advances incrementally, without a division per element.  U rows are loaded
// before any is converted, for memory-level parallelism.  The kernel uses no
// shared memory; a nonzero dynamic request (set-aside SMs of the overlapped
// pipeline) only keeps it off SMs that hold a correlate CTA.
#ifndef MWAX_U4_ROWS
#define MWAX_U4_ROWS 2  // rows in flight per thread with 16-byte units (more with narrower ones)
#endif
#ifndef MWAX_U4_CTAS_PER_SM
#define MWAX_U4_CTAS_PER_SM 8
#endif
template <int VEC>
__global__ void __launch_bounds__(256) unpack4_mn_kernel(const uint8_t *__restrict__ volt,
                                                         uint8_t *__restrict__ op, int N, int T,
                                                         int n_rows, int kb, int64_t chan0,
                                                         int n_chan) {
  constexpr int U = VEC == 16 ? MWAX_U4_ROWS : VEC == 4 ? 2 * MWAX_U4_ROWS : 4 * MWAX_U4_ROWS;
  using Vec = typename std::conditional<VEC == 16, uint4, typename std::conditional<VEC == 4, uint32_t, uint8_t>::type>::type;
  const int upr = N / VEC;  // units per row
  const bool long_rows = upr >= (int)blockDim.x;
  const int rpb = long_rows ? 1 : (int)blockDim.x / upr;
  const int r_off = long_rows ? 0 : (int)threadIdx.x / upr;
  const int g0 = long_rows ? (int)threadIdx.x : (int)threadIdx.x - r_off * upr;
  const int gstep = long_rows ? (int)blockDim.x : upr;
  if (r_off >= rpb) return;
  const int64_t rows = (int64_t)n_chan * T;
  const int64_t rstride = (int64_t)gridDim.x * rpb;
  const int64_t plane = (int64_t)64 * n_rows;
  const int64_t dc = rstride / T;
  const int dt = (int)(rstride - dc * T);
  int64_t r = (int64_t)blockIdx.x * rpb + r_off;
  int64_t c = r / T;
  int t = (int)(r - c * T);
  auto advance = [&](int64_t &cc, int &tt) {
    tt += dt;
    cc += dc;
    if (tt >= T) {
      tt -= T;
      ++cc;
    }
  };
  for (; r < rows; r += rstride * U) {
    int64_t cu[U];
    int tu[U];
    cu[0] = c;
    tu[0] = t;
#pragma unroll
    for (int k = 1; k < U; ++k) {
      cu[k] = cu[k - 1];
      tu[k] = tu[k - 1];
      advance(cu[k], tu[k]);
    }
    for (int g = g0; g < upr; g += gstep) {
      Vec w[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        if (r + k * rstride < rows) {
          const Vec *src = reinterpret_cast<const Vec *>(volt + ((chan0 + cu[k]) * T + tu[k]) * (int64_t)N) + g;
          if constexpr (VEC == 16) {
            asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(w[k].x), "=r"(w[k].y), "=r"(w[k].z), "=r"(w[k].w)
                         : "l"(src));
          } else {
            w[k] = __ldg(src);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        if (r + k * rstride >= rows) break;
        const int tk = tu[k];
        uint8_t *dst = op + ((cu[k] * kb + (tk >> 6)) * 128 + (tk & 63)) * (int64_t)n_rows + (int64_t)g * VEC;
        if constexpr (VEC == 16) {
          const uint4 re = make_uint4(nib4_to_e4m3_f16(w[k].x), nib4_to_e4m3_f16(w[k].y),
                                      nib4_to_e4m3_f16(w[k].z), nib4_to_e4m3_f16(w[k].w));
          const uint4 im = make_uint4(nib4_to_e4m3_f16(w[k].x >> 4), nib4_to_e4m3_f16(w[k].y >> 4),
                                      nib4_to_e4m3_f16(w[k].z >> 4), nib4_to_e4m3_f16(w[k].w >> 4));
          *reinterpret_cast<uint4 *>(dst) = re;
          *reinterpret_cast<uint4 *>(dst + plane) = im;
        } else if constexpr (VEC == 4) {
          *reinterpret_cast<uint32_t *>(dst) = nib4_to_e4m3_f16(w[k]);
          *reinterpret_cast<uint32_t *>(dst + plane) = nib4_to_e4m3_f16(w[k] >> 4);
        } else {
          const uint32_t b = w[k];
          dst[0] = (uint8_t)nib4_to_e4m3_f16(b);
          dst[plane] = (uint8_t)nib4_to_e4m3_f16(b >> 4);
        }
      }
    }
    c = cu[U - 1];
    t = tu[U - 1];
    advance(c, t);
  }
}

constexpr int kPersistSmem = 64 * 1024;  // > what a correlate CTA leaves free on an SM

// ---- TMA tile path --------------------------------------------------------------

__device__ __forceinline__ uint64_t u_globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool u_wait(uint32_t bar, uint32_t parity, unsigned long long tmo) {
  const uint64_t t0 = u_globaltimer();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (u_globaltimer() - t0 > tmo) return false;
  }
}

// 8-bit samples, small footprint: one task is one 128-input tile of one
// 32-sample time block.  A 2D TMA load brings the raw box (32 samples x 256
// bytes, rows 2N bytes apart; inputs past N read as zeros) into shared memory,
// each of the 128 threads converts one operand row into a 128-byte-swizzled
// 16 KB staging tile, and one TMA tensor store writes the tile.  About 25 KB
// of shared memory and at most 80 registers a thread, so a CTA fits on an SM
// beside a resident correlate CTA and the unpack of the next channel group
// can run while the current group correlates.
constexpr int kTileThreads = 128;
constexpr int kTileRawBytes = 32 * 256;

// The raw box of one task loaded by the threads (for rows that are not whole
// 16-byte units, which TMA needs): rows grow0 .. grow0 + rows_valid - 1 of the
// [rows][row_bytes] sample array, bytes x0 .. x0 + 255 (8-bit) or 127 (4-bit)
// of each, bytes past the row read as zero; consecutive threads take
// consecutive 4-byte words of a row (row_bytes % 4 == 0).  The words of the
// next task are fetched into registers while the current one is converted.
constexpr int kRawWords = kTileRawBytes / 4 / kTileThreads;  // per thread

template <int BITS>
__device__ __forceinline__ void fetch_raw_box(const uint8_t *__restrict__ volt,
                                              uint32_t (&v)[kRawWords], int64_t row_bytes,
                                              int64_t grow0, int rows_valid, int x0) {
  constexpr int row_w = BITS == 8 ? 64 : 32;  // 4-byte words per box row
#pragma unroll
  for (int j = 0; j < kRawWords; ++j) {
    const int idx = j * kTileThreads + threadIdx.x;
    const int r = idx / row_w, x = x0 + 4 * (idx % row_w);
    v[j] = r < rows_valid && x < row_bytes
               ? __ldg(reinterpret_cast<const uint32_t *>(volt + (grow0 + r) * row_bytes + x))
               : 0u;
  }
}

__device__ __forceinline__ void put_raw_box(uint8_t *raw, const uint32_t (&v)[kRawWords]) {
#pragma unroll
  for (int j = 0; j < kRawWords; ++j) reinterpret_cast<uint32_t *>(raw)[j * kTileThreads + threadIdx.x] = v[j];
}

// TMA_IN = false: the raw box is loaded by the threads (load_raw_box).
template <bool TMA_IN>
__global__ void __launch_bounds__(kTileThreads, 6)
    unpack8_tile_kernel(const __grid_constant__ CUtensorMap in_map,
                        const __grid_constant__ CUtensorMap out_map, const uint8_t *volt, int N,
                        int T, int n_tiles, int kb, int64_t chan0, int n_chan, int32_t *status,
                        unsigned long long tmo) {
  extern __shared__ __align__(1024) uint8_t sm_base[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(sm_base) + 1023) &
                                            ~static_cast<uintptr_t>(1023));
  uint8_t *stage = sm;                // 128 rows x 128 B, swizzled
  uint8_t *raw = sm + kTile * kRowBytes;  // 32 samples x 256 B
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
  const int64_t tasks = (int64_t)n_chan * kb * n_tiles;  // tile fastest
  const int n_rows = n_tiles * kTile;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (TMA_IN)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&in_map)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&out_map)) : "memory");
  }
  __syncthreads();
  const uint32_t raw_u32 = (uint32_t)__cvta_generic_to_shared(raw);
  auto issue = [&](int64_t k) {
    const int tile = (int)(k % n_tiles);
    const int64_t cb = k / n_tiles;
    const int c = (int)(cb / kb), tb = (int)(cb % kb);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                 "r"((uint32_t)kTileRawBytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(raw_u32),
        "l"(reinterpret_cast<uint64_t>(&in_map)), "r"(tile * 256),
        "r"((int)((chan0 + c) * (int64_t)T + (int64_t)tb * 32)), "r"(b)
        : "memory");
  };
  int64_t k = blockIdx.x;
  if (TMA_IN && threadIdx.x == 0 && k < tasks) issue(k);
  uint32_t rv[kRawWords];  // thread-loaded form: the raw words of the task in hand
  auto fetch = [&](int64_t kk) {
    const int tile_l = (int)(kk % n_tiles);
    const int64_t cb_l = kk / n_tiles;
    const int c_l = (int)(cb_l / kb), tb_l = (int)(cb_l % kb);
    fetch_raw_box<8>(volt, rv, 2 * (int64_t)N, (chan0 + c_l) * (int64_t)T + (int64_t)tb_l * 32,
                       min(32, T - tb_l * 32), tile_l * 256);
  };
  if (!TMA_IN && k < tasks) fetch(k);
  uint32_t phase = 0;
  bool ok = true;
  const uint32_t stage_u32 = (uint32_t)__cvta_generic_to_shared(stage);
  const int i = threadIdx.x;  // operand row within the tile
  for (int it = 0; k < tasks && ok; k += gridDim.x, ++it) {
    if constexpr (TMA_IN) {
      if (!u_wait(b, phase, tmo)) {
        if (threadIdx.x == 0) atomicExch(status, (int32_t)MWAX_ERR_TIMEOUT);
        ok = false;
        break;
      }
      phase ^= 1u;
    } else {
      // (raw was last read before the barrier that follows the conversion)
      put_raw_box(raw, rv);
    }
    // the previous task's TMA store must have finished reading the staging tile
    if (threadIdx.x == 0 && it > 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncthreads();
    const int tile = (int)(k % n_tiles);
    const int64_t cb = k / n_tiles;
    const int c = (int)(cb / kb), tb = (int)(cb % kb);
    const int rows = min(32, T - tb * 32);  // samples of this block (the box may run into the next channel)
    uint32_t v[32];
#pragma unroll
    for (int s2 = 0; s2 < 32; ++s2)
      v[s2] = s2 < rows ? (uint32_t) * reinterpret_cast<const uint16_t *>(raw + s2 * 256 + 2 * i) : 0u;
    __syncthreads();  // raw is free: fetch the next task's box while this one is converted
    if (TMA_IN && threadIdx.x == 0 && k + gridDim.x < tasks) issue(k + gridDim.x);
    if (!TMA_IN && k + gridDim.x < tasks) fetch(k + gridDim.x);
    uint8_t *row = stage + i * kRowBytes;
    const int sw = i & 7;
#pragma unroll
    for (int q = 0; q < 4; ++q) {  // chunk q: samples 8q .. 8q+7 (re), chunk 4+q (im)
      uint32_t re4[4], im4[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const uint32_t x = v[8 * q + 2 * e], y = v[8 * q + 2 * e + 1];
        re4[e] = s8pair_to_h2(__byte_perm(x, y, 0x0400));
        im4[e] = s8pair_to_h2(__byte_perm(x, y, 0x0501));
      }
      *reinterpret_cast<uint4 *>(row + ((q ^ sw) << 4)) = make_uint4(re4[0], re4[1], re4[2], re4[3]);
      *reinterpret_cast<uint4 *>(row + (((4 + q) ^ sw) << 4)) = make_uint4(im4[0], im4[1], im4[2], im4[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      const int y0 = (int)(((int64_t)c * kb + tb) * n_rows + tile * kTile);
      asm volatile(
          "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
              reinterpret_cast<uint64_t>(&out_map)),
          "r"(0), "r"(y0), "r"(stage_u32)
          : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
  if (threadIdx.x == 0) {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (TMA_IN && !ok) u_wait(b, phase, tmo);
  }
  __syncthreads();
}

// Function attributes apply to the current device: set them once per device.
constexpr int kMaxDevices = 64;
std::mutex g_attr_mu;
bool g_attr_tile[kMaxDevices], g_attr_persist[kMaxDevices];

template <class F>
cudaError_t once_per_device(bool (&done)[kMaxDevices], F &&set) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (done[dev]) return cudaSuccess;
  e = set();
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

}  // namespace

// 4-bit samples, every path: the MN-major streaming kernel on `ctas` CTAs of
// 256 threads, with `smem` bytes of (unused) dynamic shared memory.
cudaError_t launch_unpack4(const uint8_t *volt, int n_inputs, int n_time, int n_tiles, int kb,
                           int64_t chan0, int n_chan, uint8_t *op, int ctas, int smem,
                           cudaStream_t s) {
  const int n_rows = n_tiles * kTile;
  if (n_chan <= 0) return cudaSuccess;
  if (ctas < 1 || n_inputs < 1 || n_inputs > n_rows) return cudaErrorInvalidValue;
  if (smem > 0) {
    cudaError_t e = once_per_device(g_attr_persist, [smem] {
      cudaError_t r = cudaFuncSetAttribute(unpack8_persist_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, kPersistSmem);
      for (const void *f : {reinterpret_cast<const void *>(unpack4_mn_kernel<16>),
                            reinterpret_cast<const void *>(unpack4_mn_kernel<4>),
                            reinterpret_cast<const void *>(unpack4_mn_kernel<1>)})
        if (r == cudaSuccess) r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kPersistSmem);
      return r;
    });
    if (e != cudaSuccess) return e;
    if (smem > kPersistSmem) return cudaErrorInvalidValue;
  }
  if (n_inputs % 16 == 0)
    unpack4_mn_kernel<16><<<ctas, 256, smem, s>>>(volt, op, n_inputs, n_time, n_rows, kb, chan0, n_chan);
  else if (n_inputs % 4 == 0)
    unpack4_mn_kernel<4><<<ctas, 256, smem, s>>>(volt, op, n_inputs, n_time, n_rows, kb, chan0, n_chan);
  else
    unpack4_mn_kernel<1><<<ctas, 256, smem, s>>>(volt, op, n_inputs, n_time, n_rows, kb, chan0, n_chan);
  return cudaGetLastError();
}

cudaError_t launch_unpack_persistent(const uint8_t *volt, int sample_bits, int n_inputs,
                                     int n_time, int n_tiles, int kb, int64_t chan0, int n_chan,
                                     uint8_t *op, int ctas, cudaStream_t s) {
  const int n_rows = n_tiles * kTile;
  if (n_chan <= 0) return cudaSuccess;
  if (ctas < 1 || (sample_bits == 8 && n_inputs % 2)) return cudaErrorInvalidValue;
  if (sample_bits == 4)  // kept off the correlate's SMs by its dynamic shared-memory request
    return launch_unpack4(volt, n_inputs, n_time, n_tiles, kb, chan0, n_chan, op, ctas,
                          kPersistSmem, s);
  cudaError_t e = once_per_device(g_attr_persist, [] {
    cudaError_t r = cudaFuncSetAttribute(unpack8_persist_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kPersistSmem);
    for (const void *f : {reinterpret_cast<const void *>(unpack4_mn_kernel<16>),
                          reinterpret_cast<const void *>(unpack4_mn_kernel<4>),
                          reinterpret_cast<const void *>(unpack4_mn_kernel<1>)})
      if (r == cudaSuccess) r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kPersistSmem);
    return r;
  });
  if (e != cudaSuccess) return e;
  unpack8_persist_kernel<<<ctas, 512, kPersistSmem, s>>>(volt, op, n_inputs, n_time, n_rows, kb,
                                                         chan0, n_chan);
  return cudaGetLastError();
}

// Raw rows that are whole 16-byte units: the box comes by 2D TMA; rows that
// are whole 4-byte units: the threads load it (8-bit samples).
bool unpack_tile_tma_in(int sample_bits, int n_inputs) {
  return sample_bits == 8 && n_inputs % 8 == 0;
}

// The small-footprint form (the tile kernel for 8-bit samples, the streaming
// kernel for 4-bit samples, which takes any N).
bool unpack_tile_supported(int sample_bits, int n_inputs) {
  return (sample_bits == 8 && n_inputs % 2 == 0) || sample_bits == 4;
}

int unpack_tile_smem_bytes() { return 1024 + kTile * kRowBytes + kTileRawBytes; }

cudaError_t launch_unpack_tile(const uint8_t *volt, int sample_bits, int n_inputs, int n_time,
                               int n_tiles, int kb, int64_t chan0, int n_chan, uint8_t *op,
                               int ctas, int32_t *status, unsigned long long timeout_ns,
                               cudaStream_t s) {
  if (n_chan <= 0) return cudaSuccess;
  if (ctas < 1 || !unpack_tile_supported(sample_bits, n_inputs)) return cudaErrorInvalidValue;
  if (sample_bits == 4) {
    // (`ctas` counts 128-thread tile CTAs; the streaming kernel's CTAs have 256;
    // run alone it takes MWAX_U4_CTAS_PER_SM per SM)
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return cudaErrorInvalidDevice;
    const int n = ctas >= 6 * sms ? MWAX_U4_CTAS_PER_SM * sms : (ctas > 1 ? ctas / 2 : 1);
    return launch_unpack4(volt, n_inputs, n_time, n_tiles, kb, chan0, n_chan, op, n, 0, s);
  }
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  // input: [ (chan0 + n_chan) * T rows ][ 2N bytes ], no swizzle; the box is
  // one 128-input tile of one time block: 256 B x 32 rows
  const cuuint64_t in_rows = (cuuint64_t)(chan0 + n_chan) * n_time;
  const cuuint64_t out_rows = (cuuint64_t)n_chan * kb * n_tiles * kTile;
  if (in_rows > 0x7FFFFFFFull || out_rows > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  CUtensorMap in_map, out_map;
  memset(&in_map, 0, sizeof(in_map));
  const bool tma_in = unpack_tile_tma_in(sample_bits, n_inputs);
  const cuuint64_t row_bytes = (cuuint64_t)n_inputs * 2;
  cuuint64_t idims[2] = {row_bytes, in_rows};
  cuuint64_t istr[1] = {row_bytes};
  cuuint32_t ibox[2] = {256u, 32u};
  cuuint32_t estr[2] = {1, 1};
  if (tma_in &&
      encode(&in_map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(volt), idims, istr, ibox,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  cuuint64_t odims[2] = {(cuuint64_t)kRowBytes, out_rows};
  cuuint64_t ostr[1] = {(cuuint64_t)kRowBytes};
  cuuint32_t obox[2] = {(cuuint32_t)kRowBytes, (cuuint32_t)kTile};
  if (encode(&out_map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, op, odims, ostr, obox, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int smem = unpack_tile_smem_bytes();
  cudaError_t ea = once_per_device(g_attr_tile, [smem] {
    const auto set = [&](const void *f) {
      return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    };
    cudaError_t r = set(reinterpret_cast<const void *>(unpack8_tile_kernel<true>));
    if (r == cudaSuccess) r = set(reinterpret_cast<const void *>(unpack8_tile_kernel<false>));
    return r;
  });
  if (ea != cudaSuccess) return ea;
#define MWAX_TILE_ARGS in_map, out_map, volt, n_inputs, n_time, n_tiles, kb, chan0, n_chan, status, timeout_ns
  if (tma_in)
    unpack8_tile_kernel<true><<<ctas, kTileThreads, smem, s>>>(MWAX_TILE_ARGS);
  else
    unpack8_tile_kernel<false><<<ctas, kTileThreads, smem, s>>>(MWAX_TILE_ARGS);
#undef MWAX_TILE_ARGS
  return cudaGetLastError();
}

cudaError_t launch_unpack(const uint8_t *volt, int sample_bits, int n_inputs, int n_time,
                          int n_tiles, int kb, int64_t chan0, int n_chan, uint8_t *op,
                          int variant_req, cudaStream_t s) {
  const int n_rows = n_tiles * kTile;
  if (n_chan <= 0) return cudaSuccess;
  if (sample_bits == 4) {  // one form for 4-bit samples: 8 streaming CTAs per SM
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return cudaErrorInvalidDevice;
    return launch_unpack4(volt, n_inputs, n_time, n_tiles, kb, chan0, n_chan, op,
                          MWAX_U4_CTAS_PER_SM * sms, 0, s);
  }
  // variant: 0 = automatic, 1 = shared-memory transpose, 2 = full-line;
  // MWAX_UNPACK overrides the automatic choice (tuning experiments)
  static const int env_variant = [] {
    const char *e = getenv("MWAX_UNPACK");
    return e ? atoi(e) : 0;
  }();
  const int variant = variant_req != 0 ? variant_req : env_variant;
  const bool line8 = variant == 2;
  if (line8 && n_inputs % 2 == 0 && kb <= 65535 && n_chan <= 65535) {
    dim3 g((n_rows / 2 + 127) / 128, kb, n_chan);
    unpack8_line_kernel<<<g, 128, 0, s>>>(volt, op, n_inputs, n_time, n_rows, kb, chan0);
    return cudaGetLastError();
  }
  if (kb > 65535 || n_chan > 65535) return cudaErrorInvalidValue;
  dim3 grid((n_rows + kRowsPerCta - 1) / kRowsPerCta, kb, n_chan);
  unpack8_kernel<<<grid, 256, 0, s>>>(volt, op, n_inputs, n_time, n_rows, kb, chan0);
  return cudaGetLastError();
}

}  // namespace mwax
