// k_unpack.cu -- packed complex samples -> tensor-core operand rows.
//
// Input  volt[chan][t][input]: 4+4-bit (one byte, low nibble re) or 8+8-bit
//        (re byte, im byte) two's-complement samples.
// Output op[chan][kb][row][128 B]: for every block of S time samples, one
//        128-byte row per input (rows >= N are zero padding up to a multiple
//        of the 128-input tile), contiguous across inputs, holding
//            [ re(t0) .. re(t0+S-1) | im(t0) .. im(t0+S-1) ]
//        holding the samples as exact small floats:
//            8-bit samples: S = 32, IEEE binary16 (exact for |v| <= 2048),
//            4-bit samples: S = 64, FP8 E4M3 (exact for |v| <= 16).
//        Time samples past T are zero; zeros add nothing to any product.
//
// This is the K-major operand layout of the correlator's MMAs: the 128-byte
// block is one row of a 128-byte-swizzled shared-memory tile, each MMA
// consumes a 32-byte slice of it (K = 16 halves or K = 32 E4M3 values), and
// the 128 rows of one tile and time block are one contiguous 16 KB piece.
//
// HBM-bound: loads are coalesced across inputs, the transpose goes through
// shared memory, and stores are 16-byte vectors, 8 threads per 128-byte row.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "mwax_internal.h"

namespace mwax {
namespace {

constexpr int kRowsPerCta = 64;
constexpr int kStride = kRowBytes + 16;  // shared row stride (keeps 16-byte alignment)

// E4M3 encodings of the integers -7..7, indexed by the two's-complement
// nibble.  value = 2^(e-7) (1 + m/8): 1 = 0x38, 2 = 0x40, 3 = 0x44,
// 4 = 0x48, 5 = 0x4A, 6 = 0x4C, 7 = 0x4E, 8 = 0x50; the sign is bit 7.
__constant__ uint8_t kE4M3FromNibble[16] = {0x00, 0x38, 0x40, 0x44, 0x48, 0x4A, 0x4C, 0x4E,
                                            0xD0 /* -8: outside the supported range, still exact */,
                                            0xCE, 0xCC, 0xCA, 0xC8, 0xC4, 0xC0, 0xB8};

template <int BITS>
__global__ void __launch_bounds__(256) unpack_kernel(const uint8_t *__restrict__ volt,
                                                     uint8_t *__restrict__ op, int N, int T,
                                                     int n_rows, int kb, int64_t chan0) {
  constexpr int S = BITS == 4 ? 64 : 32;
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
    if (BITS == 4) {
      uint8_t b = valid ? volt[(chan * T + tg) * (int64_t)N + i] : (uint8_t)0;
      sblk[l][t] = kE4M3FromNibble[b & 15u];
      sblk[l][S + t] = kE4M3FromNibble[b >> 4];
    } else {
      short2 v = make_short2(0, 0);
      if (valid) {
        const char2 s = reinterpret_cast<const char2 *>(volt)[(chan * T + tg) * (int64_t)N + i];
        v = make_short2(s.x, s.y);
      }
      const __half hr = __short2half_rn(v.x), hi = __short2half_rn(v.y);
      *reinterpret_cast<__half *>(&sblk[l][2 * t]) = hr;
      *reinterpret_cast<__half *>(&sblk[l][2 * (S + t)]) = hi;
    }
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

// ---- full-line paths -----------------------------------------------------------
// Each thread converts whole operand-row pieces so that every store covers
// complete 32-byte sectors (4-bit) or 128-byte lines (8-bit), while every warp
// load is one contiguous 128-byte line (consecutive threads take consecutive
// inputs at the same time sample):
//   8-bit: 2 inputs x one 32-sample block (two full 128-byte rows),
//   4-bit: 4 inputs x 32 of the 64 samples of a block (32 B of re, 32 B of im each).
// Requires N even (8-bit) or N % 4 == 0 (4-bit) for aligned 4-byte loads.

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

// Four nibbles (the low nibble of each byte of x) -> four E4M3 codes, one per
// byte.  The low three bits index an 8-entry byte table held in two registers
// (byte_perm, whose selectors use three bits per byte); the sign bit picks
// the table of negative values.  The four 3-bit indices are packed into the
// selector with one shift-or and one byte permute (l | l >> 4 holds index k
// | index k+1 << 4 in byte k).
__device__ __forceinline__ uint32_t nib4_to_e4m3(uint32_t x) {
  const uint32_t pos_lo = 0x44403800u, pos_hi = 0x4E4C4A48u;  // 0..7
  const uint32_t neg_lo = 0xCACCCED0u, neg_hi = 0xB8C0C4C8u;  // -8..-1
  const uint32_t l = x & 0x07070707u;
  const uint32_t sel = __byte_perm(l | (l >> 4), 0u, 0x0020u);
  const uint32_t p = __byte_perm(pos_lo, pos_hi, sel);
  const uint32_t n = __byte_perm(neg_lo, neg_hi, sel);
  const uint32_t m = ((x >> 3) & 0x01010101u) * 0xFFu;  // 0xFF where the nibble is negative
  return (p & ~m) | (n & m);
}

// Inputs i0..i0+3, half h (samples 32h .. 32h+31) of time block tb of channel c.
__device__ __forceinline__ void unpack4_task(const uint8_t *__restrict__ volt,
                                             uint8_t *__restrict__ op, int N, int T, int n_rows,
                                             int kb, int64_t chan0, int c, int tb, int h, int i0) {
  const int64_t chan = chan0 + c;
  uint32_t re[32], im[32];  // byte k = E4M3 of input i0+k at sample r
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int t = tb * 64 + h * 32 + r;
    const uint32_t w = (i0 < N && t < T)
                           ? __ldg(reinterpret_cast<const uint32_t *>(volt + (chan * T + t) * (int64_t)N + i0))
                           : 0u;
    re[r] = nib4_to_e4m3(w);
    im[r] = nib4_to_e4m3(w >> 4);
  }
  uint8_t *row = op + (((int64_t)c * kb + tb) * n_rows + i0) * kRowBytes + 32 * h;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t sel = (uint32_t)(k | ((k + 4) << 4));  // byte k of a, byte k of b
    uint32_t vr[8], vi[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      vr[g] = __byte_perm(__byte_perm(re[4 * g], re[4 * g + 1], sel),
                          __byte_perm(re[4 * g + 2], re[4 * g + 3], sel), 0x5410);
      vi[g] = __byte_perm(__byte_perm(im[4 * g], im[4 * g + 1], sel),
                          __byte_perm(im[4 * g + 2], im[4 * g + 3], sel), 0x5410);
    }
    uint8_t *dst = row + k * kRowBytes;
    *reinterpret_cast<uint4 *>(dst) = make_uint4(vr[0], vr[1], vr[2], vr[3]);
    *reinterpret_cast<uint4 *>(dst + 16) = make_uint4(vr[4], vr[5], vr[6], vr[7]);
    *reinterpret_cast<uint4 *>(dst + 64) = make_uint4(vi[0], vi[1], vi[2], vi[3]);
    *reinterpret_cast<uint4 *>(dst + 80) = make_uint4(vi[4], vi[5], vi[6], vi[7]);
  }
}

__global__ void __launch_bounds__(128) unpack4_line_kernel(const uint8_t *__restrict__ volt,
                                                           uint8_t *__restrict__ op, int N, int T,
                                                           int n_rows, int kb, int64_t chan0) {
  const int i0 = 4 * (blockIdx.x * 128 + threadIdx.x);
  if (i0 >= n_rows) return;
  unpack4_task(volt, op, N, T, n_rows, kb, chan0, blockIdx.z, blockIdx.y >> 1, blockIdx.y & 1, i0);
}

__global__ void __launch_bounds__(512) unpack4_persist_kernel(const uint8_t *__restrict__ volt,
                                                              uint8_t *__restrict__ op, int N,
                                                              int T, int n_rows, int kb,
                                                              int64_t chan0, int n_chan) {
  const int quads = n_rows / 4;
  const int64_t tasks = (int64_t)n_chan * kb * 2 * quads;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < tasks;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int iq = (int)(k % quads);
    const int64_t r = k / quads;  // (c, tb, h)
    const int h = (int)(r & 1);
    const int64_t r2 = r >> 1;
    unpack4_task(volt, op, N, T, n_rows, kb, chan0, (int)(r2 / kb), (int)(r2 % kb), h, 4 * iq);
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

// 4-bit samples, small footprint: one task is one 128-input tile of one
// 64-sample time block.  A 2D TMA load brings the raw box (64 samples x 128
// bytes, rows N bytes apart; inputs past N read as zeros) into shared memory;
// warp w converts samples 16w .. 16w+15, lane q the inputs 4q .. 4q+3 (four-byte
// loads, nibbles -> E4M3 by byte permutes), writing one re and one im chunk
// of each of its four rows with the row rotation that keeps the stores free
// of bank conflicts; one TMA tensor store writes the 16 KB tile.  About 25 KB
// of shared memory and 128 threads, so several CTAs share an SM and hide each
// other's load latency.
template <bool TMA_IN>
__global__ void __launch_bounds__(kTileThreads)
    unpack4_tile_kernel(const __grid_constant__ CUtensorMap in_map,
                        const __grid_constant__ CUtensorMap out_map, const uint8_t *volt, int N,
                        int T, int n_tiles, int kb, int64_t chan0, int n_chan, int32_t *status,
                        unsigned long long tmo) {
  extern __shared__ __align__(1024) uint8_t sm_base[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(sm_base) + 1023) &
                                            ~static_cast<uintptr_t>(1023));
  uint8_t *stage = sm;                    // 128 rows x 128 B, swizzled
  uint8_t *raw = sm + kTile * kRowBytes;  // 64 samples x 128 B
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
        "l"(reinterpret_cast<uint64_t>(&in_map)), "r"(tile * kTile),
        "r"((int)((chan0 + c) * (int64_t)T + (int64_t)tb * 64)), "r"(b)
        : "memory");
  };
  int64_t k = blockIdx.x;
  if (TMA_IN && threadIdx.x == 0 && k < tasks) issue(k);
  uint32_t rv[kRawWords];  // thread-loaded form: the raw words of the task in hand
  auto fetch = [&](int64_t kk) {
    const int tile_l = (int)(kk % n_tiles);
    const int64_t cb_l = kk / n_tiles;
    const int c_l = (int)(cb_l / kb), tb_l = (int)(cb_l % kb);
    fetch_raw_box<4>(volt, rv, (int64_t)N, (chan0 + c_l) * (int64_t)T + (int64_t)tb_l * 64,
                       min(64, T - tb_l * 64), tile_l * 128);
  };
  if (!TMA_IN && k < tasks) fetch(k);
  uint32_t phase = 0;
  bool ok = true;
  const uint32_t stage_u32 = (uint32_t)__cvta_generic_to_shared(stage);
  const int q = threadIdx.x & 31, quarter = threadIdx.x >> 5;
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
    if (threadIdx.x == 0 && it > 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncthreads();
    const int tile = (int)(k % n_tiles);
    const int64_t cb = k / n_tiles;
    const int c = (int)(cb / kb), tb = (int)(cb % kb);
    const int rows = min(64, T - tb * 64);  // the box may run into the next channel
    uint32_t re[16], im[16];                // byte m = E4M3 of input 4q+m at sample 16 quarter + r
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int sidx = 16 * quarter + r;
      const uint32_t w = sidx < rows ? *reinterpret_cast<const uint32_t *>(raw + sidx * kTile + 4 * q) : 0u;
      re[r] = nib4_to_e4m3(w);
      im[r] = nib4_to_e4m3(w >> 4);
    }
    __syncthreads();  // raw is free: fetch the next task's box while this one is converted
    if (TMA_IN && threadIdx.x == 0 && k + gridDim.x < tasks) issue(k + gridDim.x);
    if (!TMA_IN && k + gridDim.x < tasks) fetch(k + gridDim.x);
#pragma unroll
    for (int step = 0; step < 4; ++step) {
      const int kk = (step + (q >> 1)) & 3;
      const uint32_t sel = (uint32_t)(kk | ((kk + 4) << 4));
      uint32_t vr[4], vi[4];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        vr[g] = __byte_perm(__byte_perm(re[4 * g], re[4 * g + 1], sel),
                            __byte_perm(re[4 * g + 2], re[4 * g + 3], sel), 0x5410);
        vi[g] = __byte_perm(__byte_perm(im[4 * g], im[4 * g + 1], sel),
                            __byte_perm(im[4 * g + 2], im[4 * g + 3], sel), 0x5410);
      }
      const int row = 4 * q + kk;
      const int sw = row & 7;
      uint8_t *dst = stage + row * kRowBytes;
      *reinterpret_cast<uint4 *>(dst + ((quarter ^ sw) << 4)) = make_uint4(vr[0], vr[1], vr[2], vr[3]);
      *reinterpret_cast<uint4 *>(dst + (((4 + quarter) ^ sw) << 4)) = make_uint4(vi[0], vi[1], vi[2], vi[3]);
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

cudaError_t launch_unpack_persistent(const uint8_t *volt, int sample_bits, int n_inputs,
                                     int n_time, int n_tiles, int kb, int64_t chan0, int n_chan,
                                     uint8_t *op, int ctas, cudaStream_t s) {
  const int n_rows = n_tiles * kTile;
  if (n_chan <= 0) return cudaSuccess;
  if (ctas < 1 || (sample_bits == 8 && n_inputs % 2) || (sample_bits == 4 && n_inputs % 4))
    return cudaErrorInvalidValue;
  cudaError_t e = once_per_device(g_attr_persist, [] {
    cudaError_t r = cudaFuncSetAttribute(unpack8_persist_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kPersistSmem);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(unpack4_persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kPersistSmem);
    return r;
  });
  if (e != cudaSuccess) return e;
  if (sample_bits == 8)
    unpack8_persist_kernel<<<ctas, 512, kPersistSmem, s>>>(volt, op, n_inputs, n_time, n_rows, kb,
                                                           chan0, n_chan);
  else
    unpack4_persist_kernel<<<ctas, 512, kPersistSmem, s>>>(volt, op, n_inputs, n_time, n_rows, kb,
                                                           chan0, n_chan);
  return cudaGetLastError();
}

// Raw rows that are whole 16-byte units: the box comes by 2D TMA; rows that
// are whole 4-byte units: the threads load it.
bool unpack_tile_tma_in(int sample_bits, int n_inputs) {
  return (sample_bits == 8 && n_inputs % 8 == 0) || (sample_bits == 4 && n_inputs % 16 == 0);
}

bool unpack_tile_supported(int sample_bits, int n_inputs) {
  return (sample_bits == 8 && n_inputs % 2 == 0) || (sample_bits == 4 && n_inputs % 4 == 0);
}

int unpack_tile_smem_bytes() { return 1024 + kTile * kRowBytes + kTileRawBytes; }

cudaError_t launch_unpack_tile(const uint8_t *volt, int sample_bits, int n_inputs, int n_time,
                               int n_tiles, int kb, int64_t chan0, int n_chan, uint8_t *op,
                               int ctas, int32_t *status, unsigned long long timeout_ns,
                               cudaStream_t s) {
  if (n_chan <= 0) return cudaSuccess;
  if (ctas < 1 || !unpack_tile_supported(sample_bits, n_inputs)) return cudaErrorInvalidValue;
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
  // input: [ (chan0 + n_chan) * T rows ][ row bytes ], no swizzle; the box is
  // one 128-input tile of one time block: 256 B x 32 rows (8-bit samples) or
  // 128 B x 64 rows (4-bit samples)
  const cuuint64_t in_rows = (cuuint64_t)(chan0 + n_chan) * n_time;
  const cuuint64_t out_rows = (cuuint64_t)n_chan * kb * n_tiles * kTile;
  if (in_rows > 0x7FFFFFFFull || out_rows > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  CUtensorMap in_map, out_map;
  memset(&in_map, 0, sizeof(in_map));
  const bool tma_in = unpack_tile_tma_in(sample_bits, n_inputs);
  const cuuint64_t row_bytes = (cuuint64_t)n_inputs * (sample_bits == 8 ? 2 : 1);
  cuuint64_t idims[2] = {row_bytes, in_rows};
  cuuint64_t istr[1] = {row_bytes};
  cuuint32_t ibox[2] = {sample_bits == 8 ? 256u : 128u, sample_bits == 8 ? 32u : 64u};
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
    if (r == cudaSuccess) r = set(reinterpret_cast<const void *>(unpack4_tile_kernel<true>));
    if (r == cudaSuccess) r = set(reinterpret_cast<const void *>(unpack4_tile_kernel<false>));
    return r;
  });
  if (ea != cudaSuccess) return ea;
#define MWAX_TILE_ARGS in_map, out_map, volt, n_inputs, n_time, n_tiles, kb, chan0, n_chan, status, timeout_ns
  if (sample_bits == 8 && tma_in)
    unpack8_tile_kernel<true><<<ctas, kTileThreads, smem, s>>>(MWAX_TILE_ARGS);
  else if (sample_bits == 8)
    unpack8_tile_kernel<false><<<ctas, kTileThreads, smem, s>>>(MWAX_TILE_ARGS);
  else if (tma_in)
    unpack4_tile_kernel<true><<<ctas, kTileThreads, smem, s>>>(MWAX_TILE_ARGS);
  else
    unpack4_tile_kernel<false><<<ctas, kTileThreads, smem, s>>>(MWAX_TILE_ARGS);
#undef MWAX_TILE_ARGS
  return cudaGetLastError();
}

cudaError_t launch_unpack(const uint8_t *volt, int sample_bits, int n_inputs, int n_time,
                          int n_tiles, int kb, int64_t chan0, int n_chan, uint8_t *op,
                          int variant_req, cudaStream_t s) {
  const int n_rows = n_tiles * kTile;
  if (n_chan <= 0) return cudaSuccess;
  // variant: 0 = automatic, 1 = shared-memory transpose, 2 = full-line;
  // MWAX_UNPACK overrides the automatic choice (tuning experiments)
  static const int env_variant = [] {
    const char *e = getenv("MWAX_UNPACK");
    return e ? atoi(e) : 0;
  }();
  const int variant = variant_req != 0 ? variant_req : env_variant;
  const bool line8 = variant == 2;
  const bool line4 = variant != 1;
  if (line8 && sample_bits == 8 && n_inputs % 2 == 0 && kb <= 65535 && n_chan <= 65535) {
    dim3 g((n_rows / 2 + 127) / 128, kb, n_chan);
    unpack8_line_kernel<<<g, 128, 0, s>>>(volt, op, n_inputs, n_time, n_rows, kb, chan0);
    return cudaGetLastError();
  }
  if (line4 && sample_bits == 4 && n_inputs % 4 == 0 && kb * 2 <= 65535 && n_chan <= 65535) {
    dim3 g((n_rows / 4 + 127) / 128, kb * 2, n_chan);
    unpack4_line_kernel<<<g, 128, 0, s>>>(volt, op, n_inputs, n_time, n_rows, kb, chan0);
    return cudaGetLastError();
  }
  if (kb > 65535 || n_chan > 65535) return cudaErrorInvalidValue;
  dim3 grid((n_rows + kRowsPerCta - 1) / kRowsPerCta, kb, n_chan);
  if (sample_bits == 4)
    unpack_kernel<4><<<grid, 256, 0, s>>>(volt, op, n_inputs, n_time, n_rows, kb, chan0);
  else
    unpack_kernel<8><<<grid, 256, 0, s>>>(volt, op, n_inputs, n_time, n_rows, kb, chan0);
  return cudaGetLastError();
}

}  // namespace mwax
