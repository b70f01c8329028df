// unpack_rows.cuh -- packed samples -> tensor-core operand rows, one thread
// per piece of rows, registers only (no shared memory): the row conversions
// shared by the full-line and persistent unpack kernels and by the pair-mode
// correlate, whose spare epilogue warps unpack the next channel group while
// the tensor cores work on the current one.
//
// Layouts: samples [chan][T][N] (8-bit: re, im bytes; 4-bit: re low nibble,
// im high nibble), two's complement; operand rows [chan][kb][row][128 B],
// each row [re x S | im x S] of binary16 (8-bit, S = 32) or E4M3 (4-bit,
// S = 64), rows past N zero.  Every load is one 4-byte word of consecutive
// inputs at one time sample, so a warp reads one contiguous 128-byte line;
// every store is a 16-byte piece of a row.  Requires N even (8-bit samples) or
// N % 4 == 0 (4-bit samples).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "mwax_internal.h"

namespace mwax {

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

// Tasks first, first + stride, ... of the channel group [chan0, chan0 +
// n_chan): 8-bit, one input pair x one 32-sample block per task; 4-bit, four
// inputs x half of a 64-sample block; input pair / quad fastest.
template <int BITS>
__device__ __forceinline__ void unpack_rows(const uint8_t *__restrict__ volt,
                                                   uint8_t *__restrict__ op, int N, int T,
                                                   int n_rows, int kb, int64_t chan0, int n_chan,
                                                   int64_t first, int64_t stride) {
  if constexpr (BITS == 8) {
    const int pairs = n_rows / 2;
    const int64_t tasks = (int64_t)n_chan * kb * pairs;
    for (int64_t k = first; k < tasks; k += stride) {
      const int ip = (int)(k % pairs);
      const int64_t r = k / pairs;
      unpack8_task(volt, op, N, T, n_rows, kb, chan0, (int)(r / kb), (int)(r % kb), 2 * ip);
    }
  } else {
    const int quads = n_rows / 4;
    const int64_t tasks = (int64_t)n_chan * kb * 2 * quads;
    for (int64_t k = first; k < tasks; k += stride) {
      const int iq = (int)(k % quads);
      const int64_t r = k / quads;  // (c, tb, h)
      const int h = (int)(r & 1);
      const int64_t r2 = r >> 1;
      unpack4_task(volt, op, N, T, n_rows, kb, chan0, (int)(r2 / kb), (int)(r2 % kb), h, 4 * iq);
    }
  }
}

}  // namespace mwax
