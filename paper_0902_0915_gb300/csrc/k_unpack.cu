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
#include <cuda_fp16.h>
#include <stdlib.h>

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

__global__ void __launch_bounds__(128) unpack8_line_kernel(const uint8_t *__restrict__ volt,
                                                           uint8_t *__restrict__ op, int N, int T,
                                                           int n_rows, int kb, int64_t chan0) {
  const int i0 = 2 * (blockIdx.x * 128 + threadIdx.x);
  if (i0 >= n_rows) return;
  const int tb = blockIdx.y, c = blockIdx.z;
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
// (byte_perm); the sign bit picks the table of negative values.
__device__ __forceinline__ uint32_t nib4_to_e4m3(uint32_t x) {
  const uint32_t pos_lo = 0x44403800u, pos_hi = 0x4E4C4A48u;  // 0..7
  const uint32_t neg_lo = 0xCACCCED0u, neg_hi = 0xB8C0C4C8u;  // -8..-1
  const uint32_t l = x & 0x07070707u;
  const uint32_t sel = (l & 0x7u) | ((l >> 4) & 0x70u) | ((l >> 8) & 0x700u) | ((l >> 12) & 0x7000u);
  const uint32_t p = __byte_perm(pos_lo, pos_hi, sel);
  const uint32_t n = __byte_perm(neg_lo, neg_hi, sel);
  const uint32_t m = ((x >> 3) & 0x01010101u) * 0xFFu;  // 0xFF where the nibble is negative
  return (p & ~m) | (n & m);
}

__global__ void __launch_bounds__(128) unpack4_line_kernel(const uint8_t *__restrict__ volt,
                                                           uint8_t *__restrict__ op, int N, int T,
                                                           int n_rows, int kb, int64_t chan0) {
  const int i0 = 4 * (blockIdx.x * 128 + threadIdx.x);
  if (i0 >= n_rows) return;
  const int tb = blockIdx.y >> 1, h = blockIdx.y & 1;  // half block: samples 32h .. 32h+31
  const int c = blockIdx.z;
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

}  // namespace

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
