// k_unpack.cu -- packed complex samples -> tensor-core operand rows.
//
// Input  volt[chan][t][input]: 4+4-bit (one byte, low nibble re) or 8+8-bit
//        (re byte, im byte) two's-complement samples.
// Output op[chan][row][kb][128 B]: one row per input (rows >= N are zero
//        padding up to a multiple of the 128-input tile), and for every
//        block of S time samples a 128-byte block
//            [ re(t0) .. re(t0+S-1) | im(t0) .. im(t0+S-1) ]
//        holding the samples as exact small floats:
//            8-bit samples: S = 32, IEEE binary16 (exact for |v| <= 2048),
//            4-bit samples: S = 64, FP8 E4M3 (exact for |v| <= 16).
//        Time samples past T are zero; zeros add nothing to any product.
//
// This is the K-major operand layout of the correlator's MMAs: the 128-byte
// block is one row of a 128-byte-swizzled shared-memory tile, and each MMA
// consumes a 32-byte slice of it (K = 16 halves or K = 32 E4M3 values).
//
// HBM-bound: loads are coalesced across inputs, the transpose goes through
// shared memory, and stores are 16-byte vectors, 8 threads per 128-byte row.
#include <cuda_fp16.h>

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

  const int tb = blockIdx.x;        // time block
  const int r0 = blockIdx.y * kRowsPerCta;
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
    uint8_t *dst = op + (((int64_t)c * n_rows + i) * kb + tb) * kRowBytes + piece * 16;
    *reinterpret_cast<uint4 *>(dst) = v;
  }
}

}  // namespace

cudaError_t launch_unpack(const uint8_t *volt, int sample_bits, int n_inputs, int n_time,
                          int n_tiles, int kb, int64_t chan0, int n_chan, uint8_t *op,
                          cudaStream_t s) {
  const int n_rows = n_tiles * kTile;
  if (n_chan <= 0) return cudaSuccess;
  dim3 grid(kb, (n_rows + kRowsPerCta - 1) / kRowsPerCta, n_chan);
  if (sample_bits == 4)
    unpack_kernel<4><<<grid, 256, 0, s>>>(volt, op, n_inputs, n_time, n_rows, kb, chan0);
  else
    unpack_kernel<8><<<grid, 256, 0, s>>>(volt, op, n_inputs, n_time, n_rows, kb, chan0);
  return cudaGetLastError();
}

}  // namespace mwax
