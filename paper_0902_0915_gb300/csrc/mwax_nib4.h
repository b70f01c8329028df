// mwax_nib4.h -- 4-bit samples to E4M3 operand codes (device code, shared by
// the unpack kernel and the correlate kernel's fused pair mode).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace mwax {

// Four nibbles (the low nibble of each byte of x, two's complement) -> four
// E4M3 codes, one per byte.  Each nibble n, biased to n + 8 in [0, 15], is the
// low byte of the binary16 1024 + (n + 8) (exponent 10: the byte is the
// integer part of the fraction); subtracting 1032 leaves n exactly, and the
// hardware's packed binary16 -> E4M3 conversion, exact for |n| <= 16, gives
// the codes.  (Integer work: one logic op and two byte permutes per four
// nibbles; a byte-permute lookup of the 16 codes with a sign select took
// about three times as many integer instructions.)
__device__ __forceinline__ uint32_t nib4_to_e4m3_f16(uint32_t x) {
  const uint32_t u = (x & 0x0F0F0F0Fu) ^ 0x08080808u;  // n + 8 in each byte
  uint32_t lo = __byte_perm(u, 0x64646464u, 0x4140), hi = __byte_perm(u, 0x64646464u, 0x4342);
  const __half2 bias = __halves2half2(__ushort_as_half(0x6408), __ushort_as_half(0x6408));  // 1032
  const __half2 hl = __hsub2(*reinterpret_cast<const __half2 *>(&lo), bias);
  const __half2 hh = __hsub2(*reinterpret_cast<const __half2 *>(&hi), bias);
  uint16_t el, eh;
  asm("cvt.rn.satfinite.e4m3x2.f16x2 %0, %1;" : "=h"(el) : "r"(*reinterpret_cast<const uint32_t *>(&hl)));
  asm("cvt.rn.satfinite.e4m3x2.f16x2 %0, %1;" : "=h"(eh) : "r"(*reinterpret_cast<const uint32_t *>(&hh)));
  return (uint32_t)el | ((uint32_t)eh << 16);
}

}  // namespace mwax
