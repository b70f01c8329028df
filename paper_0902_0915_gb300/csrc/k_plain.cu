// k_plain.cu -- plain CUDA-core correlator: one launch per fine channel.
//
// The "plain form" of the X-engine (paper Sec. 2: cross-correlate every
// antenna pair per channel, then integrate): integer dot products on the
// CUDA cores, no tensor cores, no batching across channels.  It is the
// comparison point for the tensor-core path and a second, independent GPU
// implementation of the same definition.
//
// Each CTA owns one P x P tile pair (I >= J) of the lower triangle and one
// range of the integration (blockIdx.y: where a channel has too few tile
// pairs to fill the GPU, the integration is cut into ranges whose int32
// partial sums are added into the zeroed output with integer atomics, exact
// and independent of their order); every thread holds a 4x4 block of complex
// int32 accumulators.  Time goes through
// shared memory in pairs of samples: input i's pair (t, t+1) is one 32-bit
// word of four signed bytes [re_t, im_t, re_t+1, im_t+1] (A for the tile's
// rows), and column input j has the same word B and C = [-im_t, re_t,
// -im_t+1, re_t+1].  With x_i conj(x_j):
//   Re += a_re b_re + a_im b_im  = dp4a(A_i, B_j)
//   Im += a_im b_re - a_re b_im  = dp4a(A_i, C_j)
// so one byte dot-product instruction does two complex multiply-adds' worth
// of a component.  Samples are in [-7, 7] or [-127, 127] (the ABI excludes
// -8 and -128), so the byte negation is exact; the int32 sums are exact
// because the plan rejects T * 2 * max^2 > INT32_MAX.
#include <algorithm>

#include "mwax_internal.h"

namespace mwax {
namespace {

constexpr int kTP = 16;  // time pairs per shared-memory chunk (32 samples)

// (re, im) of input i at one time row as two sign-extended bytes (low half)
__device__ __forceinline__ uint32_t sample_bytes(const uint8_t *row, int i, int bits) {
  if (bits == 4) {
    const uint32_t b = row[i];
    const uint32_t re = (uint32_t)(((int)(b << 28)) >> 28) & 0xFFu;
    const uint32_t im = (uint32_t)(((int)(b << 24)) >> 28) & 0xFFu;
    return re | (im << 8);
  }
  return (uint32_t)reinterpret_cast<const uint16_t *>(row)[i];
}

template <int P, bool ADD>
__global__ void __launch_bounds__((P / 4) * (P / 4)) plain_kernel(const uint8_t *__restrict__ volt,
                                                                   int bits, int N, int T, int Ts,
                                                                   int32_t *__restrict__ out) {
  constexpr int kThreads = (P / 4) * (P / 4);
  constexpr int kSide = P / 4;  // threads per tile side
  __shared__ __align__(16) uint32_t sA[kTP][P];
  __shared__ __align__(16) uint32_t sB[kTP][P];
  __shared__ __align__(16) uint32_t sC[kTP][P];

  // tile pair p -> (I, J) with I >= J, p = I(I+1)/2 + J
  const int p = blockIdx.x;
  int I = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
  while ((I + 1) * (I + 2) / 2 <= p) ++I;
  while (I * (I + 1) / 2 > p) --I;
  const int J = p - I * (I + 1) / 2;
  const int i0 = I * P, j0 = J * P;

  const int tid = threadIdx.x;
  const int ty = tid / kSide, tx = tid % kSide;
  const int64_t row_bytes = (int64_t)N * (bits == 4 ? 1 : 2);

  int acc_re[4][4], acc_im[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc_re[a][b] = acc_im[a][b] = 0;

  // this CTA's range of the integration: [t_begin, t_end), Ts a multiple of 2.
  // 64 x 64 tiles load the next chunk's words into registers while the
  // current one is multiplied (kIt words of each side per thread); 32 x 32
  // tiles load each chunk just before storing it (the registers the early
  // loads would hold cost more there than the latency they hide: measured).
  constexpr int kIt = kTP * P / kThreads;
  constexpr bool kPrefetch = P == 64;
  const int t_begin = blockIdx.y * Ts, t_end = min(T, t_begin + Ts);
  uint32_t na[kIt], nb[kIt];
  auto fetch = [&](int t0) {  // this thread's words of the chunk at t0, into na / nb
#pragma unroll
    for (int m = 0; m < kIt; ++m) {
      const int k = tid + m * kThreads;
      const int tp = k / P, l = k % P;
      const int t = t0 + 2 * tp;
      uint32_t wa = 0, wb = 0;
      if (t < t_end) {
        const uint8_t *r0 = volt + (int64_t)t * row_bytes;
        const bool second = t + 1 < t_end;
        if (i0 + l < N) {
          wa = sample_bytes(r0, i0 + l, bits);
          if (second) wa |= sample_bytes(r0 + row_bytes, i0 + l, bits) << 16;
        }
        if (j0 + l < N) {
          wb = sample_bytes(r0, j0 + l, bits);
          if (second) wb |= sample_bytes(r0 + row_bytes, j0 + l, bits) << 16;
        }
      }
      na[m] = wa;
      nb[m] = wb;
    }
  };
  if (kPrefetch && t_begin < t_end) fetch(t_begin);
  for (int t0 = t_begin; t0 < t_end; t0 += 2 * kTP) {
    if constexpr (kPrefetch) {
#pragma unroll
      for (int m = 0; m < kIt; ++m) {
        const int k = tid + m * kThreads;
        const int tp = k / P, l = k % P;
        sA[tp][l] = na[m];
        sB[tp][l] = nb[m];
        // C = [-im_t, re_t, -im_t+1, re_t+1]: bytes 1, 0, 3, 2 of (-B, B)
        sC[tp][l] = __byte_perm(nb[m], __vneg4(nb[m]), 0x2705);
      }
    } else {
      for (int k = tid; k < kTP * P; k += kThreads) {
        const int tp = k / P, l = k % P;
        const int t = t0 + 2 * tp;
        uint32_t wa = 0, wb = 0;
        if (t < t_end) {
          const uint8_t *r0 = volt + (int64_t)t * row_bytes;
          const bool second = t + 1 < t_end;
          if (i0 + l < N) {
            wa = sample_bytes(r0, i0 + l, bits);
            if (second) wa |= sample_bytes(r0 + row_bytes, i0 + l, bits) << 16;
          }
          if (j0 + l < N) {
            wb = sample_bytes(r0, j0 + l, bits);
            if (second) wb |= sample_bytes(r0 + row_bytes, j0 + l, bits) << 16;
          }
        }
        sA[tp][l] = wa;
        sB[tp][l] = wb;
        sC[tp][l] = __byte_perm(wb, __vneg4(wb), 0x2705);
      }
    }
    __syncthreads();
    if (kPrefetch && t0 + 2 * kTP < t_end) fetch(t0 + 2 * kTP);
#pragma unroll 4
    for (int tp = 0; tp < kTP; ++tp) {
      const uint4 a = *reinterpret_cast<const uint4 *>(&sA[tp][ty * 4]);
      const uint4 b = *reinterpret_cast<const uint4 *>(&sB[tp][tx * 4]);
      const uint4 c = *reinterpret_cast<const uint4 *>(&sC[tp][tx * 4]);
      const int av[4] = {(int)a.x, (int)a.y, (int)a.z, (int)a.w};
      const int bv[4] = {(int)b.x, (int)b.y, (int)b.z, (int)b.w};
      const int cv[4] = {(int)c.x, (int)c.y, (int)c.z, (int)c.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          acc_re[u][v] = __dp4a(av[u], bv[v], acc_re[u][v]);
          acc_im[u][v] = __dp4a(av[u], cv[v], acc_im[u][v]);
        }
    }
    __syncthreads();
  }

#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty * 4 + u;
    if (i >= N) continue;
    const int64_t rowb = (int64_t)i * (i + 1) / 2;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + tx * 4 + v;
      if (j > i || j >= N) continue;
      if constexpr (ADD) {
        atomicAdd(out + 2 * (rowb + j), acc_re[u][v]);
        atomicAdd(out + 2 * (rowb + j) + 1, acc_im[u][v]);
      } else {
        *reinterpret_cast<int2 *>(out + 2 * (rowb + j)) = make_int2(acc_re[u][v], acc_im[u][v]);
      }
    }
  }
}

// CTA shape and integration ranges of one channel's launch.
template <int P>
cudaError_t launch_plain(const uint8_t *volt_chan, int bits, int N, int T, int32_t *out_chan,
                         int sm_count, cudaStream_t s) {
  constexpr int kWarps = (P / 4) * (P / 4) / 32;
  const int nt = (N + P - 1) / P;
  const int pairs = nt * (nt + 1) / 2;
  // enough CTAs for about 16 warps per SM, ranges of at least 128 samples
  const int want = (16 * std::max(sm_count, 1) + kWarps - 1) / kWarps;
  int S = pairs >= want ? 1 : std::min((want + pairs - 1) / pairs, std::max(1, T / 128));
  const int Ts = ((T + S - 1) / S + 1) / 2 * 2;
  S = (T + Ts - 1) / Ts;
  if (S <= 1) {
    plain_kernel<P, false><<<pairs, (P / 4) * (P / 4), 0, s>>>(volt_chan, bits, N, T, T, out_chan);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(out_chan, 0, (size_t)N * (N + 1) / 2 * 2 * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  plain_kernel<P, true><<<dim3(pairs, S), (P / 4) * (P / 4), 0, s>>>(volt_chan, bits, N, T, Ts,
                                                                      out_chan);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_plain_channel(const uint8_t *volt_chan, int sample_bits, int n_inputs,
                                 int n_time, int32_t *out_chan, int sm_count, cudaStream_t s) {
  // 64 x 64 tile pairs (256 threads) for larger arrays, 32 x 32 (64 threads)
  // for smaller ones
  if (n_inputs > 256)
    return launch_plain<64>(volt_chan, sample_bits, n_inputs, n_time, out_chan, sm_count, s);
  return launch_plain<32>(volt_chan, sample_bits, n_inputs, n_time, out_chan, sm_count, s);
}

}  // namespace mwax
