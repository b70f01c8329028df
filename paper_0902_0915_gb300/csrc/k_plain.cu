// k_plain.cu -- plain CUDA-core correlator: one launch per fine channel.
//
// The "plain form" of the X-engine (paper Sec. 2: cross-correlate every
// antenna pair per channel, then integrate): int32 multiply-adds on the
// CUDA cores, no tensor cores, no batching across channels.  It is the
// comparison point for the tensor-core path and a second, independent GPU
// implementation of the same definition.
//
// Each CTA owns one 32x32 tile pair (I >= J) of the lower triangle; 64
// threads each hold a 4x4 block of complex int32 accumulators.  Time is
// staged through shared memory 64 samples at a time, decoded to (re, im)
// int2 so the inner loop is pure IMAD.  The int32 accumulators are exact
// because the plan rejects T * 2 * max^2 > INT32_MAX.
#include "mwax_internal.h"

namespace mwax {
namespace {

constexpr int kPT = 32;  // inputs per plain tile
constexpr int kTC = 64;  // time samples per shared-memory chunk

__device__ __forceinline__ int nib(uint32_t v) { return (v & 8u) ? (int)v - 16 : (int)v; }

__device__ __forceinline__ int2 load_sample(const uint8_t *row, int i, int bits) {
  if (bits == 4) {
    uint32_t b = row[i];
    return make_int2(nib(b & 15u), nib(b >> 4));
  }
  const int8_t *r8 = reinterpret_cast<const int8_t *>(row);
  return make_int2((int)r8[2 * i], (int)r8[2 * i + 1]);
}

__global__ void __launch_bounds__(64) plain_kernel(const uint8_t *__restrict__ volt, int bits,
                                                   int N, int T, int32_t *__restrict__ out) {
  __shared__ __align__(16) int2 sI[kTC][kPT];
  __shared__ __align__(16) int2 sJ[kTC][kPT];

  // tile pair p -> (I, J) with I >= J, p = I(I+1)/2 + J
  const int p = blockIdx.x;
  int I = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
  while ((I + 1) * (I + 2) / 2 <= p) ++I;
  while (I * (I + 1) / 2 > p) --I;
  const int J = p - I * (I + 1) / 2;
  const int i0 = I * kPT, j0 = J * kPT;

  const int tid = threadIdx.x;
  const int ty = tid >> 3, tx = tid & 7;
  const int bps = bits == 4 ? 1 : 2;
  const int64_t row_bytes = (int64_t)N * bps;

  int acc_re[4][4], acc_im[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc_re[a][b] = acc_im[a][b] = 0;

  for (int t0 = 0; t0 < T; t0 += kTC) {
    for (int k = tid; k < kTC * kPT; k += 64) {
      const int t = k / kPT, l = k % kPT;
      int2 vi = make_int2(0, 0), vj = make_int2(0, 0);
      if (t0 + t < T) {
        const uint8_t *row = volt + (int64_t)(t0 + t) * row_bytes;
        if (i0 + l < N) vi = load_sample(row, i0 + l, bits);
        if (j0 + l < N) vj = load_sample(row, j0 + l, bits);
      }
      sI[t][l] = vi;
      sJ[t][l] = vj;
    }
    __syncthreads();
#pragma unroll 4
    for (int t = 0; t < kTC; ++t) {
      int2 a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = sI[t][ty * 4 + q];
        b[q] = sJ[t][tx * 4 + q];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          // x_i conj(x_j): re = ar br + ai bi, im = ai br - ar bi
          acc_re[u][v] += a[u].x * b[v].x + a[u].y * b[v].y;
          acc_im[u][v] += a[u].y * b[v].x - a[u].x * b[v].y;
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
      int2 val = make_int2(acc_re[u][v], acc_im[u][v]);
      *reinterpret_cast<int2 *>(out + 2 * (rowb + j)) = val;
    }
  }
}

}  // namespace

cudaError_t launch_plain_channel(const uint8_t *volt_chan, int sample_bits, int n_inputs,
                                 int n_time, int32_t *out_chan, cudaStream_t s) {
  const int nt = (n_inputs + kPT - 1) / kPT;
  const int pairs = nt * (nt + 1) / 2;
  plain_kernel<<<pairs, 64, 0, s>>>(volt_chan, sample_bits, n_inputs, n_time, out_chan);
  return cudaGetLastError();
}

}  // namespace mwax
