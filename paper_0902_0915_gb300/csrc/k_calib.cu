// k_calib.cu -- direction-independent gain-calibration loss and its adjoint.
//
// Paper Sec. 2: the complex gain of each antenna element is estimated by a
// large linear least-squares fit against catalogue sources; the visibility
// data are measured against a model and each measurement constrains the
// gains.  The loss consumed here is
//     R_ij(nu) = g_i conj(g_j) M_ij(nu) - V_ij(nu)
//     L(g)     = sum_nu sum_{i>j} |R_ij(nu)|^2          (autos carry weight 0)
//     grad_k   = 2 dL/d conj(g_k) = 2 sum_nu sum_{j != k} R_kj g_j conj(M_kj)
// with R, M extended to the upper triangle by Hermitian symmetry.  For one
// stored pair (i > j) the two gradient terms are
//     to k = i:  R_ij g_j conj(M_ij)
//     to k = j:  conj(R_ij) g_i M_ij.
//
// Paper Sec. 3.2 replaces scatter with gather because the GPU of the time had
// no floating-point atomic add; the same rule gives determinism here: each
// CTA owns a 32x32 tile of input pairs for a fixed group of channels and
// writes its row / column / loss partial sums to a workspace, and a second
// kernel gathers them per input in a fixed order.  No atomics, FP32 only
// (plain 32-term sums inside a channel, Kahan-compensated accumulation across
// channels, fixed trees across lanes and warps).  One pass reads V and M once.
//
// Gain solve (alternating least squares): with every gain but g_k fixed, L
// is a linear least-squares problem in g_k whose minimiser is
//     h_k = num_k / den_k,  num_k = sum V_kj g_j conj(M_kj),
//                           den_k = sum |g_j|^2 |M_kj|^2   (j != k, all nu)
// and since grad_k / 2 = g_k den_k - num_k,  h_k = g_k - (grad_k / 2) / den_k.
// One sweep is therefore the loss/adjoint pass with one more accumulator
// (den) per row and column, followed by a gather that applies the update in
// place: g = h on odd sweeps, g = (g + h) / 2 on even sweeps (the damping of
// Salvini & Wijnholds 2014, which keeps the simultaneous update from
// oscillating).  Working from the residual keeps the FP32 update accurate
// near convergence, where num and g den nearly cancel.
#include <mutex>

#include "mwax_internal.h"

namespace mwax {
namespace {

constexpr int kCT = 32;        // inputs per calibration tile side
constexpr int kCalThreads = 256;
constexpr int kMaxChanGroups = 12;  // 528 tiles x 12 = 13.9 waves of 3 CTAs per SM at 1024 inputs

struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

int chan_groups(int n_chan) { return n_chan < kMaxChanGroups ? n_chan : kMaxChanGroups; }

__device__ __forceinline__ void tile_of(int p, int &I, int &J) {
  int i = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  while (i * (i + 1) / 2 > p) --i;
  I = i;
  J = p - i * (i + 1) / 2;
}

// Reduce-scatter of eight values across a warp (used by both tile kernels):
// a[0..7] (one value per row of a group of eight rows) -> the full-warp sum
// of value (lane >> 2) & 7, in a fixed order.  A butterfly over lane bits 4,
// 3, 2 halves the values each lane carries, then a sum over bits 1, 0 leaves
// lanes 4s..4s+3 all holding the sum of value s.
__device__ __forceinline__ float reduce_scatter8(float (&a)[8], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float send = b4 ? a[k] : a[k + 4];
    const float keep = b4 ? a[k + 4] : a[k];
    a[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = b3 ? a[k] : a[k + 2];
    const float keep = b3 ? a[k + 2] : a[k];
    a[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const float send = b2 ? a[0] : a[1];
  float x = (b2 ? a[1] : a[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  return x;
}

// One channel of one 32x32 tile, processed by one warp: lane = column
// j = J*32 + lane, rows i = I*32 + r in four groups of eight.  Returns, per
// lane, this channel's column sums (to input j), its row sums for row
// 8 (lane & 3) + ((lane >> 2) & 7) (to input i; the eight rows of a group are
// reduce-scattered across the warp, lane 4s + t keeping group t's value) and
// its part of the loss.  sgi: g of the tile's 32 rows.  Entries outside the
// stored triangle load V = M = 0, whose residual and contributions are 0.
struct TileSums {
  float loss, rre, rim, rden, cre, cim, cden;
};

template <bool DEN>
__device__ __forceinline__ TileSums tile_channel(const float2 *__restrict__ Vn,
                                                 const float2 *__restrict__ Mn,
                                                 const float2 *sgi, float2 gj, int I, int j,
                                                 int N, int lane) {
  const float2 zero = make_float2(0.f, 0.f);
  const float gj2 = gj.x * gj.x + gj.y * gj.y;
  TileSums t = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
  for (int q = 0; q < 4; ++q) {
    float2 v[8], m[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int i = I * kCT + 8 * q + s;
      const bool ok = i < N && j < i;
      const int64_t b = (int64_t)i * (i + 1) / 2 + j;
      v[s] = ok ? __ldcs(Vn + b) : zero;
      m[s] = ok ? __ldcs(Mn + b) : zero;
    }
    float ar[8], ai[8], ad[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const float2 gi = sgi[8 * q + s];
      const float Gr = gi.x * gj.x + gi.y * gj.y;  // g_i conj(g_j)
      const float Gi = gi.y * gj.x - gi.x * gj.y;
      const float Rr = Gr * m[s].x - Gi * m[s].y - v[s].x;  // R = G M - V
      const float Ri = Gr * m[s].y + Gi * m[s].x - v[s].y;
      t.loss += Rr * Rr + Ri * Ri;
      const float Pr = Rr * gj.x - Ri * gj.y, Pi = Rr * gj.y + Ri * gj.x;  // R g_j
      ar[s] = Pr * m[s].x + Pi * m[s].y;                                     // to row i
      ai[s] = Pi * m[s].x - Pr * m[s].y;
      const float Qr = Rr * gi.x + Ri * gi.y, Qi = Rr * gi.y - Ri * gi.x;  // conj(R) g_i
      t.cre += Qr * m[s].x - Qi * m[s].y;                                    // to column j
      t.cim += Qr * m[s].y + Qi * m[s].x;
      if constexpr (DEN) {
        const float m2 = m[s].x * m[s].x + m[s].y * m[s].y;
        ad[s] = gj2 * m2;                              // row i: |g_j|^2 |M_ij|^2
        t.cden += (gi.x * gi.x + gi.y * gi.y) * m2;    // column j: |g_i|^2 |M_ij|^2
      }
    }
    const float xr = reduce_scatter8(ar, lane);
    const float xi = reduce_scatter8(ai, lane);
    if ((lane & 3) == q) {
      t.rre = xr;
      t.rim = xi;
    }
    if constexpr (DEN) {
      const float xd = reduce_scatter8(ad, lane);
      if ((lane & 3) == q) t.rden = xd;
    }
  }
  return t;
}

__device__ __forceinline__ int tile_row_of_lane(int lane) {
  return 8 * (lane & 3) + ((lane >> 2) & 7);
}

// grid: (tiles, channel groups).  CTA (tile, cg) covers channels cg,
// cg + n_cg, ...; its warp w takes every eighth of them
// (nu = cg + n_cg (w + 8k)), each channel with tile_channel, and adds the
// channel's sums into Kahan accumulators (one compensated add per channel;
// the 32-term sums inside a channel are plain FP32).  The eight warps' totals
// are then summed in a fixed order.  DEN: also the per-row and per-column
// sums of |g_other|^2 |M|^2 (the gain solve's normal-equation weight; sums of
// positive terms, plain FP32).
template <bool DEN>
__global__ void __launch_bounds__(kCalThreads, 3) calib_tile_kernel(
    const float2 *__restrict__ V, const float2 *__restrict__ M, const float2 *__restrict__ g,
    int N, int C, int n_cg, float *__restrict__ part_loss, float2 *__restrict__ part_row,
    float2 *__restrict__ part_col, float *__restrict__ part_rden, float *__restrict__ part_cden) {
  constexpr int kWarps = kCalThreads / 32;
  __shared__ float2 sgi[kCT];
  __shared__ float2 srow[kWarps][kCT], scol[kWarps][kCT];
  __shared__ float srden[kWarps][kCT], scden[kWarps][kCT];
  __shared__ float sloss[kWarps];
  const int tile = blockIdx.x, cg = blockIdx.y;
  int I, J;
  tile_of(tile, I, J);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = J * kCT + lane;
  if (threadIdx.x < kCT) {
    const int il = I * kCT + threadIdx.x;
    sgi[threadIdx.x] = il < N ? g[il] : make_float2(0.f, 0.f);
  }
  const float2 gj = j < N ? g[j] : make_float2(0.f, 0.f);
  __syncthreads();
  const int64_t B = (int64_t)N * (N + 1) / 2;
  Kahan loss, rre, rim, cre, cim;
  float rden = 0.f, cden = 0.f;
  for (int nu = cg + n_cg * w; nu < C; nu += n_cg * kWarps) {
    const TileSums t = tile_channel<DEN>(V + (int64_t)nu * B, M + (int64_t)nu * B, sgi, gj, I, j,
                                         N, lane);
    loss.add(t.loss);
    rre.add(t.rre);
    rim.add(t.rim);
    cre.add(t.cre);
    cim.add(t.cim);
    if constexpr (DEN) {
      rden += t.rden;
      cden += t.cden;
    }
  }
  const int row = tile_row_of_lane(lane);
  srow[w][row] = make_float2(rre.s, rim.s);
  scol[w][lane] = make_float2(cre.s, cim.s);
  if constexpr (DEN) {
    srden[w][row] = rden;
    scden[w][lane] = cden;
  }
  float l = loss.s;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if (lane == 0) sloss[w] = l;
  __syncthreads();
  const int out_idx = tile * n_cg + cg;
  if (w == 0) {
    float2 ar = srow[0][lane], ac = scol[0][lane];
#pragma unroll
    for (int k = 1; k < kWarps; ++k) {
      ar.x += srow[k][lane].x;
      ar.y += srow[k][lane].y;
      ac.x += scol[k][lane].x;
      ac.y += scol[k][lane].y;
    }
    part_row[(int64_t)out_idx * kCT + lane] = ar;
    part_col[(int64_t)out_idx * kCT + lane] = ac;
    if constexpr (DEN) {
      float dr = srden[0][lane], dc = scden[0][lane];
#pragma unroll
      for (int k = 1; k < kWarps; ++k) {
        dr += srden[k][lane];
        dc += scden[k][lane];
      }
      part_rden[(int64_t)out_idx * kCT + lane] = dr;
      part_cden[(int64_t)out_idx * kCT + lane] = dc;
    }
    if (lane == 0) {
      float t = 0.f;
      for (int k = 0; k < kWarps; ++k) t += sloss[k];
      part_loss[out_idx] = t;
    }
  }
}

// grid: n_blocks + 1.  Block K < n_blocks gathers grad for inputs K*32..;
// the last block sums the loss partials.  SOLVE: instead of grad, apply one
// gain-solve sweep to g in place (each block reads and writes only its own
// 32 gains): g = h (avg == 0) or g = (g + h) / 2 (avg == 1).
template <bool SOLVE>
__global__ void __launch_bounds__(kCalThreads) calib_gather_kernel(
    int N, int n_blocks, int n_cg, const float *__restrict__ part_loss,
    const float2 *__restrict__ part_row, const float2 *__restrict__ part_col,
    const float *__restrict__ part_rden, const float *__restrict__ part_cden,
    float *__restrict__ loss, float2 *__restrict__ grad, float2 *__restrict__ g_io, int avg) {
  const int K = blockIdx.x;
  if (K == n_blocks) {
    if (!loss) return;
    __shared__ float sred[kCalThreads];
    const int n_part = n_blocks * (n_blocks + 1) / 2 * n_cg;
    Kahan acc;
    for (int k = threadIdx.x; k < n_part; k += kCalThreads) acc.add(part_loss[k]);
    sred[threadIdx.x] = acc.s;
    __syncthreads();
    for (int w = kCalThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sred[threadIdx.x] += sred[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) *loss = sred[0];
    return;
  }
  if (!SOLVE && !grad) return;
  // 32 inputs x 8 partial lanes: thread (r, l) sums every 8th contribution
  __shared__ float2 sacc[8][kCT];
  __shared__ float sden[8][kCT];
  const int r = threadIdx.x & 31, l = threadIdx.x >> 5;
  Kahan ar, ai, ad;
  // contributions n = 0, 1, ...: the row partials of tiles (K, J <= K), then
  // the column partials of tiles (I >= K, K), each over the channel groups;
  // thread l takes n = l, l + 8, ...
  const int n_row = (K + 1) * n_cg;
  const int n_tot = n_row + (n_blocks - K) * n_cg;
  for (int n = l; n < n_tot; n += 8) {
    const bool is_row = n < n_row;
    const int m = is_row ? n : n - n_row;
    const int t = m / n_cg, cg = m - t * n_cg;
    const int tile = is_row ? K * (K + 1) / 2 + t : (K + t) * (K + t + 1) / 2 + K;
    const int64_t idx = ((int64_t)tile * n_cg + cg) * kCT + r;
    const float2 v = is_row ? part_row[idx] : part_col[idx];
    ar.add(v.x);
    ai.add(v.y);
    if constexpr (SOLVE) ad.add(is_row ? part_rden[idx] : part_cden[idx]);
  }
  sacc[l][r] = make_float2(ar.s, ai.s);
  if constexpr (SOLVE) sden[l][r] = ad.s;
  __syncthreads();
  if (l == 0) {
    float2 acc = sacc[0][r];
#pragma unroll
    for (int w = 1; w < 8; ++w) {
      acc.x += sacc[w][r].x;
      acc.y += sacc[w][r].y;
    }
    const int k = K * kCT + r;
    if constexpr (SOLVE) {
      float den = sden[0][r];
#pragma unroll
      for (int w = 1; w < 8; ++w) den += sden[w][r];
      if (k < N && den > 0.f) {
        // h = g - (grad / 2) / den; acc holds grad / 2
        const float2 gk = g_io[k];
        const float inv = 1.f / den;
        float2 h = make_float2(gk.x - acc.x * inv, gk.y - acc.y * inv);
        if (avg) h = make_float2(0.5f * (gk.x + h.x), 0.5f * (gk.y + h.y));
        g_io[k] = h;
      }
    } else {
      if (k < N) grad[k] = make_float2(2.f * acc.x, 2.f * acc.y);
    }
  }
}

// ---- per-channel gains ----------------------------------------------------------
// g_k(nu), stored [C][N]: the channels decouple, so every (tile, channel) is a
// reduction of its own and nothing is carried across channels.  One warp owns
// one 32x32 tile of one channel (tile_channel) and writes that channel's row
// and column sums; the eight warps of a CTA take eight consecutive channels of
// the same tile.

// grid: (tiles, ceil(C / 8)).  Partial sums per (tile, channel):
// part_row / part_col [tile][C][32], DEN: part_rden / part_cden likewise;
// part_loss [tile][gridDim.y] (the CTA's eight channels).
template <bool DEN>
__global__ void __launch_bounds__(kCalThreads, 3) calib_chan_tile_kernel(
    const float2 *__restrict__ V, const float2 *__restrict__ M, const float2 *__restrict__ g,
    int N, int C, float *__restrict__ part_loss, float2 *__restrict__ part_row,
    float2 *__restrict__ part_col, float *__restrict__ part_rden, float *__restrict__ part_cden) {
  __shared__ float2 sgi[kCalThreads / 32][kCT];
  __shared__ float sloss[kCalThreads / 32];
  const int tile = blockIdx.x;
  int I, J;
  tile_of(tile, I, J);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nu = blockIdx.y * (kCalThreads / 32) + w;
  float lsum = 0.f;
  if (nu < C) {
    const int64_t B = (int64_t)N * (N + 1) / 2;
    const float2 *gn = g + (int64_t)nu * N;
    const int j = J * kCT + lane, il = I * kCT + lane;
    const float2 gj = j < N ? gn[j] : make_float2(0.f, 0.f);
    sgi[w][lane] = il < N ? gn[il] : make_float2(0.f, 0.f);
    __syncwarp();
    const TileSums t = tile_channel<DEN>(V + (int64_t)nu * B, M + (int64_t)nu * B, sgi[w], gj, I,
                                         j, N, lane);
    const int64_t base = ((int64_t)tile * C + nu) * kCT;
    const int row = tile_row_of_lane(lane);
    part_row[base + row] = make_float2(t.rre, t.rim);
    part_col[base + lane] = make_float2(t.cre, t.cim);
    if constexpr (DEN) {
      part_rden[base + row] = t.rden;
      part_cden[base + lane] = t.cden;
    }
    lsum = t.loss;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  }
  if (lane == 0) sloss[w] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int k = 0; k < kCalThreads / 32; ++k) t += sloss[k];
    part_loss[(int64_t)tile * gridDim.y + blockIdx.y] = t;
  }
}

// grid: (n_blocks + 1, ceil(C / 8)).  Block (K, y), warp w: channel
// nu = 8y + w, lane r: input k = 32K + r, summing its row partials over tiles
// (K, J <= K) and its column partials over tiles (I >= K, K) in that order.
// Block (n_blocks, 0) sums the loss partials.  SOLVE: one sweep's update of
// g[nu][k] in place, as in calib_gather_kernel.
template <bool SOLVE>
__global__ void __launch_bounds__(kCalThreads) calib_chan_gather_kernel(
    int N, int C, int n_blocks, const float *__restrict__ part_loss,
    const float2 *__restrict__ part_row, const float2 *__restrict__ part_col,
    const float *__restrict__ part_rden, const float *__restrict__ part_cden,
    float *__restrict__ loss, float2 *__restrict__ grad, float2 *__restrict__ g_io, int avg) {
  const int K = blockIdx.x;
  if (K == n_blocks) {
    if (blockIdx.y != 0 || !loss) return;
    __shared__ float sred[kCalThreads];
    const int64_t n_part = (int64_t)n_blocks * (n_blocks + 1) / 2 * gridDim.y;
    Kahan acc;
    for (int64_t k = threadIdx.x; k < n_part; k += kCalThreads) acc.add(part_loss[k]);
    sred[threadIdx.x] = acc.s;
    __syncthreads();
    for (int h = kCalThreads / 2; h > 0; h >>= 1) {
      if (threadIdx.x < h) sred[threadIdx.x] += sred[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) *loss = sred[0];
    return;
  }
  if (!SOLVE && !grad) return;
  const int lane = threadIdx.x & 31;
  const int nu = blockIdx.y * (kCalThreads / 32) + (threadIdx.x >> 5);
  const int k = K * kCT + lane;
  if (nu >= C || k >= N) return;
  float ar = 0.f, ai = 0.f, ad = 0.f;
  for (int Jt = 0; Jt <= K; ++Jt) {
    const int64_t idx = ((int64_t)(K * (K + 1) / 2 + Jt) * C + nu) * kCT + lane;
    const float2 v = part_row[idx];
    ar += v.x;
    ai += v.y;
    if constexpr (SOLVE) ad += part_rden[idx];
  }
  for (int It = K; It < n_blocks; ++It) {
    const int64_t idx = ((int64_t)(It * (It + 1) / 2 + K) * C + nu) * kCT + lane;
    const float2 v = part_col[idx];
    ar += v.x;
    ai += v.y;
    if constexpr (SOLVE) ad += part_cden[idx];
  }
  const int64_t o = (int64_t)nu * N + k;
  if constexpr (SOLVE) {
    if (ad > 0.f) {
      const float2 gk = g_io[o];
      const float inv = 1.f / ad;
      float2 h = make_float2(gk.x - ar * inv, gk.y - ai * inv);  // (ar, ai) = grad / 2
      if (avg) h = make_float2(0.5f * (gk.x + h.x), 0.5f * (gk.y + h.y));
      g_io[o] = h;
    }
  } else {
    grad[o] = make_float2(2.f * ar, 2.f * ai);
  }
}

// ---- full 2x2 Jones matrices per tile ---------------------------------------------
// Inputs 2a, 2a + 1 are the two polarisations of tile a.  Block (a, b), a > b,
// of V and M is the 2x2 matrix of inputs (2a + p, 2b + q), modelled as
// J_a M_ab J_b^H.  With B = M J_b^H, A = J_a M and R = J_a B - V:
//     loss   += ||R||^2
//     tile a: G += R B^H,  D += B B^H     (the least-squares problem in J_a)
//     tile b: G += R^H A,  D += A^H A     (the same for J_b, from V^H)
// so that grad_t = 2 G_t (= 2 dL/d conj(J_t)) and the alternating least-squares
// target is H_t = J_t - G_t D_t^-1, D_t Hermitian.  A calibration tile is
// 32 x 32 blocks (64 x 64 inputs): lane = column block b, rows a walked two
// at a time.  The twelve tile-a quantities of a row (G: 8 floats, D: d00,
// d11, Re d10, Im d10) are reduce-scattered across the warp together with
// those of the row four on (see reduce_scatter24); the tile-b quantities
// stay in the lane.  Entries outside the stored blocks (a >= n_tiles,
// b >= a) load V = M = 0 and contribute exactly 0.
constexpr int kJT = 32;  // Jones blocks per calibration tile side
constexpr int kJQ = 12;  // per-tile partial quantities
#ifndef MWAX_JONES_CHAN_GROUPS
#define MWAX_JONES_CHAN_GROUPS 12  // channel groups of the Jones pass (CTAs per calibration tile)
#endif
constexpr int kJonesChanGroups = MWAX_JONES_CHAN_GROUPS;

// acc + a b,  acc + a conj(b),  acc + conj(a) b
__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 b) {
  return make_float2(acc.x + a.x * b.x - a.y * b.y, acc.y + a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cfmac(float2 acc, float2 a, float2 b) {
  return make_float2(acc.x + a.x * b.x + a.y * b.y, acc.y + a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 ccfma(float2 acc, float2 a, float2 b) {
  return make_float2(acc.x + a.x * b.x + a.y * b.y, acc.y + a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Two rows per step: the 24 tile-a quantities of rows ra and rb = ra + 4 (12
// each) reduce-scattered together -- halving over lane bits 4 (row), 3 and 2,
// then a sum over bits 1 and 0: 27 shuffles for the two rows instead of 36,
// and twice the independent work in flight.  Lanes 4h .. 4h + 3 then hold
// quantities 3h .. 3h + 2 of the 24 (h < 4: row ra, h >= 4: row rb).
__device__ __forceinline__ void reduce_scatter24(float (&v)[2 * kJQ], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float send = b4 ? v[k] : v[k + 12];
    const float keep = b4 ? v[k + 12] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float send = b3 ? v[k] : v[k + 6];
    const float keep = b3 ? v[k + 6] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float send = b2 ? v[k] : v[k + 3];
    const float keep = b2 ? v[k + 3] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
#pragma unroll
  for (int o = 2; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// One row's block (a, b) of V and M into the lane's 64-byte slot
// [V row 2a | V row 2a+1 | M row 2a | M row 2a+1], 16 bytes each (the two
// entries of the block in that row).  Of the two rows of the triangle one
// starts the block on a 16-byte boundary (one 16-byte copy), the other on an
// 8-byte one (two 8-byte copies); the alignment is the same for every lane of
// the warp.
__device__ __forceinline__ void jones_load_row(float4 *slot, const float2 *Vn, const float2 *Mn,
                                               int a, int b) {
  const int64_t i0 = 2 * (int64_t)a, i1 = i0 + 1;
  const int64_t o0 = i0 * (i0 + 1) / 2 + 2 * b, o1 = i1 * (i1 + 1) / 2 + 2 * b;
  const float2 *src[4] = {Vn + o0, Vn + o1, Mn + o0, Mn + o1};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if ((reinterpret_cast<uintptr_t>(src[e]) & 15u) == 0) {
      cp_async16(slot + e * 32, src[e]);
    } else {
      cp_async8(reinterpret_cast<float2 *>(slot + e * 32), src[e]);
      cp_async8(reinterpret_cast<float2 *>(slot + e * 32) + 1, src[e] + 1);
    }
  }
}

// The per-row work of the Jones pass: loss, the lane's tile-b sums (col) and
// the row's twelve tile-a quantities, added into v (the lane's sums over its
// channels, reduce-scattered once per row pair; v[8..11] stay as they are
// without DEN).
template <bool DEN>
__device__ __forceinline__ float jones_row(const float4 *slot, float2 ja00, float2 ja01,
                                           float2 ja10, float2 ja11, float2 jb00, float2 jb01,
                                           float2 jb10, float2 jb11, float (&col)[kJQ],
                                           float *v) {
  const float4 va = slot[0 * 32], vb = slot[1 * 32], ma = slot[2 * 32], mb = slot[3 * 32];
  const float2 v00 = make_float2(va.x, va.y), v01 = make_float2(va.z, va.w);
  const float2 v10 = make_float2(vb.x, vb.y), v11 = make_float2(vb.z, vb.w);
  const float2 m00 = make_float2(ma.x, ma.y), m01 = make_float2(ma.z, ma.w);
  const float2 m10 = make_float2(mb.x, mb.y), m11 = make_float2(mb.z, mb.w);
  const float2 z = make_float2(0.f, 0.f);
  const float2 B00 = cfmac(cfmac(z, m00, jb00), m01, jb01);
  const float2 B01 = cfmac(cfmac(z, m00, jb10), m01, jb11);
  const float2 B10 = cfmac(cfmac(z, m10, jb00), m11, jb01);
  const float2 B11 = cfmac(cfmac(z, m10, jb10), m11, jb11);
  const float2 R00 = cfma(cfma(make_float2(-v00.x, -v00.y), ja00, B00), ja01, B10);
  const float2 R01 = cfma(cfma(make_float2(-v01.x, -v01.y), ja00, B01), ja01, B11);
  const float2 R10 = cfma(cfma(make_float2(-v10.x, -v10.y), ja10, B00), ja11, B10);
  const float2 R11 = cfma(cfma(make_float2(-v11.x, -v11.y), ja10, B01), ja11, B11);
  const float l = cabs2(R00) + cabs2(R01) + cabs2(R10) + cabs2(R11);
  {
    const float2 g00 = cfmac(cfmac(make_float2(v[0], v[1]), R00, B00), R01, B01);
    const float2 g01 = cfmac(cfmac(make_float2(v[2], v[3]), R00, B10), R01, B11);
    const float2 g10 = cfmac(cfmac(make_float2(v[4], v[5]), R10, B00), R11, B01);
    const float2 g11 = cfmac(cfmac(make_float2(v[6], v[7]), R10, B10), R11, B11);
    v[0] = g00.x; v[1] = g00.y; v[2] = g01.x; v[3] = g01.y;
    v[4] = g10.x; v[5] = g10.y; v[6] = g11.x; v[7] = g11.y;
    if constexpr (DEN) {
      const float2 d10 = cfmac(cfmac(make_float2(v[10], v[11]), B10, B00), B11, B01);
      v[8] += cabs2(B00) + cabs2(B01);
      v[9] += cabs2(B10) + cabs2(B11);
      v[10] = d10.x;
      v[11] = d10.y;
    }
  }
  const float2 A00 = cfma(cfma(z, ja00, m00), ja01, m10);
  const float2 A01 = cfma(cfma(z, ja00, m01), ja01, m11);
  const float2 A10 = cfma(cfma(z, ja10, m00), ja11, m10);
  const float2 A11 = cfma(cfma(z, ja10, m01), ja11, m11);
  const float2 g00 = ccfma(ccfma(z, R00, A00), R10, A10);
  const float2 g01 = ccfma(ccfma(z, R00, A01), R10, A11);
  const float2 g10 = ccfma(ccfma(z, R01, A00), R11, A10);
  const float2 g11 = ccfma(ccfma(z, R01, A01), R11, A11);
  col[0] += g00.x; col[1] += g00.y; col[2] += g01.x; col[3] += g01.y;
  col[4] += g10.x; col[5] += g10.y; col[6] += g11.x; col[7] += g11.y;
  if constexpr (DEN) {
    const float2 d10 = ccfma(ccfma(z, A01, A00), A11, A10);
    col[8] += cabs2(A00) + cabs2(A10);
    col[9] += cabs2(A01) + cabs2(A11);
    col[10] += d10.x;
    col[11] += d10.y;
  }
  return l;
}

// The Jones pass, two rows per step (see reduce_scatter24).  Each lane stages
// the blocks of row pairs PAIRS - 1 pairs ahead in its own 128-byte slots of a
// PAIRS-deep shared-memory ring (reads back only what it copied: no barrier);
// the tile's 32 rows of J_a are staged once per CTA.  grid: (calibration
// tiles, channel groups); CTA (tile, cg) covers channels cg, cg + n_cg, ...,
// its warp w every eighth of them.  A warp walks its row pairs, each over all
// its channels: the lane adds the pair's tile-a quantities over the channels
// and the warp reduce-scatters them once per row pair; each row pair's loss
// goes into a Kahan accumulator; the eight warps' partials are summed in a
// fixed order.
// Outputs per (tile, cg): part_row [32 rows][12], part_col [32 columns][12],
// part_loss.  DEN: the D quantities (left at 0 otherwise).
#ifndef MWAX_JONES_PAIRS
#define MWAX_JONES_PAIRS 3
#endif
constexpr int kJPairs = MWAX_JONES_PAIRS;  // row pairs in the ring: loads kJPairs - 1 pairs ahead
constexpr int jones2_smem_bytes() {
  return (kCalThreads / 32) * kJPairs * 2 * 4 * 32 * 16 + kJT * 4 * 8;
}
template <bool DEN>
__global__ void __launch_bounds__(kCalThreads, 2) calib_jones_tile2_kernel(
    const float2 *__restrict__ V, const float2 *__restrict__ M, const float2 *__restrict__ Jm,
    int n_tiles, int C, int n_cg, float *__restrict__ part_loss, float *__restrict__ part_row,
    float *__restrict__ part_col) {
  constexpr int kWarps = kCalThreads / 32;
  extern __shared__ __align__(16) float4 sdyn[];
  // ring [warp][pair slot][row 0/1][4 entries][lane]; afterwards the same memory
  // holds the per-warp partials [warp][32][12] and the per-warp losses
  float4 *ringbase = sdyn;
  float2 *sJ = reinterpret_cast<float2 *>(sdyn + kWarps * kJPairs * 2 * 4 * 32);  // [32 rows][4]
  static_assert(sizeof(float) * (kWarps * kJT * kJQ + kWarps) <= sizeof(float4) * kWarps * kJPairs * 2 * 4 * 32,
                "aliasing");
  const int tile = blockIdx.x, cg = blockIdx.y;
  int I, Jt;
  tile_of(tile, I, Jt);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = Jt * kJT + lane;
  for (int e = threadIdx.x; e < kJT * 4; e += kCalThreads) {
    const int a = I * kJT + e / 4;
    sJ[e] = a < n_tiles ? Jm[(int64_t)a * 4 + (e & 3)] : make_float2(0.f, 0.f);
  }
  float2 jb00 = make_float2(0.f, 0.f), jb01 = jb00, jb10 = jb00, jb11 = jb00;
  if (b < n_tiles) {
    jb00 = Jm[(int64_t)b * 4 + 0];
    jb01 = Jm[(int64_t)b * 4 + 1];
    jb10 = Jm[(int64_t)b * 4 + 2];
    jb11 = Jm[(int64_t)b * 4 + 3];
  }
  __syncthreads();
  const int64_t N = 2 * (int64_t)n_tiles, Bn = N * (N + 1) / 2;
  const int first = cg + n_cg * w, stride = n_cg * kWarps;
  const int n_mine = first < C ? (C - 1 - first) / stride + 1 : 0;
  // pair p = q n_mine + k: row pair q (rows 8 (q >> 2) + (q & 3) + {0, 4}) of
  // the warp's k-th channel; row pairs outer, channels inner, so each lane
  // sums a row pair's tile-a quantities over its channels before the one
  // reduce-scatter of the row pair
  const int n_pairs = n_mine * (kJT / 2);
  float4 *ring = ringbase + (int64_t)w * kJPairs * 2 * 4 * 32 + lane;
  int iq = 0, ik = 0;  // row pair and channel of the next pair to issue
  auto issue = [&](int p) {
    if (p < n_pairs) {
      const int nu = first + stride * ik;
      const float2 *Vn = V + (int64_t)nu * Bn, *Mn = M + (int64_t)nu * Bn;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float4 *slot = ring + ((p % kJPairs) * 2 + h) * 4 * 32;
        const int a = I * kJT + 8 * (iq >> 2) + (iq & 3) + 4 * h;
        if (a < n_tiles && b < a) {
          jones_load_row(slot, Vn, Mn, a, b);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) slot[e * 32] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      if (++ik == n_mine) {
        ik = 0;
        ++iq;
      }
    }
    cp_async_commit();
  };
  float col[kJQ];
  float row[4][3];
#pragma unroll
  for (int q = 0; q < kJQ; ++q) col[q] = 0.f;
#pragma unroll
  for (int m = 0; m < 4; ++m) row[m][0] = row[m][1] = row[m][2] = 0.f;
  Kahan loss;
#pragma unroll
  for (int k = 0; k < kJPairs - 1; ++k) issue(k);
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll 1
    for (int u = 0; u < 4; ++u) {
      const int q = 4 * m + u;
      float v[2 * kJQ];
#pragma unroll
      for (int k = 0; k < 2 * kJQ; ++k) v[k] = 0.f;
      float lq = 0.f;
#pragma unroll 1
      for (int kc = 0; kc < n_mine; ++kc) {
        const int p = q * n_mine + kc;
        issue(p + kJPairs - 1);
        cp_async_wait<kJPairs - 1>();  // this thread's copies of pair p have landed
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = 8 * m + u + 4 * h;
          const float4 *slot = ring + ((p % kJPairs) * 2 + h) * 4 * 32;
          lq += jones_row<DEN>(slot, sJ[4 * r + 0], sJ[4 * r + 1], sJ[4 * r + 2], sJ[4 * r + 3],
                               jb00, jb01, jb10, jb11, col, v + kJQ * h);
        }
      }
      reduce_scatter24(v, lane);
      if ((lane & 3) == u) {
        row[m][0] += v[0];
        row[m][1] += v[1];
        row[m][2] += v[2];
      }
      loss.add(lq);
    }
  cp_async_wait<0>();
  __syncthreads();  // every warp is done with the ring
  float(*sred)[kJT][kJQ] = reinterpret_cast<float(*)[kJT][kJQ]>(ringbase);
  float *sloss = reinterpret_cast<float *>(ringbase) + kWarps * kJT * kJQ;
  const int out_idx = tile * n_cg + cg;
  // lane 16 hi + 4 g + u keeps quantities 3g .. 3g + 2 of row 8m + u + 4 hi
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      sred[w][8 * m + (lane & 3) + 4 * (lane >> 4)][3 * ((lane >> 2) & 3) + k] = row[m][k];
  float l = loss.s;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if (lane == 0) sloss[w] = l;
  __syncthreads();
  for (int e = threadIdx.x; e < kJT * kJQ; e += kCalThreads) {
    float t = 0.f;
    for (int k = 0; k < kWarps; ++k) t += (&sred[k][0][0])[e];
    part_row[(int64_t)out_idx * kJT * kJQ + e] = t;
  }
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int k = 0; k < kWarps; ++k) t += sloss[k];
    part_loss[out_idx] = t;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kJQ; ++q) sred[w][lane][q] = col[q];
  __syncthreads();
  for (int e = threadIdx.x; e < kJT * kJQ; e += kCalThreads) {
    float t = 0.f;
    for (int k = 0; k < kWarps; ++k) t += (&sred[k][0][0])[e];
    part_col[(int64_t)out_idx * kJT * kJQ + e] = t;
  }
}

// grid: n_jt + 1 blocks of kJT * kJQ threads.  Block K < n_jt: thread (t, q)
// sums quantity q of tile K*32 + t over the row partials of calibration tiles
// (K, J <= K) and the column partials of tiles (I >= K, K), every channel
// group, in that order; then thread t < 32 writes grad = 2 G or (SOLVE) the
// update J <- J - G D^-1 (averaged with J when avg), J kept where
// det D <= 0.  The last block sums the loss partials.
template <bool SOLVE>
__global__ void __launch_bounds__(kJT * kJQ) calib_jones_gather_kernel(
    int n_tiles, int n_jt, int n_cg, const float *__restrict__ part_loss,
    const float *__restrict__ part_row, const float *__restrict__ part_col,
    float *__restrict__ loss, float2 *__restrict__ grad, float2 *__restrict__ J_io, int avg) {
  const int K = blockIdx.x;
  __shared__ float sacc[kJT * kJQ];
  if (K == n_jt) {
    if (!loss) return;
    const int n_part = n_jt * (n_jt + 1) / 2 * n_cg;
    Kahan acc;
    for (int k = threadIdx.x; k < n_part; k += blockDim.x) acc.add(part_loss[k]);
    sacc[threadIdx.x] = acc.s;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int k = 0; k < (int)blockDim.x; ++k) t += sacc[k];
      *loss = t;
    }
    return;
  }
  if (!SOLVE && !grad) return;
  const int e = threadIdx.x;  // = t * kJQ + q
  Kahan acc;
  for (int Jt = 0; Jt <= K; ++Jt) {
    const int tile = K * (K + 1) / 2 + Jt;
    for (int cg = 0; cg < n_cg; ++cg)
      acc.add(part_row[((int64_t)tile * n_cg + cg) * kJT * kJQ + e]);
  }
  for (int It = K; It < n_jt; ++It) {
    const int tile = It * (It + 1) / 2 + K;
    for (int cg = 0; cg < n_cg; ++cg)
      acc.add(part_col[((int64_t)tile * n_cg + cg) * kJT * kJQ + e]);
  }
  sacc[e] = acc.s;
  __syncthreads();
  const int t = threadIdx.x;
  const int a = K * kJT + t;
  if (t >= kJT || a >= n_tiles) return;
  const float *q = sacc + t * kJQ;
  const float2 G00 = make_float2(q[0], q[1]), G01 = make_float2(q[2], q[3]);
  const float2 G10 = make_float2(q[4], q[5]), G11 = make_float2(q[6], q[7]);
  if constexpr (SOLVE) {
    const float d00 = q[8], d11 = q[9];
    const float2 d10 = make_float2(q[10], q[11]);
    const float det = d00 * d11 - cabs2(d10);
    if (!(det > 0.f)) return;
    const float inv = 1.f / det;
    // D^-1 = [[d11, -conj(d10)], [-d10, d00]] / det
    const float2 i00 = make_float2(d11 * inv, 0.f), i11 = make_float2(d00 * inv, 0.f);
    const float2 i01 = make_float2(-d10.x * inv, d10.y * inv), i10 = make_float2(-d10.x * inv, -d10.y * inv);
    const float2 z = make_float2(0.f, 0.f);
    const float2 s00 = cfma(cfma(z, G00, i00), G01, i10), s01 = cfma(cfma(z, G00, i01), G01, i11);
    const float2 s10 = cfma(cfma(z, G10, i00), G11, i10), s11 = cfma(cfma(z, G10, i01), G11, i11);
    float2 *Ja = J_io + (int64_t)a * 4;
    const float2 s[4] = {s00, s01, s10, s11};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 j = Ja[k];
      float2 h = make_float2(j.x - s[k].x, j.y - s[k].y);
      if (avg) h = make_float2(0.5f * (j.x + h.x), 0.5f * (j.y + h.y));
      Ja[k] = h;
    }
  } else {
    float2 *g = grad + (int64_t)a * 4;
    g[0] = make_float2(2.f * G00.x, 2.f * G00.y);
    g[1] = make_float2(2.f * G01.x, 2.f * G01.y);
    g[2] = make_float2(2.f * G10.x, 2.f * G10.y);
    g[3] = make_float2(2.f * G11.x, 2.f * G11.y);
  }
}

bool dev_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct Ws {
  float *loss;
  float2 *row, *col;
  float *rden, *cden;  // gain solve only
};

// Layout: row and column partials, loss partials, then (gain solve) the row
// and column den partials.
Ws carve(void *ws, int n_blocks, int n_cg, bool solve) {
  const int64_t tiles = (int64_t)n_blocks * (n_blocks + 1) / 2;
  uint8_t *p = reinterpret_cast<uint8_t *>(ws);
  Ws w;
  w.row = reinterpret_cast<float2 *>(p);
  p += tiles * n_cg * kCT * sizeof(float2);
  w.col = reinterpret_cast<float2 *>(p);
  p += tiles * n_cg * kCT * sizeof(float2);
  w.loss = reinterpret_cast<float *>(p);
  p += (tiles * n_cg * (int64_t)sizeof(float) + 255) / 256 * 256;
  w.rden = solve ? reinterpret_cast<float *>(p) : nullptr;
  p += tiles * n_cg * kCT * sizeof(float);
  w.cden = solve ? reinterpret_cast<float *>(p) : nullptr;
  return w;
}

constexpr int kChanPerCta = kCalThreads / 32;
constexpr int kMaxCalibChan = 65535 * kChanPerCta;  // grid.y limit

struct ChanWs {
  float *loss;
  float2 *row, *col;
  float *rden, *cden;  // gain solve only
};

int64_t chan_ws_bytes(int n_inputs, int n_chan, bool solve) {
  if (n_inputs < 2 || n_chan < 1 || n_inputs > 65536 || n_chan > kMaxCalibChan) return -1;
  const int64_t nb = (n_inputs + kCT - 1) / kCT;
  const int64_t tiles = nb * (nb + 1) / 2;
  const int64_t n_cy = (n_chan + kChanPerCta - 1) / kChanPerCta;
  const int64_t slots = tiles * n_chan * kCT;
  int64_t b = slots * (int64_t)sizeof(float2) * 2 +
              (tiles * n_cy * (int64_t)sizeof(float) + 255) / 256 * 256;
  if (solve) b += slots * (int64_t)sizeof(float) * 2;
  return b;
}

// Layout: row and column partials, loss partials (256-byte padded), then (gain
// solve) the row and column den partials.
ChanWs chan_carve(void *ws, int nb, int n_chan, int n_cy, bool solve) {
  const int64_t tiles = (int64_t)nb * (nb + 1) / 2;
  const int64_t slots = tiles * n_chan * kCT;
  uint8_t *p = reinterpret_cast<uint8_t *>(ws);
  ChanWs w;
  w.row = reinterpret_cast<float2 *>(p);
  p += slots * sizeof(float2);
  w.col = reinterpret_cast<float2 *>(p);
  p += slots * sizeof(float2);
  w.loss = reinterpret_cast<float *>(p);
  p += (tiles * n_cy * (int64_t)sizeof(float) + 255) / 256 * 256;
  w.rden = solve ? reinterpret_cast<float *>(p) : nullptr;
  p += slots * sizeof(float);
  w.cden = solve ? reinterpret_cast<float *>(p) : nullptr;
  return w;
}

int jones_chan_groups(int n_chan) {
  return n_chan < kJonesChanGroups ? n_chan : kJonesChanGroups;
}

// Layout: row partials, column partials ([tile][cg][32][12] floats each), loss
// partials [tile][cg].
int64_t jones_ws_bytes(int n_inputs, int n_chan) {
  if (n_inputs < 2 || (n_inputs & 1) || n_inputs > 65536 || n_chan < 1) return -1;
  const int64_t n_jt = (n_inputs / 2 + kJT - 1) / kJT;
  const int64_t slots = n_jt * (n_jt + 1) / 2 * jones_chan_groups(n_chan);
  return slots * kJT * kJQ * (int64_t)sizeof(float) * 2 + slots * (int64_t)sizeof(float);
}

}  // namespace
}  // namespace mwax

using namespace mwax;

extern "C" {

int64_t mwax_calib_workspace_bytes(int n_inputs, int n_chan) {
  if (n_inputs < 2 || n_chan < 1) return -1;
  const int64_t nb = (n_inputs + kCT - 1) / kCT;
  const int64_t tiles = nb * (nb + 1) / 2;
  const int64_t cg = chan_groups(n_chan);
  return tiles * cg * kCT * (int64_t)sizeof(float2) * 2 + tiles * cg * (int64_t)sizeof(float) + 256;
}

mwax_status mwax_calib_loss_grad(const float *V, const float *M, const float *g, int n_inputs,
                                 int n_chan, void *workspace, float *loss, float *grad,
                                 cudaStream_t stream) {
  mwax::NvtxRange nvtx_("mwax_calib_loss_grad");
  if (n_inputs < 2 || n_chan < 1 || n_inputs > 65536) return MWAX_ERR_INVALID_ARG;
  if (!loss && !grad) return MWAX_ERR_INVALID_ARG;
  if (!dev_ptr(V) || !dev_ptr(M) || !dev_ptr(g) || !dev_ptr(workspace)) return MWAX_ERR_INVALID_ARG;
  if ((loss && !dev_ptr(loss)) || (grad && !dev_ptr(grad))) return MWAX_ERR_INVALID_ARG;
  const int nb = (n_inputs + kCT - 1) / kCT;
  const int tiles = nb * (nb + 1) / 2;
  const int n_cg = chan_groups(n_chan);
  Ws w = carve(workspace, nb, n_cg, false);
  calib_tile_kernel<false><<<dim3(tiles, n_cg), kCalThreads, 0, stream>>>(
      reinterpret_cast<const float2 *>(V), reinterpret_cast<const float2 *>(M),
      reinterpret_cast<const float2 *>(g), n_inputs, n_chan, n_cg, w.loss, w.row, w.col, nullptr,
      nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return MWAX_ERR_CUDA;
  calib_gather_kernel<false><<<nb + 1, kCalThreads, 0, stream>>>(
      n_inputs, nb, n_cg, w.loss, w.row, w.col, nullptr, nullptr, loss,
      reinterpret_cast<float2 *>(grad), nullptr, 0);
  return cudaGetLastError() == cudaSuccess ? MWAX_OK : MWAX_ERR_CUDA;
}

int64_t mwax_calib_solve_workspace_bytes(int n_inputs, int n_chan) {
  if (n_inputs < 2 || n_chan < 1) return -1;
  const int64_t nb = (n_inputs + kCT - 1) / kCT;
  const int64_t tiles = nb * (nb + 1) / 2;
  const int64_t cg = chan_groups(n_chan);
  return tiles * cg * kCT * (int64_t)sizeof(float2) * 2 +
         (tiles * cg * (int64_t)sizeof(float) + 255) / 256 * 256 +
         tiles * cg * kCT * (int64_t)sizeof(float) * 2 + 256;
}

mwax_status mwax_calib_solve(const float *V, const float *M, float *g, int n_inputs, int n_chan,
                             int n_iter, void *workspace, float *loss_hist, cudaStream_t stream) {
  mwax::NvtxRange nvtx_("mwax_calib_solve");
  if (n_inputs < 2 || n_chan < 1 || n_inputs > 65536 || n_iter < 0) return MWAX_ERR_INVALID_ARG;
  if (!dev_ptr(V) || !dev_ptr(M) || !dev_ptr(g) || !dev_ptr(workspace)) return MWAX_ERR_INVALID_ARG;
  if (loss_hist && !dev_ptr(loss_hist)) return MWAX_ERR_INVALID_ARG;
  const int nb = (n_inputs + kCT - 1) / kCT;
  const int tiles = nb * (nb + 1) / 2;
  const int n_cg = chan_groups(n_chan);
  Ws w = carve(workspace, nb, n_cg, true);
  float2 *g2 = reinterpret_cast<float2 *>(g);
  for (int t = 1; t <= n_iter; ++t) {
    calib_tile_kernel<true><<<dim3(tiles, n_cg), kCalThreads, 0, stream>>>(
        reinterpret_cast<const float2 *>(V), reinterpret_cast<const float2 *>(M), g2, n_inputs,
        n_chan, n_cg, w.loss, w.row, w.col, w.rden, w.cden);
    if (cudaGetLastError() != cudaSuccess) return MWAX_ERR_CUDA;
    calib_gather_kernel<true><<<nb + 1, kCalThreads, 0, stream>>>(
        n_inputs, nb, n_cg, w.loss, w.row, w.col, w.rden, w.cden,
        loss_hist ? loss_hist + (t - 1) : nullptr, nullptr, g2, (t % 2 == 0) ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess) return MWAX_ERR_CUDA;
  }
  return MWAX_OK;
}

int64_t mwax_calib_chan_workspace_bytes(int n_inputs, int n_chan) {
  return chan_ws_bytes(n_inputs, n_chan, false);
}

int64_t mwax_calib_chan_solve_workspace_bytes(int n_inputs, int n_chan) {
  return chan_ws_bytes(n_inputs, n_chan, true);
}

mwax_status mwax_calib_chan_loss_grad(const float *V, const float *M, const float *g,
                                      int n_inputs, int n_chan, void *workspace, float *loss,
                                      float *grad, cudaStream_t stream) {
  mwax::NvtxRange nvtx_("mwax_calib_chan_loss_grad");
  if (chan_ws_bytes(n_inputs, n_chan, false) < 0) return MWAX_ERR_INVALID_ARG;
  if (!loss && !grad) return MWAX_ERR_INVALID_ARG;
  if (!dev_ptr(V) || !dev_ptr(M) || !dev_ptr(g) || !dev_ptr(workspace)) return MWAX_ERR_INVALID_ARG;
  if ((loss && !dev_ptr(loss)) || (grad && !dev_ptr(grad))) return MWAX_ERR_INVALID_ARG;
  const int nb = (n_inputs + kCT - 1) / kCT;
  const int tiles = nb * (nb + 1) / 2;
  const int n_cy = (n_chan + kChanPerCta - 1) / kChanPerCta;
  ChanWs w = chan_carve(workspace, nb, n_chan, n_cy, false);
  calib_chan_tile_kernel<false><<<dim3(tiles, n_cy), kCalThreads, 0, stream>>>(
      reinterpret_cast<const float2 *>(V), reinterpret_cast<const float2 *>(M),
      reinterpret_cast<const float2 *>(g), n_inputs, n_chan, w.loss, w.row, w.col, nullptr,
      nullptr);
  if (cudaGetLastError() != cudaSuccess) return MWAX_ERR_CUDA;
  calib_chan_gather_kernel<false><<<dim3(nb + 1, n_cy), kCalThreads, 0, stream>>>(
      n_inputs, n_chan, nb, w.loss, w.row, w.col, nullptr, nullptr, loss,
      reinterpret_cast<float2 *>(grad), nullptr, 0);
  return cudaGetLastError() == cudaSuccess ? MWAX_OK : MWAX_ERR_CUDA;
}

mwax_status mwax_calib_chan_solve(const float *V, const float *M, float *g, int n_inputs,
                                  int n_chan, int n_iter, void *workspace, float *loss_hist,
                                  cudaStream_t stream) {
  mwax::NvtxRange nvtx_("mwax_calib_chan_solve");
  if (chan_ws_bytes(n_inputs, n_chan, true) < 0 || n_iter < 0) return MWAX_ERR_INVALID_ARG;
  if (!dev_ptr(V) || !dev_ptr(M) || !dev_ptr(g) || !dev_ptr(workspace)) return MWAX_ERR_INVALID_ARG;
  if (loss_hist && !dev_ptr(loss_hist)) return MWAX_ERR_INVALID_ARG;
  const int nb = (n_inputs + kCT - 1) / kCT;
  const int tiles = nb * (nb + 1) / 2;
  const int n_cy = (n_chan + kChanPerCta - 1) / kChanPerCta;
  ChanWs w = chan_carve(workspace, nb, n_chan, n_cy, true);
  float2 *g2 = reinterpret_cast<float2 *>(g);
  for (int t = 1; t <= n_iter; ++t) {
    calib_chan_tile_kernel<true><<<dim3(tiles, n_cy), kCalThreads, 0, stream>>>(
        reinterpret_cast<const float2 *>(V), reinterpret_cast<const float2 *>(M), g2, n_inputs,
        n_chan, w.loss, w.row, w.col, w.rden, w.cden);
    if (cudaGetLastError() != cudaSuccess) return MWAX_ERR_CUDA;
    calib_chan_gather_kernel<true><<<dim3(nb + 1, n_cy), kCalThreads, 0, stream>>>(
        n_inputs, n_chan, nb, w.loss, w.row, w.col, w.rden, w.cden,
        loss_hist ? loss_hist + (t - 1) : nullptr, nullptr, g2, (t % 2 == 0) ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess) return MWAX_ERR_CUDA;
  }
  return MWAX_OK;
}

// ---- full 2x2 Jones matrices ------------------------------------------------------
int64_t mwax_calib_jones_workspace_bytes(int n_inputs, int n_chan) {
  return jones_ws_bytes(n_inputs, n_chan);
}

static mwax_status jones_run(const float *V, const float *M, float *J, int n_inputs, int n_chan,
                             int n_iter, bool solve, void *workspace, float *loss, float *grad,
                             cudaStream_t stream) {
  const int n_tiles = n_inputs / 2;
  const int n_jt = (n_tiles + kJT - 1) / kJT;
  const int tiles = n_jt * (n_jt + 1) / 2;
  const int n_cg = jones_chan_groups(n_chan);
  const int64_t slots = (int64_t)tiles * n_cg;
  float *prow = reinterpret_cast<float *>(workspace);
  float *pcol = prow + slots * kJT * kJQ;
  float *ploss = pcol + slots * kJT * kJQ;
  const float2 *V2 = reinterpret_cast<const float2 *>(V), *M2 = reinterpret_cast<const float2 *>(M);
  float2 *J2 = reinterpret_cast<float2 *>(J);
  // the two-rows-per-step pass needs more than the default 48 KB of shared memory
  constexpr int smem2 = jones2_smem_bytes();
  if (cudaFuncSetAttribute(calib_jones_tile2_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem2) != cudaSuccess ||
      cudaFuncSetAttribute(calib_jones_tile2_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem2) != cudaSuccess)
    return MWAX_ERR_CUDA;
  auto tile_pass = [&](bool den) {
    if (den)
      calib_jones_tile2_kernel<true><<<dim3(tiles, n_cg), kCalThreads, smem2, stream>>>(
          V2, M2, J2, n_tiles, n_chan, n_cg, ploss, prow, pcol);
    else
      calib_jones_tile2_kernel<false><<<dim3(tiles, n_cg), kCalThreads, smem2, stream>>>(
          V2, M2, J2, n_tiles, n_chan, n_cg, ploss, prow, pcol);
  };
  if (!solve) {
    tile_pass(false);
    if (cudaGetLastError() != cudaSuccess) return MWAX_ERR_CUDA;
    calib_jones_gather_kernel<false><<<n_jt + 1, kJT * kJQ, 0, stream>>>(
        n_tiles, n_jt, n_cg, ploss, prow, pcol, loss, reinterpret_cast<float2 *>(grad), nullptr, 0);
    return cudaGetLastError() == cudaSuccess ? MWAX_OK : MWAX_ERR_CUDA;
  }
  for (int t = 1; t <= n_iter; ++t) {
    tile_pass(true);
    if (cudaGetLastError() != cudaSuccess) return MWAX_ERR_CUDA;
    calib_jones_gather_kernel<true><<<n_jt + 1, kJT * kJQ, 0, stream>>>(
        n_tiles, n_jt, n_cg, ploss, prow, pcol, loss ? loss + (t - 1) : nullptr, nullptr, J2,
        (t % 2 == 0) ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess) return MWAX_ERR_CUDA;
  }
  return MWAX_OK;
}

mwax_status mwax_calib_jones_loss_grad(const float *V, const float *M, const float *J,
                                       int n_inputs, int n_chan, void *workspace, float *loss,
                                       float *grad, cudaStream_t stream) {
  mwax::NvtxRange nvtx_("mwax_calib_jones_loss_grad");
  if (jones_ws_bytes(n_inputs, n_chan) < 0) return MWAX_ERR_INVALID_ARG;
  if (!loss && !grad) return MWAX_ERR_INVALID_ARG;
  if (!dev_ptr(V) || !dev_ptr(M) || !dev_ptr(J) || !dev_ptr(workspace)) return MWAX_ERR_INVALID_ARG;
  if ((loss && !dev_ptr(loss)) || (grad && !dev_ptr(grad))) return MWAX_ERR_INVALID_ARG;
  return jones_run(V, M, const_cast<float *>(J), n_inputs, n_chan, 0, false, workspace, loss, grad,
                   stream);
}

mwax_status mwax_calib_jones_solve(const float *V, const float *M, float *J, int n_inputs,
                                   int n_chan, int n_iter, void *workspace, float *loss_hist,
                                   cudaStream_t stream) {
  mwax::NvtxRange nvtx_("mwax_calib_jones_solve");
  if (jones_ws_bytes(n_inputs, n_chan) < 0 || n_iter < 0) return MWAX_ERR_INVALID_ARG;
  if (!dev_ptr(V) || !dev_ptr(M) || !dev_ptr(J) || !dev_ptr(workspace)) return MWAX_ERR_INVALID_ARG;
  if (loss_hist && !dev_ptr(loss_hist)) return MWAX_ERR_INVALID_ARG;
  return jones_run(V, M, J, n_inputs, n_chan, n_iter, true, workspace, loss_hist, nullptr, stream);
}

mwax_status mwax_calib_loss(const float *V, const float *M, const float *g, int n_inputs,
                            int n_chan, void *workspace, float *loss, cudaStream_t stream) {
  if (!loss) return MWAX_ERR_INVALID_ARG;
  return mwax_calib_loss_grad(V, M, g, n_inputs, n_chan, workspace, loss, nullptr, stream);
}

mwax_status mwax_calib_grad(const float *V, const float *M, const float *g, int n_inputs,
                            int n_chan, void *workspace, float *grad, cudaStream_t stream) {
  if (!grad) return MWAX_ERR_INVALID_ARG;
  return mwax_calib_loss_grad(V, M, g, n_inputs, n_chan, workspace, nullptr, grad, stream);
}

}  // extern "C"

// ---- allocation-free variant ---------------------------------------------------
// Some callers cannot allocate device memory at the point where they evaluate
// the loss: a real-time loop (like the MWA's) where cudaMalloc/cudaFree would
// add device-wide synchronisation and unbounded latency to every integration,
// or a host application whose device memory is entirely owned by another
// allocator.  For them, the partial sums live in this fixed array instead of
// a caller-provided workspace.  Every GPU that loads the library holds the
// array until the process exits.
namespace mwax {
namespace {

constexpr int64_t kStaticWsBytes = int64_t(4) << 20;  // 4 MiB: 1024 inputs need ~3.3 MB
static __device__ __align__(256) uint8_t g_calib_static_ws[kStaticWsBytes];

constexpr int kMaxStaticDevices = 256;
std::mutex g_static_ws_mu;
void *g_static_ws_addr[kMaxStaticDevices];

// Device address of the array on the current device.  Host code cannot use
// the array's name as a device pointer, so the address is asked of the
// runtime with the device current.  Outside stream capture it is looked up
// on every call (no allocation; this also follows a cudaDeviceReset, after
// which the module is loaded again at another address); during a capture the
// address remembered from the device's last uncaptured call is used, and a
// device with no such call is refused.
cudaError_t static_ws_address(cudaStream_t stream, void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxStaticDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_static_ws_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_calib_static_ws);
    if (e != cudaSuccess) return e;
    g_static_ws_addr[dev] = p;
  } else if (!g_static_ws_addr[dev]) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_static_ws_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace mwax

extern "C" int64_t mwax_calib_static_workspace_bytes(void) { return mwax::kStaticWsBytes; }

extern "C" mwax_status mwax_calib_loss_grad_static(const float *V, const float *M, const float *g,
                                                   int n_inputs, int n_chan, float *loss,
                                                   float *grad, cudaStream_t stream) {
  const int64_t need = mwax_calib_workspace_bytes(n_inputs, n_chan);
  if (need < 0 || need > mwax::kStaticWsBytes) return MWAX_ERR_INVALID_ARG;
  void *ws = nullptr;
  if (mwax::static_ws_address(stream, &ws) != cudaSuccess) return MWAX_ERR_CUDA;
  // Every partial-sum slot the gather kernel reads is written first by the
  // tile kernel of the same call, so nothing in the array needs clearing.
  return mwax_calib_loss_grad(V, M, g, n_inputs, n_chan, ws, loss, grad, stream);
}
