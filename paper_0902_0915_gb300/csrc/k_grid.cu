// k_grid.cu -- gridding of correlator output onto polarisation uv grids.
//
// Paper Sec. 2.1: the calibrated visibilities are convolved onto a regular
// grid so that an FFT can form the images; Sec. 3.2: on the GPU every
// "scatter" step of the CPU code became a "gather" step, each thread
// collecting the values of its own output location (no floating-point
// atomics).  Definition (the paper names no kernel or sizes):
//   every tile baseline a > b and channel c (nu = f0 + c df) is a point at
//       x = (X_a - X_b) nu / c_light / du + Ng/2,  y = (Y_a - Y_b) nu / c_light / du + Ng/2
//   carrying its four polarisation products V_pq (input 2a+p with 2b+q), and
//   the reversed baseline is the point (Ng - x, Ng - y) carrying
//   conj(V_qp).  A point adds V w(s - x, r - y) to cell (r, s) of grid
//   2p+q for |s - x| < W/2 and |r - y| < W/2, w(dx, dy) =
//   exp(-(dx^2 + dy^2) / (2 sigma^2)); cells outside [0, Ng) are dropped.
//
// Plan (geometry only, once per array layout and band):
//   1. per point: position (FP64, so the support sets match an FP64
//      definition exactly), support bounds, and its bin = the first cell of
//      its support (r_lo, s_lo), shifted by W-1 so bins of points that reach
//      row or column 0 are >= 0;
//   2. counting sort by bin (integer atomics for counts and slots, an
//      exclusive prefix sum for bin offsets), then every bin's ids sorted
//      ascending so the order of each gathered sum is fixed;
//   3. per sorted point: last support cell (r_hi, s_hi), first support
//      column, point id;
//   4. the weights: the cells are cut into patches of 4 x 8 (one warp each);
//      the candidates of a patch are the points whose support can reach it,
//      in a fixed order (bin rows, then bin columns, then point id: per bin
//      row one contiguous range of the sorted points).  The Gaussian is
//      separable, w = wx(s - x) wy(r - y), and the support is a rectangle, so
//      for every candidate the plan stores its 8 column factors and 4 row
//      factors (12 floats, computed in FP64, 0 outside the support), and the
//      patches in order of decreasing candidate count (the dense centre of
//      the uv plane first, so the longest warps do not start last).
// Grid call (per integration): one kernel gathers each sorted point's four
// polarisation values from the int32 correlator output; then each warp walks
// its patch's candidates in the plan's order, reads the candidate's values
// once for the whole warp (a broadcast) and its 12 factors, and every lane
// adds wx[col] wy[row] x values (four complex multiply-adds).  No support
// tests and no exponentials per call; deterministic.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "mwax_internal.h"

namespace mwax {
namespace {

constexpr double kCLight = 299792458.0;
constexpr int kScanBlock = 1024;

// Weights are formed at plan time from the FP64 position, recomputed from the
// point id (an absolute float coordinate up to Ng would lose ~1e-4 cells).
struct GeomRec {  // sorted point (12 B)
  int hi;        // r_hi << 16 | s_hi (both in [0, Ng))
  int id;        // point id: ((c * n_tbl) + tbl) * 2 + side
  int slo;       // s_lo + W - 1
};

__device__ __forceinline__ void tbl_pair(int tbl, int &a, int &b) {
  // tbl = a(a-1)/2 + b, a > b >= 0
  int i = (int)((sqrtf(8.0f * (float)tbl + 1.0f) + 1.0f) * 0.5f);
  while (i * (i - 1) / 2 > tbl) --i;
  while ((i + 1) * i / 2 <= tbl) ++i;
  a = i;
  b = tbl - i * (i - 1) / 2;
}

struct GridGeom {
  const double *tile_xy;
  int n_tiles, n_chan, n_tbl, Ng, W;
  double f0, df, du;
  int nbw;  // bins per row: Ng + W - 1
};

// 1. positions, support bounds and bins (bin -1: no cell of the grid reached)
__global__ void grid_points_kernel(GridGeom g, int64_t n_pts, int *__restrict__ bin,
                                   int *__restrict__ hi) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n_pts) return;
  const int side = (int)(k & 1);
  const int64_t ct = k >> 1;
  const int c = (int)(ct / g.n_tbl), tbl = (int)(ct % g.n_tbl);
  int a, b;
  tbl_pair(tbl, a, b);
  const double nu = g.f0 + (double)c * g.df;
  double x = (g.tile_xy[2 * a] - g.tile_xy[2 * b]) * nu / kCLight / g.du + 0.5 * g.Ng;
  double y = (g.tile_xy[2 * a + 1] - g.tile_xy[2 * b + 1]) * nu / kCLight / g.du + 0.5 * g.Ng;
  if (side) {
    x = (double)g.Ng - x;
    y = (double)g.Ng - y;
  }
  const double half = 0.5 * g.W;
  // cells strictly within half the support: the smallest integer above x - W/2
  // and the largest below x + W/2
  const int s_lo = (int)floor(x - half) + 1, s_hi = (int)ceil(x + half) - 1;
  const int r_lo = (int)floor(y - half) + 1, r_hi = (int)ceil(y + half) - 1;
  const bool reach = s_hi >= 0 && s_lo <= g.Ng - 1 && r_hi >= 0 && r_lo <= g.Ng - 1 &&
                     s_lo >= -(g.W - 1) && r_lo >= -(g.W - 1);
  if (!reach) {
    bin[k] = -1;
    hi[k] = 0;
    return;
  }
  bin[k] = (r_lo + g.W - 1) * g.nbw + (s_lo + g.W - 1);
  hi[k] = (min(r_hi, g.Ng - 1) << 16) | min(s_hi, g.Ng - 1);
}

__global__ void grid_count_kernel(const int *__restrict__ bin, int64_t n_pts, int *__restrict__ count) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n_pts && bin[k] >= 0) atomicAdd(&count[bin[k]], 1);
}

// exclusive prefix sum in three passes: per-block scan with block totals,
// scan of the totals (one block), add the block offsets
__global__ void __launch_bounds__(kScanBlock) scan_blocks_kernel(const int *__restrict__ in, int n,
                                                                 int *__restrict__ out,
                                                                 int *__restrict__ totals) {
  __shared__ int sh[kScanBlock];
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  const int v = i < n ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < kScanBlock; o <<= 1) {
    const int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = sh[threadIdx.x] - v;  // exclusive
  if (threadIdx.x == kScanBlock - 1) totals[blockIdx.x] = sh[threadIdx.x];
}

__global__ void __launch_bounds__(kScanBlock) scan_totals_kernel(int *__restrict__ totals, int n) {
  // one block: exclusive scan of n block totals in chunks of kScanBlock
  __shared__ int sh[kScanBlock];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += kScanBlock) {
    const int i = base + threadIdx.x;
    const int v = i < n ? totals[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kScanBlock; o <<= 1) {
      const int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < n) totals[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) carry += sh[threadIdx.x];
    __syncthreads();
  }
}

// (the count array carries one extra zero entry, so the last exclusive offset
// is the total)
__global__ void scan_add_kernel(int *__restrict__ out, int n, const int *__restrict__ totals) {
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) out[i] += totals[blockIdx.x];
}

__global__ void grid_fill_kernel(const int *__restrict__ bin, int64_t n_pts,
                                 const int *__restrict__ offsets, int *__restrict__ fill,
                                 int *__restrict__ ids) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n_pts || bin[k] < 0) return;
  const int b = bin[k];
  ids[offsets[b] + atomicAdd(&fill[b], 1)] = (int)k;
}

// ids of every bin ascending (insertion sort; bins are short)
__global__ void grid_sort_bins_kernel(const int *__restrict__ offsets, int n_bins,
                                      int *__restrict__ ids) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_bins) return;
  const int lo = offsets[b], hi = offsets[b + 1];
  for (int i = lo + 1; i < hi; ++i) {
    const int v = ids[i];
    int j = i - 1;
    while (j >= lo && ids[j] > v) {
      ids[j + 1] = ids[j];
      --j;
    }
    ids[j + 1] = v;
  }
}

__global__ void grid_records_kernel(const int *__restrict__ ids, int n_kept,
                                    const int *__restrict__ hi,
                                    const int *__restrict__ bin, int nbw, GeomRec *__restrict__ rec) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_kept) return;
  const int k = ids[p];
  GeomRec r;
  r.hi = hi[k];
  r.id = k;
  r.slo = bin[k] % nbw;
  rec[p] = r;
}

// Cell position of a point in FP64, from its id ((c * n_tbl + tbl) * 2 + side).
__device__ __forceinline__ void point_xy(const GridGeom &g, int id, double &x, double &y) {
  const int side = id & 1;
  const int ct = id >> 1;
  const int c = ct / g.n_tbl, tbl = ct % g.n_tbl;
  int a, b;
  tbl_pair(tbl, a, b);
  const double nu = g.f0 + (double)c * g.df;
  x = (g.tile_xy[2 * a] - g.tile_xy[2 * b]) * nu / kCLight / g.du + 0.5 * g.Ng;
  y = (g.tile_xy[2 * a + 1] - g.tile_xy[2 * b + 1]) * nu / kCLight / g.du + 0.5 * g.Ng;
  if (side) {
    x = (double)g.Ng - x;
    y = (double)g.Ng - y;
  }
}

// Patches: a warp owns rows r0 .. r0+3, columns s0 .. s0+7.  The warp's lanes
// form kGroups groups of 32 / kGroups lanes; group g takes candidates
// j = g (mod kGroups), and lane l of a group holds kGroups cells of one row
// (r0 + l / (8 / kGroups), columns s0 + kGroups (l % (8 / kGroups)) + {0 ..
// kGroups-1}), so one value broadcast and one load of kGroups column factors
// serve kGroups cells; the groups' sums are added at the end.  A CTA runs 8
// patches.
#ifndef MWAX_GRID_GROUPS
#define MWAX_GRID_GROUPS 2
#endif
constexpr int kGroups = MWAX_GRID_GROUPS;  // 1, 2 or 4 (measured: 1.64, 1.42, 1.46 ms per c5 call)
constexpr int kGLanes = 32 / kGroups, kRowLanes = 8 / kGroups;
constexpr int kPatchR = 4, kPatchC = 8;
constexpr int kPatchThreads = 32 * 8;

constexpr int kFactors = kPatchC + kPatchR;  // per candidate: 8 column, 4 row factors

struct Patch {
  int r0, s0, br_end, bc_end;
};

// Patch `idx` (row-major over patch rows and columns).
__device__ __forceinline__ Patch patch_at(int idx, int n_patch_c, int W, int nbw) {
  Patch pt;
  pt.r0 = (idx / n_patch_c) * kPatchR;
  pt.s0 = (idx % n_patch_c) * kPatchC;
  // bin row br holds points with r_lo = br - (W - 1); those reaching rows
  // r0 .. r0+3 have br in [r0, r0 + 3 + W - 1]; likewise bin columns
  pt.br_end = min(pt.r0 + kPatchR - 1 + W - 1, nbw - 1);
  pt.bc_end = min(pt.s0 + kPatchC + W - 1, nbw);  // exclusive
  return pt;
}

// 4a. candidates per patch (into cnt[patch])
__global__ void __launch_bounds__(kPatchThreads) grid_patch_count_kernel(
    const int *__restrict__ offsets, int n_patches, int W, int nbw, int n_patch_c,
    int *__restrict__ cnt) {
  const int idx = blockIdx.x * (kPatchThreads / 32) + (threadIdx.x >> 5);
  if (idx >= n_patches) return;
  const Patch pt = patch_at(idx, n_patch_c, W, nbw);
  const int lane = threadIdx.x & 31;
  int n = 0;
  for (int br = pt.r0 + lane; br <= pt.br_end; br += 32)
    n += offsets[br * nbw + pt.bc_end] - offsets[br * nbw + pt.s0];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if (lane == 0) cnt[idx] = n;
}

// 4b. the factors of every candidate of a patch, from w_off[patch] * 12:
// lanes 0..7 the column factors wx(s0 + l - x), lanes 8..11 the row factors
// wy(r0 + l - 8 - y), each 0 outside the support or the grid.
__global__ void __launch_bounds__(kPatchThreads) grid_patch_weights_kernel(
    GridGeom g, const GeomRec *__restrict__ rec, const int *__restrict__ offsets, double inv_2s2d,
    int n_patches, int n_patch_c, const int *__restrict__ w_off, float *__restrict__ wts) {
  const int idx = blockIdx.x * (kPatchThreads / 32) + (threadIdx.x >> 5);
  if (idx >= n_patches) return;
  const int W = g.W, nbw = g.nbw;
  const Patch pt = patch_at(idx, n_patch_c, W, nbw);
  const int lane = threadIdx.x & 31;
  const bool col = lane < kPatchC, row = lane >= kPatchC && lane < kFactors;
  const int s = pt.s0 + lane, r = pt.r0 + lane - kPatchC;
  int64_t k = (int64_t)w_off[idx] * kFactors + lane;
  for (int br = pt.r0; br <= pt.br_end; ++br) {
    const int r_lo = br - (W - 1);
    const int lo = offsets[br * nbw + pt.s0], hi = offsets[br * nbw + pt.bc_end];
    for (int q = lo; q < hi; ++q, k += kFactors) {
      if (!col && !row) continue;
      const GeomRec p = rec[q];
      const int s_lo = p.slo - (W - 1);
      float f = 0.f;
      double x, y;
      if (col && s >= s_lo && s <= (p.hi & 0xFFFF) && s < g.Ng) {
        point_xy(g, p.id, x, y);
        const double d = (double)s - x;
        f = (float)exp(-d * d * inv_2s2d);
      } else if (row && r >= r_lo && r <= (p.hi >> 16) && r < g.Ng) {
        point_xy(g, p.id, x, y);
        const double d = (double)r - y;
        f = (float)exp(-d * d * inv_2s2d);
      }
      wts[k] = f;
    }
  }
}

// sorted position of every point id (-1: the point reaches no cell)
__global__ void grid_slot_kernel(const GeomRec *__restrict__ rec, int n_kept, int *__restrict__ slot) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n_kept) slot[rec[p].id] = p;
}

// grid call, step 1: the four polarisation values of every point, read in
// point-id order (channel, then baseline: nearly sequential in the
// correlator output) and written to the point's sorted position
__global__ void grid_values_kernel(const int *__restrict__ slot, int n_pts, int n_tbl,
                                   int64_t n_bl, const int2 *__restrict__ vis,
                                   float4 *__restrict__ vals) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n_pts) return;
  const int p = slot[id];
  if (p < 0) return;
  const int side = id & 1;
  const int ct = id >> 1;
  const int c = ct / n_tbl, tbl = ct % n_tbl;
  int a, b;
  tbl_pair(tbl, a, b);
  const int2 *vc = vis + (int64_t)c * n_bl;
  float v[8];
#pragma unroll
  for (int pp = 0; pp < 2; ++pp)
#pragma unroll
    for (int qq = 0; qq < 2; ++qq) {
      // forward point: product (pp, qq) of (a, b); reversed: conj of (qq, pp)
      const int ip = side ? qq : pp, jq = side ? pp : qq;
      const int64_t i = 2 * a + ip, j = 2 * b + jq;
      const int2 x = vc[i * (i + 1) / 2 + j];
      v[2 * (2 * pp + qq)] = (float)x.x;
      v[2 * (2 * pp + qq) + 1] = side ? -(float)x.y : (float)x.y;
    }
  vals[2 * (int64_t)p] = make_float4(v[0], v[1], v[2], v[3]);
  vals[2 * (int64_t)p + 1] = make_float4(v[4], v[5], v[6], v[7]);
}

// grid call, step 2: every cell of a patch sums, in the plan's candidate order,
// wx[col] wy[row] x values.  apply_range adds candidates [k0, k1) of a patch
// for this lane's cell.
constexpr int kHeavy = 1024;  // patches with more candidates get a whole CTA

struct Acc {
  float2 v[kGroups][4];  // the lane's cells x four polarisation products
};

// Per-warp staging of 32 candidates: their values (8 floats) and factors
// (12 floats), double-buffered; plus the patch's bin rows (first candidate
// index and first sorted point of each).
constexpr int kMaxRows = 40;  // >= kPatchR - 1 + W for W <= 31
struct WarpStage {
  float4 v[2][32][2];
  float f[2][32][kFactors];
  int row_k[kMaxRows + 1], row_q[kMaxRows];
};

__device__ __forceinline__ void cp16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}

// Adds candidates [k0, k1) of the patch to this lane's cell: 32 candidates at
// a time are copied (one per lane) into the warp's staging buffer while the
// previous 32 are applied, in candidate order.
__device__ __forceinline__ void apply_range(const Patch &pt, int nbw, const int *__restrict__ offsets,
                                            const float *__restrict__ wf0,
                                            const float4 *__restrict__ vals, int k0, int k1,
                                            int lane, WarpStage &st, Acc &acc) {
  // group hw takes candidates j + hw; this lane's column factors
  // kGroups (l % kRowLanes) + {0 .. kGroups-1} and its row factor, l = lane % kGLanes
  const int hw = lane / kGLanes, hl = lane % kGLanes;
  const int fx = kGroups * (hl % kRowLanes), fy = kPatchC + hl / kRowLanes;
  // bin rows of the patch: candidate index of each row's first point
  const int n_rows = pt.br_end - pt.r0 + 1;
  if (lane == 0) {
    int k = 0;
    for (int i = 0; i < n_rows; ++i) {
      const int br = pt.r0 + i;
      const int lo = __ldg(offsets + br * nbw + pt.s0), hi = __ldg(offsets + br * nbw + pt.bc_end);
      st.row_k[i] = k;
      st.row_q[i] = lo;
      k += hi - lo;
    }
    st.row_k[n_rows] = k;
  }
  __syncwarp();
  auto issue = [&](int base, int buf) {  // candidates base .. base+31 (those < k1)
    const int kk = base + lane;
    if (kk < k1) {
      int i = 0;
      while (st.row_k[i + 1] <= kk) ++i;
      const int q = st.row_q[i] + (kk - st.row_k[i]);
      cp16(&st.v[buf][lane][0], vals + 2 * (int64_t)q);
      cp16(&st.v[buf][lane][1], vals + 2 * (int64_t)q + 1);
      const float *f = wf0 + (int64_t)kk * kFactors;
      cp16(&st.f[buf][lane][0], f);
      cp16(&st.f[buf][lane][4], f + 4);
      cp16(&st.f[buf][lane][8], f + 8);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  int buf = 0;
  if (k0 < k1) issue(k0, 0);
  for (int base = k0; base < k1; base += 32, buf ^= 1) {
    if (base + 32 < k1) {
      issue(base + 32, buf ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncwarp();
    const int n = min(32, k1 - base);
    for (int j0 = 0; j0 < n; j0 += kGroups) {
      const int j = j0 + hw;
      if (j < n) {
        float wx[kGroups];
        if constexpr (kGroups == 4) {
          const float4 t = *reinterpret_cast<const float4 *>(&st.f[buf][j][fx]);
          wx[0] = t.x;
          wx[1] = t.y;
          wx[2] = t.z;
          wx[3] = t.w;
        } else if constexpr (kGroups == 2) {
          const float2 t = *reinterpret_cast<const float2 *>(&st.f[buf][j][fx]);
          wx[0] = t.x;
          wx[1] = t.y;
        } else {
          wx[0] = st.f[buf][j][fx];
        }
        const float wy = st.f[buf][j][fy];
        const float4 a = st.v[buf][j][0], b = st.v[buf][j][1];
#pragma unroll
        for (int c = 0; c < kGroups; ++c) {
          const float w = wx[c] * wy;
          acc.v[c][0].x += w * a.x;
          acc.v[c][0].y += w * a.y;
          acc.v[c][1].x += w * a.z;
          acc.v[c][1].y += w * a.w;
          acc.v[c][2].x += w * b.x;
          acc.v[c][2].y += w * b.y;
          acc.v[c][3].x += w * b.z;
          acc.v[c][3].y += w * b.w;
        }
      }
    }
    __syncwarp();  // this buffer is refilled two steps on
  }
  // the groups' sums into every lane of group 0 (fixed order: a butterfly
  // over the group bits)
#pragma unroll
  for (int o = kGLanes; o < 32; o <<= 1)
#pragma unroll
    for (int c = 0; c < kGroups; ++c)
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        acc.v[c][p].x += __shfl_xor_sync(0xffffffffu, acc.v[c][p].x, o);
        acc.v[c][p].y += __shfl_xor_sync(0xffffffffu, acc.v[c][p].y, o);
      }
}

// The lanes of group 0 store their cells (the other groups hold the same sums).
__device__ __forceinline__ void store_cell(const Patch &pt, int lane, int Ng, const Acc &acc,
                                           float2 *__restrict__ grids) {
  if (lane >= kGLanes) return;
  const int r = pt.r0 + lane / kRowLanes, s = pt.s0 + kGroups * (lane % kRowLanes);
  if (r >= Ng) return;
  const int64_t cell = (int64_t)r * Ng + s;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    float2 *g = grids + (int64_t)p * Ng * Ng + cell;
#pragma unroll
    for (int c = 0; c < kGroups; ++c)
      if (s + c < Ng) g[c] = acc.v[c][p];
  }
}

// Heavy patches (order[0 .. n_heavy)): one CTA each; warp w takes the w-th
// eighth of the candidates, and warp 0 adds the eight partial sums in warp
// order.
__global__ void __launch_bounds__(kPatchThreads) grid_apply_heavy_kernel(
    const int *__restrict__ offsets, const int *__restrict__ order, const int *__restrict__ w_off,
    const float *__restrict__ wts, const float4 *__restrict__ vals, int Ng, int W, int nbw,
    int n_patch_c, float2 *__restrict__ grids) {
  __shared__ WarpStage stage[kPatchThreads / 32];
  const int idx = __ldg(order + blockIdx.x);
  const Patch pt = patch_at(idx, n_patch_c, W, nbw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int first = __ldg(w_off + idx), count = __ldg(w_off + idx + 1) - first;
  const int nw = kPatchThreads / 32;
  Acc acc;
#pragma unroll
  for (int c = 0; c < kGroups; ++c)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc.v[c][p] = make_float2(0.f, 0.f);
  apply_range(pt, nbw, offsets, wts + (int64_t)first * kFactors, vals,
              (int)((int64_t)count * warp / nw), (int)((int64_t)count * (warp + 1) / nw), lane,
              stage[warp], acc);
  // the partial sums reuse the staging memory once every warp is done with it
  __syncthreads();
  float2(*part)[kGroups][4][kGLanes] = reinterpret_cast<float2(*)[kGroups][4][kGLanes]>(stage);
  static_assert(sizeof(float2) * (kPatchThreads / 32) * 4 * 32 <= sizeof(WarpStage) * (kPatchThreads / 32),
                "aliasing");
  if (lane < kGLanes)
#pragma unroll
    for (int c = 0; c < kGroups; ++c)
#pragma unroll
      for (int p = 0; p < 4; ++p) part[warp][c][p][lane] = acc.v[c][p];
  __syncthreads();
  if (warp == 0 && lane < kGLanes) {
#pragma unroll
    for (int c = 0; c < kGroups; ++c)
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        float2 t = part[0][c][p][lane];
#pragma unroll 1
        for (int w = 1; w < nw; ++w) {
          t.x += part[w][c][p][lane].x;
          t.y += part[w][c][p][lane].y;
        }
        acc.v[c][p] = t;
      }
    store_cell(pt, lane, Ng, acc, grids);
  }
}

// The other patches (order[n_heavy .. n_patches)): one warp each.
__global__ void __launch_bounds__(kPatchThreads) grid_apply_kernel(
    const int *__restrict__ offsets, const int *__restrict__ order, const int *__restrict__ w_off,
    const float *__restrict__ wts, const float4 *__restrict__ vals, int Ng, int W, int nbw,
    int slot0, int n_patches, int n_patch_c, float2 *__restrict__ grids) {
  __shared__ WarpStage stage[kPatchThreads / 32];
  const int slot = slot0 + blockIdx.x * (kPatchThreads / 32) + (threadIdx.x >> 5);
  if (slot >= n_patches) return;
  const int idx = __ldg(order + slot);
  const Patch pt = patch_at(idx, n_patch_c, W, nbw);
  const int lane = threadIdx.x & 31;
  const int first = __ldg(w_off + idx), count = __ldg(w_off + idx + 1) - first;
  Acc acc;
#pragma unroll
  for (int c = 0; c < kGroups; ++c)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc.v[c][p] = make_float2(0.f, 0.f);
  apply_range(pt, nbw, offsets, wts + (int64_t)first * kFactors, vals, 0, count, lane,
              stage[threadIdx.x >> 5], acc);
  store_cell(pt, lane, Ng, acc, grids);
}

}  // namespace
}  // namespace mwax

using namespace mwax;

struct mwax_grid_plan_s {
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_tiles = 0, n_chan = 0, n_tbl = 0, Ng = 0, W = 0, nbw = 0;
  int64_t n_pts = 0;
  int n_kept = 0, n_patches = 0, n_patch_c = 0, n_heavy = 0;
  int64_t n_entries = 0;     // stored factors (12 per patch candidate)
  int *offsets = nullptr;    // [n_bins + 1]
  GeomRec *rec = nullptr;    // [n_kept]
  int *slot = nullptr;       // [n_pts]: sorted position of each point id, or -1
  int *w_off = nullptr;      // [n_patches + 1]: first candidate of each patch
  int *order = nullptr;      // [n_patches]: patches by decreasing candidate count
  float *wts = nullptr;      // [n_entries]: [candidate][8 column | 4 row factors] per patch
  float4 *vals = nullptr;    // [n_kept][2], filled per call
};

namespace {

void free_grid_plan(mwax_grid_plan_s *p) {
  if (!p) return;
  for (void *q : {(void *)p->offsets, (void *)p->rec, (void *)p->slot, (void *)p->w_off,
                  (void *)p->order, (void *)p->wts, (void *)p->vals})
    if (q) cudaFree(q);
  delete p;
}

bool is_dev(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

mwax_status mwax_grid_plan(mwax_grid_plan_t *out, const double *tile_xy, int n_tiles, int n_chan,
                           double f0, double df, int Ng, double du, int W, double sigma,
                           cudaStream_t stream) {
  mwax::NvtxRange nvtx_("mwax_grid_plan");
  if (!out || !tile_xy) return MWAX_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_tiles < 2 || n_tiles > 4096 || n_chan < 1 || Ng < 8 || Ng > 16384 || Ng % 2 || W < 1 ||
      W > 31 || !(du > 0.0) || !(sigma > 0.0) || !(f0 > 0.0) || df < 0.0)
    return MWAX_ERR_INVALID_ARG;
  const int64_t n_tbl = (int64_t)n_tiles * (n_tiles - 1) / 2;
  const int64_t n_pts = n_tbl * n_chan * 2;
  const int64_t nbw = (int64_t)Ng + W - 1;
  const int64_t n_bins = nbw * nbw;
  if (n_pts > 0x7FFFFFFFll || n_bins + 1 > 0x7FFFFFFFll) return MWAX_ERR_INVALID_ARG;
  mwax_grid_plan_s *p = new mwax_grid_plan_s;
  p->stream = stream;
  cudaGetDevice(&p->device);
  p->n_tiles = n_tiles;
  p->n_chan = n_chan;
  p->n_tbl = (int)n_tbl;
  p->Ng = Ng;
  p->W = W;
  p->nbw = (int)nbw;
  p->n_pts = n_pts;
  // plan-time scratch
  double *d_xy = nullptr;
  int *bin = nullptr, *hi = nullptr, *count = nullptr, *fill = nullptr, *ids = nullptr,
      *totals = nullptr;
  const int n_scan = (int)(n_bins + 1);
  const int scan_blocks = (n_scan + kScanBlock - 1) / kScanBlock;
  cudaError_t e = cudaMalloc(&d_xy, sizeof(double) * 2 * n_tiles);
  if (e == cudaSuccess) e = cudaMalloc(&bin, sizeof(int) * n_pts);
  if (e == cudaSuccess) e = cudaMalloc(&hi, sizeof(int) * n_pts);
  if (e == cudaSuccess) e = cudaMalloc(&count, sizeof(int) * n_scan);
  if (e == cudaSuccess) e = cudaMalloc(&fill, sizeof(int) * n_bins);
  if (e == cudaSuccess) e = cudaMalloc(&totals, sizeof(int) * scan_blocks);
  if (e == cudaSuccess) e = cudaMalloc(&p->offsets, sizeof(int) * n_scan);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_xy, tile_xy, sizeof(double) * 2 * n_tiles, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int) * n_scan, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(fill, 0, sizeof(int) * n_bins, stream);
  GridGeom g{d_xy, n_tiles, n_chan, (int)n_tbl, Ng, W, f0, df, du, (int)nbw};
  const int T = 256;
  const unsigned nblk = (unsigned)((n_pts + T - 1) / T);
  if (e == cudaSuccess) {
    grid_points_kernel<<<nblk, T, 0, stream>>>(g, n_pts, bin, hi);
    grid_count_kernel<<<nblk, T, 0, stream>>>(bin, n_pts, count);
    scan_blocks_kernel<<<scan_blocks, kScanBlock, 0, stream>>>(count, n_scan, p->offsets, totals);
    scan_totals_kernel<<<1, kScanBlock, 0, stream>>>(totals, scan_blocks);
    scan_add_kernel<<<scan_blocks, kScanBlock, 0, stream>>>(p->offsets, n_scan, totals);
    e = cudaGetLastError();
  }
  // number of points that reach the grid, and the largest bin (for the record)
  int kept = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&kept, p->offsets + n_bins, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e == cudaSuccess) {
    p->n_kept = kept;
    e = cudaMalloc(&ids, sizeof(int) * std::max(kept, 1));
  }
  if (e == cudaSuccess) e = cudaMalloc(&p->rec, sizeof(GeomRec) * std::max(kept, 1));
  if (e == cudaSuccess) e = cudaMalloc(&p->vals, 2 * sizeof(float4) * std::max(kept, 1));
  if (e == cudaSuccess) {
    grid_fill_kernel<<<nblk, T, 0, stream>>>(bin, n_pts, p->offsets, fill, ids);
    grid_sort_bins_kernel<<<(unsigned)((n_bins + T - 1) / T), T, 0, stream>>>(p->offsets,
                                                                             (int)n_bins, ids);
    if (kept > 0)
      grid_records_kernel<<<(kept + T - 1) / T, T, 0, stream>>>(ids, kept, hi, bin, (int)nbw,
                                                                p->rec);
    e = cudaGetLastError();
  }
  // sorted position of every point id
  if (e == cudaSuccess) e = cudaMalloc(&p->slot, sizeof(int) * n_pts);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->slot, 0xFF, sizeof(int) * n_pts, stream);
  if (e == cudaSuccess && kept > 0) {
    grid_slot_kernel<<<(kept + T - 1) / T, T, 0, stream>>>(p->rec, kept, p->slot);
    e = cudaGetLastError();
  }
  // the weights: candidates per patch, their prefix sum, then [candidate][cell]
  // (a point is a candidate of at most this many patches; the int32 prefix
  // sum must hold the total)
  const int64_t per_point = (int64_t)((W + kPatchR - 1) / kPatchR + 1) * ((W + kPatchC - 1) / kPatchC + 1);
  if (e == cudaSuccess && (int64_t)kept * per_point > 0x7FFFFFFFll) {
    for (void *q : {(void *)d_xy, (void *)bin, (void *)hi, (void *)count, (void *)fill, (void *)ids,
                    (void *)totals})
      if (q) cudaFree(q);
    free_grid_plan(p);
    return MWAX_ERR_UNSUPPORTED;
  }
  const int npr = (Ng + kPatchR - 1) / kPatchR, npc = (Ng + kPatchC - 1) / kPatchC;
  const int n_patches = npr * npc;
  const int n_pscan = n_patches + 1;  // one extra zero: the last offset is the total
  const int pscan_blocks = (n_pscan + kScanBlock - 1) / kScanBlock;
  int *pcnt = nullptr, *ptot = nullptr;
  p->n_patches = n_patches;
  p->n_patch_c = npc;
  const double inv_2s2d = 1.0 / (2.0 * sigma * sigma);
  const unsigned pgrid = (unsigned)((n_patches + kPatchThreads / 32 - 1) / (kPatchThreads / 32));
  if (e == cudaSuccess) e = cudaMalloc(&pcnt, sizeof(int) * n_pscan);
  if (e == cudaSuccess) e = cudaMalloc(&ptot, sizeof(int) * pscan_blocks);
  if (e == cudaSuccess) e = cudaMalloc(&p->w_off, sizeof(int) * n_pscan);
  if (e == cudaSuccess) e = cudaMemsetAsync(pcnt, 0, sizeof(int) * n_pscan, stream);
  if (e == cudaSuccess) {
    grid_patch_count_kernel<<<pgrid, kPatchThreads, 0, stream>>>(p->offsets, n_patches, W,
                                                                   (int)nbw, npc, pcnt);
    scan_blocks_kernel<<<pscan_blocks, kScanBlock, 0, stream>>>(pcnt, n_pscan, p->w_off, ptot);
    scan_totals_kernel<<<1, kScanBlock, 0, stream>>>(ptot, pscan_blocks);
    scan_add_kernel<<<pscan_blocks, kScanBlock, 0, stream>>>(p->w_off, n_pscan, ptot);
    e = cudaGetLastError();
  }
  int total = 0;
  std::vector<int> hcnt(n_patches), horder(n_patches);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&total, p->w_off + n_patches, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hcnt.data(), pcnt, sizeof(int) * n_patches, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e == cudaSuccess) {
    // heaviest patches first (ties in patch order)
    for (int i = 0; i < n_patches; ++i) horder[i] = i;
    std::stable_sort(horder.begin(), horder.end(),
                     [&](int a, int b) { return hcnt[a] > hcnt[b]; });
    while (p->n_heavy < n_patches && hcnt[horder[p->n_heavy]] > kHeavy) ++p->n_heavy;
    e = cudaMalloc(&p->order, sizeof(int) * n_patches);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(p->order, horder.data(), sizeof(int) * n_patches, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    p->n_entries = (int64_t)total * kFactors;
    e = cudaMalloc(&p->wts, sizeof(float) * std::max<int64_t>(p->n_entries, 1));
  }
  if (e == cudaSuccess) {
    grid_patch_weights_kernel<<<pgrid, kPatchThreads, 0, stream>>>(
        g, p->rec, p->offsets, inv_2s2d, n_patches, npc, p->w_off, p->wts);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  for (void *q : {(void *)d_xy, (void *)bin, (void *)hi, (void *)count, (void *)fill,
                  (void *)ids, (void *)totals, (void *)pcnt, (void *)ptot})
    if (q) cudaFree(q);
  if (e != cudaSuccess) {
    free_grid_plan(p);
    return e == cudaErrorMemoryAllocation ? MWAX_ERR_OOM : MWAX_ERR_CUDA;
  }
  *out = p;
  return MWAX_OK;
}

int64_t mwax_grid_plan_points(mwax_grid_plan_t plan) { return plan ? plan->n_kept : -1; }

int64_t mwax_grid_plan_entries(mwax_grid_plan_t plan) { return plan ? plan->n_entries : -1; }

mwax_status mwax_grid(mwax_grid_plan_t plan, const int32_t *vis, float *grids) {
  mwax::NvtxRange nvtx_("mwax_grid");
  if (!plan || !is_dev(vis) || !is_dev(grids)) return MWAX_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(vis) & 7u) || (reinterpret_cast<uintptr_t>(grids) & 7u))
    return MWAX_ERR_INVALID_ARG;
  const int64_t N = 2 * (int64_t)plan->n_tiles;
  const int T = 256;
  if (plan->n_kept > 0)
    grid_values_kernel<<<(unsigned)((plan->n_pts + T - 1) / T), T, 0, plan->stream>>>(
        plan->slot, (int)plan->n_pts, plan->n_tbl, N * (N + 1) / 2,
        reinterpret_cast<const int2 *>(vis), plan->vals);
  float2 *g2 = reinterpret_cast<float2 *>(grids);
  if (plan->n_heavy > 0)
    grid_apply_heavy_kernel<<<plan->n_heavy, kPatchThreads, 0, plan->stream>>>(
        plan->offsets, plan->order, plan->w_off, plan->wts, plan->vals, plan->Ng, plan->W,
        plan->nbw, plan->n_patch_c, g2);
  const int n_light = plan->n_patches - plan->n_heavy;
  if (n_light > 0)
    grid_apply_kernel<<<(unsigned)((n_light + kPatchThreads / 32 - 1) / (kPatchThreads / 32)),
                        kPatchThreads, 0, plan->stream>>>(
        plan->offsets, plan->order, plan->w_off, plan->wts, plan->vals, plan->Ng, plan->W,
        plan->nbw, plan->n_heavy, plan->n_patches, plan->n_patch_c, g2);
  return cudaGetLastError() == cudaSuccess ? MWAX_OK : MWAX_ERR_CUDA;
}

mwax_status mwax_grid_destroy(mwax_grid_plan_t plan) {
  if (!plan) return MWAX_ERR_INVALID_ARG;
  cudaStreamSynchronize(plan->stream);
  free_grid_plan(plan);
  return MWAX_OK;
}

}  // extern "C"
