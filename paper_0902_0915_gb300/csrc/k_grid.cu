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
//   3. per sorted point: float offset of the position from the first
//      support cell, last support cell (r_hi, s_hi), point id.
// Grid call (per integration): a gather kernel reads each point's four
// polarisation values from the int32 correlator output into the sorted
// record; then every warp gathers a 4 x 8 patch of cells: it streams the
// points whose support can reach the patch (per bin row, one contiguous range
// of the sorted points) with broadcast loads, and each lane keeps the points
// whose support contains its cell, in a fixed order.  Deterministic.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "mwax_internal.h"

namespace mwax {
namespace {

constexpr double kCLight = 299792458.0;
constexpr int kScanBlock = 1024;

// Positions are kept as offsets from the first support cell (x - s_lo,
// y - r_lo, in [W/2 - 1, W/2]): a float holds those to ~1e-7 cells, where the
// absolute coordinate (up to Ng) would lose ~1e-4.
struct GeomRec {  // sorted point, geometry part (20 B)
  float fx, fy;  // x - s_lo, y - r_lo
  int hi;        // r_hi << 16 | s_hi (both in [0, Ng))
  int id;        // point id: ((c * n_tbl) + tbl) * 2 + side
  int slo;       // s_lo + W - 1
};

struct __align__(16) PointRec {  // sorted point with its values (48 B)
  float fx, fy;
  int hi;
  int slo;  // s_lo + W - 1 (the bin column, >= 0)
  float2 v[4];
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
                                   float2 *__restrict__ xy, int *__restrict__ hi) {
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
  xy[k] = make_float2((float)(x - s_lo), (float)(y - r_lo));
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
                                    const float2 *__restrict__ xy, const int *__restrict__ hi,
                                    const int *__restrict__ bin, int nbw, GeomRec *__restrict__ rec) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_kept) return;
  const int k = ids[p];
  GeomRec r;
  r.fx = xy[k].x;
  r.fy = xy[k].y;
  r.hi = hi[k];
  r.id = k;
  r.slo = bin[k] % nbw;
  rec[p] = r;
}

// grid call, step 1: the four polarisation values of every sorted point
__global__ void grid_values_kernel(const GeomRec *__restrict__ rec, int n_kept, int n_tbl,
                                   int64_t n_bl, const int2 *__restrict__ vis,
                                   PointRec *__restrict__ pts) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_kept) return;
  const GeomRec g = rec[p];
  const int side = g.id & 1;
  const int ct = g.id >> 1;
  const int c = ct / n_tbl, tbl = ct % n_tbl;
  int a, b;
  tbl_pair(tbl, a, b);
  const int2 *vc = vis + (int64_t)c * n_bl;
  PointRec o;
  o.fx = g.fx;
  o.fy = g.fy;
  o.hi = g.hi;
  o.slo = g.slo;
#pragma unroll
  for (int pp = 0; pp < 2; ++pp)
#pragma unroll
    for (int qq = 0; qq < 2; ++qq) {
      // forward point: product (pp, qq) of (a, b); reversed: conj of (qq, pp)
      const int ip = side ? qq : pp, jq = side ? pp : qq;
      const int64_t i = 2 * a + ip, j = 2 * b + jq;
      const int2 v = vc[i * (i + 1) / 2 + j];
      o.v[2 * pp + qq] = make_float2((float)v.x, side ? -(float)v.y : (float)v.y);
    }
  pts[p] = o;
}

// grid call, step 2: gather.  A warp owns a 4 x 8 patch of cells (lane =
// row i = lane / 8, column j = lane % 8) and streams, once for the whole
// warp, every point whose support can reach the patch: for each bin row
// r0 - W + 1 .. r0 + 3 (shifted by W - 1), the bins of columns
// s0 - W + 1 .. s0 + 7, one contiguous range of the sorted points.  All lanes
// read the same point (a broadcast); each lane keeps it if its cell lies in
// the point's support.  A 7 x 7 support covers up to 28 of the 32 cells.
// Each cell's sum runs over bin rows, then bin columns, then point ids: a
// fixed order.
constexpr int kPatchR = 4, kPatchC = 8;
constexpr int kGatherWarpsR = 4, kGatherWarpsC = 2;  // CTA = 16 x 16 cells

__global__ void __launch_bounds__(32 * kGatherWarpsR * kGatherWarpsC) grid_gather_kernel(
    const PointRec *__restrict__ pts, const int *__restrict__ offsets, int Ng, int W, int nbw,
    float inv_2s2, float2 *__restrict__ grids) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = (blockIdx.y * kGatherWarpsR + warp / kGatherWarpsC) * kPatchR;
  const int s0 = (blockIdx.x * kGatherWarpsC + warp % kGatherWarpsC) * kPatchC;
  if (r0 >= Ng || s0 >= Ng) return;  // whole warp
  const int r = r0 + lane / kPatchC, s = s0 + lane % kPatchC;
  float2 acc[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) acc[p] = make_float2(0.f, 0.f);
  // bin row br holds points with r_lo = br - (W - 1); those reaching rows
  // r0 .. r0 + 3 have br in [r0, r0 + 3 + W - 1]; likewise bin columns
  const int br_end = min(r0 + kPatchR - 1 + W - 1, nbw - 1);
  const int bc_end = min(s0 + kPatchC + W - 1, nbw);  // exclusive
  for (int br = r0; br <= br_end; ++br) {
    const int lo = __ldg(offsets + br * nbw + s0), hi = __ldg(offsets + br * nbw + bc_end);
    const float dy0 = (float)(r - (br - (W - 1)));  // r - r_lo
    // four points per step: their geometry loads are issued together
    auto take = [&](const float4 g, int q) {
      const int phi = __float_as_int(g.z), slo = __float_as_int(g.w);
      const int ds = s - (slo - (W - 1));  // s - s_lo
      if (dy0 >= 0.f && ds >= 0 && r <= (phi >> 16) && s <= (phi & 0xFFFF)) {
        const float dx = (float)ds - g.x, dy = dy0 - g.y;
        const float w = expf(-(dx * dx + dy * dy) * inv_2s2);
        const float4 v01 = __ldg(reinterpret_cast<const float4 *>(pts + q) + 1);
        const float4 v23 = __ldg(reinterpret_cast<const float4 *>(pts + q) + 2);
        acc[0].x += w * v01.x;
        acc[0].y += w * v01.y;
        acc[1].x += w * v01.z;
        acc[1].y += w * v01.w;
        acc[2].x += w * v23.x;
        acc[2].y += w * v23.y;
        acc[3].x += w * v23.z;
        acc[3].y += w * v23.w;
      }
    };
    int q = lo;
    for (; q + 4 <= hi; q += 4) {
      float4 g[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) g[u] = __ldg(reinterpret_cast<const float4 *>(pts + q + u));
#pragma unroll
      for (int u = 0; u < 4; ++u) take(g[u], q + u);
    }
    for (; q < hi; ++q) take(__ldg(reinterpret_cast<const float4 *>(pts + q)), q);
  }
  if (r < Ng && s < Ng) {
    const int64_t cell = (int64_t)r * Ng + s;
#pragma unroll
    for (int p = 0; p < 4; ++p) grids[(int64_t)p * Ng * Ng + cell] = acc[p];
  }
}

}  // namespace
}  // namespace mwax

using namespace mwax;

struct mwax_grid_plan_s {
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_tiles = 0, n_chan = 0, n_tbl = 0, Ng = 0, W = 0, nbw = 0;
  float inv_2s2 = 0.f;
  int64_t n_pts = 0;
  int n_kept = 0, max_bin = 0;
  int *offsets = nullptr;   // [n_bins + 1]
  GeomRec *rec = nullptr;   // [n_kept]
  PointRec *pts = nullptr;  // [n_kept], filled per call
};

namespace {

void free_grid_plan(mwax_grid_plan_s *p) {
  if (!p) return;
  if (p->offsets) cudaFree(p->offsets);
  if (p->rec) cudaFree(p->rec);
  if (p->pts) cudaFree(p->pts);
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
  p->inv_2s2 = (float)(1.0 / (2.0 * sigma * sigma));
  p->n_pts = n_pts;
  // plan-time scratch
  double *d_xy = nullptr;
  int *bin = nullptr, *hi = nullptr, *count = nullptr, *fill = nullptr, *ids = nullptr,
      *totals = nullptr;
  float2 *xy = nullptr;
  const int n_scan = (int)(n_bins + 1);
  const int scan_blocks = (n_scan + kScanBlock - 1) / kScanBlock;
  cudaError_t e = cudaMalloc(&d_xy, sizeof(double) * 2 * n_tiles);
  if (e == cudaSuccess) e = cudaMalloc(&bin, sizeof(int) * n_pts);
  if (e == cudaSuccess) e = cudaMalloc(&hi, sizeof(int) * n_pts);
  if (e == cudaSuccess) e = cudaMalloc(&xy, sizeof(float2) * n_pts);
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
    grid_points_kernel<<<nblk, T, 0, stream>>>(g, n_pts, bin, xy, hi);
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
  if (e == cudaSuccess) e = cudaMalloc(&p->pts, sizeof(PointRec) * std::max(kept, 1));
  if (e == cudaSuccess) {
    grid_fill_kernel<<<nblk, T, 0, stream>>>(bin, n_pts, p->offsets, fill, ids);
    grid_sort_bins_kernel<<<(unsigned)((n_bins + T - 1) / T), T, 0, stream>>>(p->offsets,
                                                                             (int)n_bins, ids);
    if (kept > 0)
      grid_records_kernel<<<(kept + T - 1) / T, T, 0, stream>>>(ids, kept, xy, hi, bin, (int)nbw,
                                                                p->rec);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  for (void *q : {(void *)d_xy, (void *)bin, (void *)hi, (void *)xy, (void *)count, (void *)fill,
                  (void *)ids, (void *)totals})
    if (q) cudaFree(q);
  if (e != cudaSuccess) {
    free_grid_plan(p);
    return e == cudaErrorMemoryAllocation ? MWAX_ERR_OOM : MWAX_ERR_CUDA;
  }
  *out = p;
  return MWAX_OK;
}

int64_t mwax_grid_plan_points(mwax_grid_plan_t plan) { return plan ? plan->n_kept : -1; }

mwax_status mwax_grid(mwax_grid_plan_t plan, const int32_t *vis, float *grids) {
  mwax::NvtxRange nvtx_("mwax_grid");
  if (!plan || !is_dev(vis) || !is_dev(grids)) return MWAX_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(vis) & 7u) || (reinterpret_cast<uintptr_t>(grids) & 7u))
    return MWAX_ERR_INVALID_ARG;
  const int64_t N = 2 * (int64_t)plan->n_tiles;
  const int T = 256;
  if (plan->n_kept > 0)
    grid_values_kernel<<<(plan->n_kept + T - 1) / T, T, 0, plan->stream>>>(
        plan->rec, plan->n_kept, plan->n_tbl, N * (N + 1) / 2, reinterpret_cast<const int2 *>(vis),
        plan->pts);
  const int tile_r = kPatchR * kGatherWarpsR, tile_c = kPatchC * kGatherWarpsC;
  dim3 grd((plan->Ng + tile_c - 1) / tile_c, (plan->Ng + tile_r - 1) / tile_r);
  grid_gather_kernel<<<grd, 32 * kGatherWarpsR * kGatherWarpsC, 0, plan->stream>>>(plan->pts, plan->offsets, plan->Ng, plan->W,
                                                    plan->nbw, plan->inv_2s2,
                                                    reinterpret_cast<float2 *>(grids));
  return cudaGetLastError() == cudaSuccess ? MWAX_OK : MWAX_ERR_CUDA;
}

mwax_status mwax_grid_destroy(mwax_grid_plan_t plan) {
  if (!plan) return MWAX_ERR_INVALID_ARG;
  cudaStreamSynchronize(plan->stream);
  free_grid_plan(plan);
  return MWAX_OK;
}

}  // extern "C"
