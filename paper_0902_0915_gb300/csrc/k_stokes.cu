// k_stokes.cu -- per-pixel Stokes conversion of instrumental-polarisation images.
//
// Paper Sec. 2.1: the instrumental polarisation images are converted into
// Stokes I, Q, U, V by a 4x4 matrix that depends on time and on the position
// on the sky and is computed by the real-time system for every pixel.  The
// paper gives no beam model; this uses the ideal crossed-dipole response:
// pixel (r, c) of an n x n slant-orthographic image has direction cosines
// l = (c - n/2) dl, m = (r - n/2) dl, rho = sqrt(l^2 + m^2); above the horizon
// (rho < 1), cos(theta) = sqrt(1 - rho^2) and phi = atan2(m, l) + chi (chi:
// the parallactic rotation at the time), and
//     J = [[cos(theta) cos(phi), -sin(phi)], [cos(theta) sin(phi), cos(phi)]],
//     J^-1 = (1 / cos(theta)) [[cos(phi), sin(phi)], [-cos(theta) sin(phi), cos(theta) cos(phi)]].
// The sky brightness is B = J^-1 C J^-T (J is real) for the instrumental
// coherency C = [[XX, XY], [YX, YY]], i.e. vec(B) = (J^-1 (x) J^-1) vec(C),
// and (I, Q, U, V) = (B00 + B11, B00 - B11, B01 + B10, -i (B01 - B10)):
// one 4x4 matrix per pixel, built here explicitly and applied to the four
// instrumental values.  Pixels with rho >= 1 are zero.
//
// HBM-bound: 4 complex values read and 4 written per pixel (64 B), each of
// the 8 planes accessed contiguously across a warp.
#include "mwax_internal.h"

namespace mwax {
namespace {

__global__ void __launch_bounds__(256) stokes_kernel(const float2 *__restrict__ inst, int n,
                                                     float dl, float cchi, float schi,
                                                     float2 *__restrict__ out) {
  const int64_t npix = (int64_t)n * n;
  const int64_t pix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  const int r = (int)(pix / n), c = (int)(pix % n);
  const float l = (float)(c - n / 2) * dl, m = (float)(r - n / 2) * dl;
  const float rho2 = l * l + m * m;
  float2 S[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                 make_float2(0.f, 0.f)};
  if (rho2 < 1.f) {
    const float ct = sqrtf(1.f - rho2);
    const float rho = sqrtf(rho2);
    // cos, sin of atan2(m, l) + chi (phi = chi at the centre pixel)
    float cp = cchi, sp = schi;
    if (rho > 0.f) {
      const float inv = 1.f / rho;
      cp = (l * cchi - m * schi) * inv;
      sp = (m * cchi + l * schi) * inv;
    }
    const float ic = 1.f / ct;
    const float a = cp * ic, b = sp * ic, cc = -sp, d = cp;  // J^-1 = [[a, b], [cc, d]]
    // rows of J^-1 (x) J^-1 over vec(C) = (XX, XY, YX, YY)
    const float k00[4] = {a * a, a * b, b * a, b * b};
    const float k01[4] = {a * cc, a * d, b * cc, b * d};
    const float k10[4] = {cc * a, cc * b, d * a, d * b};
    const float k11[4] = {cc * cc, cc * d, d * cc, d * d};
    float2 C[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) C[k] = inst[(int64_t)k * npix + pix];
    float2 B00 = make_float2(0.f, 0.f), B01 = B00, B10 = B00, B11 = B00;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      B00.x += k00[k] * C[k].x;
      B00.y += k00[k] * C[k].y;
      B01.x += k01[k] * C[k].x;
      B01.y += k01[k] * C[k].y;
      B10.x += k10[k] * C[k].x;
      B10.y += k10[k] * C[k].y;
      B11.x += k11[k] * C[k].x;
      B11.y += k11[k] * C[k].y;
    }
    S[0] = make_float2(B00.x + B11.x, B00.y + B11.y);
    S[1] = make_float2(B00.x - B11.x, B00.y - B11.y);
    S[2] = make_float2(B01.x + B10.x, B01.y + B10.y);
    // -i (B01 - B10)
    S[3] = make_float2(B01.y - B10.y, -(B01.x - B10.x));
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) out[(int64_t)k * npix + pix] = S[k];
}

bool dev_ptr8(const void *p) {
  if (!p || (reinterpret_cast<uintptr_t>(p) & 7u)) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace mwax

extern "C" mwax_status mwax_stokes(const float *inst, int n, double dl, double chi, float *stokes,
                                   cudaStream_t stream) {
  using namespace mwax;
  NvtxRange nvtx_("mwax_stokes");
  if (n < 2 || n % 2 || n > 65536 || !(dl > 0.0)) return MWAX_ERR_INVALID_ARG;
  if (!dev_ptr8(inst) || !dev_ptr8(stokes)) return MWAX_ERR_INVALID_ARG;
  const int64_t npix = (int64_t)n * n;
  // each thread reads its pixel's four inputs and writes its four outputs,
  // so any overlap of the two ranges lets one pixel's writes clobber the
  // inputs of another: reject it
  const uintptr_t bytes = (uintptr_t)(4 * npix) * sizeof(float2);
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(inst), b0 = reinterpret_cast<uintptr_t>(stokes);
  if (a0 < b0 + bytes && b0 < a0 + bytes) return MWAX_ERR_INVALID_ARG;
  const int T = 256;
  stokes_kernel<<<(unsigned)((npix + T - 1) / T), T, 0, stream>>>(
      reinterpret_cast<const float2 *>(inst), n, (float)dl, (float)cos(chi), (float)sin(chi),
      reinterpret_cast<float2 *>(stokes));
  return cudaGetLastError() == cudaSuccess ? MWAX_OK : MWAX_ERR_CUDA;
}
