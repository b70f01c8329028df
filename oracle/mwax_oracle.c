/*
 * mwax_oracle.c -- plain, slow CPU oracle for the MWA X-engine correlator and
 * the gain-calibration loss that consumes its output.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
 * it is used by the tests, by the smoke check and by the benchmark's CPU
 * baseline leg.  It shares no code with the CUDA library (own sample
 * decoding, own index arithmetic, own loops).
 *
 * What it computes (paper Sec. 2: an FPGA correlator cross-correlates the
 * signals of all antennas -- 512 antennas, ~130,000 baseline pairs, 768
 * channels, 4 polarisation products -- and the stream is then integrated,
 * calibrated and imaged):
 *
 *   correlation, per channel c and input pair i >= j (lower triangle with
 *   autocorrelations), integrated over T time samples:
 *       V_ij = sum_t x_i(t) conj(x_j(t))
 *       Re V_ij = sum_t xr_i xr_j + xi_i xi_j
 *       Im V_ij = sum_t xi_i xr_j - xr_i xi_j
 *   with int64 accumulators, stored as int32 pairs at
 *   out[c][i(i+1)/2 + j][re, im].
 *
 *   calibration (Sec. 2: the complex gain of each antenna element is found
 *   by a least-squares fit against catalogue sources), in FP64:
 *       R_ij = g_i conj(g_j) M_ij - V_ij
 *       L(g) = sum_nu sum_{i>j} |R_ij,nu|^2          (w = 1 off-diagonal, 0 on autos)
 *       grad_k = 2 dL/d conj(g_k)
 *              = 2 sum_nu sum_{j != k} R_kj g_j conj(M_kj)
 *   where R and M are extended to the upper triangle by Hermitian symmetry
 *   (R_kj = conj(R_jk), M_kj = conj(M_jk)).  grad is the PyTorch convention
 *   for a real loss of a complex parameter: dL/dRe g + i dL/dIm g.
 *
 *   gain solve (Sec. 2: the gains come from an iterative least-squares fit
 *   in which every measurement constrains the gains): with every gain but
 *   g_k held fixed, L is a linear least-squares problem in g_k, minimised by
 *       h_k = num_k / den_k
 *       num_k = sum_nu sum_{j != k} V_kj g_j conj(M_kj)
 *       den_k = sum_nu sum_{j != k} |g_j|^2 |M_kj|^2
 *   (V_kj, M_kj extended by Hermitian symmetry; h_k = g_k when den_k = 0).
 *   oracle_calib_als_target computes h for all k from one g; the iteration
 *   that uses it lives in the Python wrapper.
 *
 * Sample format (the correlator input): voltages[chan][time][input];
 *   4+4-bit: one byte, low nibble = re, high nibble = im, two's complement;
 *   8+8-bit: two bytes, re then im, int8.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ---- sample decoding ---------------------------------------------------- */

static int32_t nibble_to_int(uint32_t v) { return (v & 0x8u) ? (int32_t)v - 16 : (int32_t)v; }

/* Decode n packed complex samples into separate re / im arrays.
 * Returns 0, or 1 for an unsupported sample width. */
int oracle_decode(const uint8_t *raw, int sample_bits, int64_t n, int32_t *re, int32_t *im) {
  if (sample_bits == 4) {
    for (int64_t k = 0; k < n; ++k) {
      re[k] = nibble_to_int(raw[k] & 0xFu);
      im[k] = nibble_to_int((raw[k] >> 4) & 0xFu);
    }
    return 0;
  }
  if (sample_bits == 8) {
    for (int64_t k = 0; k < n; ++k) {
      re[k] = (int32_t)(int8_t)raw[2 * k];
      im[k] = (int32_t)(int8_t)raw[2 * k + 1];
    }
    return 0;
  }
  return 1;
}

/* ---- correlation -------------------------------------------------------- */

typedef struct {
  const int32_t *re, *im; /* decoded, [chan][input][time] */
  int n_inputs, n_chan, n_time;
  int32_t *out;   /* [chan][b][2] */
  int64_t *out64; /* optional [chan][b][2] int64 */
  int tid, n_threads;
  int overflow;
} corr_job;

static void *corr_worker(void *arg) {
  corr_job *j = (corr_job *)arg;
  const int64_t N = j->n_inputs, T = j->n_time;
  const int64_t B = N * (N + 1) / 2;
  /* one unit of work = one (channel, row i) */
  const int64_t units = (int64_t)j->n_chan * N;
  for (int64_t u = j->tid; u < units; u += j->n_threads) {
    const int64_t c = u / N, i = u % N;
    const int32_t *xr_i = j->re + (c * N + i) * T;
    const int32_t *xi_i = j->im + (c * N + i) * T;
    for (int64_t jj = 0; jj <= i; ++jj) {
      const int32_t *xr_j = j->re + (c * N + jj) * T;
      const int32_t *xi_j = j->im + (c * N + jj) * T;
      int64_t sre = 0, sim = 0;
      for (int64_t t = 0; t < T; ++t) {
        sre += (int64_t)xr_i[t] * xr_j[t] + (int64_t)xi_i[t] * xi_j[t];
        sim += (int64_t)xi_i[t] * xr_j[t] - (int64_t)xr_i[t] * xi_j[t];
      }
      const int64_t b = i * (i + 1) / 2 + jj;
      if (sre > INT32_MAX || sre < -(int64_t)INT32_MAX || sim > INT32_MAX ||
          sim < -(int64_t)INT32_MAX)
        j->overflow = 1;
      if (j->out) {
        j->out[(c * B + b) * 2] = (int32_t)sre;
        j->out[(c * B + b) * 2 + 1] = (int32_t)sim;
      }
      if (j->out64) {
        j->out64[(c * B + b) * 2] = sre;
        j->out64[(c * B + b) * 2 + 1] = sim;
      }
    }
  }
  return NULL;
}

/*
 * Correlate packed voltages[n_chan][n_time][n_inputs].
 * out   (may be NULL): int32 [n_chan][N(N+1)/2][2]
 * out64 (may be NULL): int64 [n_chan][N(N+1)/2][2]
 * Returns 0; 1 bad argument; 2 out of memory; 3 a visibility exceeds the
 * int32 range (the int64 values in out64 are still exact).
 */
int oracle_correlate(const uint8_t *volt, int sample_bits, int n_inputs, int n_chan, int n_time,
                     int32_t *out, int64_t *out64, int n_threads) {
  if (!volt || n_inputs < 0 || n_chan < 0 || n_time < 0) return 1;
  if (sample_bits != 4 && sample_bits != 8) return 1;
  const int64_t N = n_inputs, T = n_time, C = n_chan;
  const int64_t n = C * T * N;
  int32_t *re_ct = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  int32_t *im_ct = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  int32_t *re = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  int32_t *im = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  if (!re_ct || !im_ct || !re || !im) {
    free(re_ct); free(im_ct); free(re); free(im);
    return 2;
  }
  oracle_decode(volt, sample_bits, n, re_ct, im_ct);
  /* [chan][time][input] -> [chan][input][time] so each input's series is contiguous */
  for (int64_t c = 0; c < C; ++c)
    for (int64_t t = 0; t < T; ++t)
      for (int64_t i = 0; i < N; ++i) {
        re[(c * N + i) * T + t] = re_ct[(c * T + t) * N + i];
        im[(c * N + i) * T + t] = im_ct[(c * T + t) * N + i];
      }
  free(re_ct);
  free(im_ct);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  corr_job jobs[256];
  int rc = 0, started = 0;
  for (int k = 0; k < n_threads; ++k) {
    jobs[k] = (corr_job){re, im, n_inputs, n_chan, n_time, out, out64, k, n_threads, 0};
    if (pthread_create(&th[k], NULL, corr_worker, &jobs[k]) != 0) { rc = 2; break; }
    ++started;
  }
  for (int k = 0; k < started; ++k) {
    pthread_join(th[k], NULL);
    if (jobs[k].overflow) rc = rc ? rc : 3;
  }
  free(re);
  free(im);
  return rc;
}

/* ---- baseline triangle -------------------------------------------------- */

int64_t oracle_n_baselines(int64_t n_inputs) { return n_inputs * (n_inputs + 1) / 2; }

int64_t oracle_baseline_index(int64_t i, int64_t j) {
  if (j < 0 || i < j) return -1;
  return i * (i + 1) / 2 + j;
}

/* ---- calibration loss and gradient (FP64) ------------------------------- */

/* complex helpers on (re, im) pairs */
typedef struct { double re, im; } cplx;
static cplx cmul(cplx a, cplx b) { return (cplx){a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
static cplx cconj(cplx a) { return (cplx){a.re, -a.im}; }
static cplx csub(cplx a, cplx b) { return (cplx){a.re - b.re, a.im - b.im}; }
static cplx cld(const double *p) { return (cplx){p[0], p[1]}; }

/* R_ij for i > j at channel nu: g_i conj(g_j) M_ij - V_ij.  V, M: [chan][b][2]. */
static cplx resid(const double *V, const double *M, const double *g, int64_t B, int64_t nu,
                  int64_t i, int64_t j) {
  const int64_t b = i * (i + 1) / 2 + j;
  cplx gi = cld(g + 2 * i), gj = cld(g + 2 * j);
  cplx m = cld(M + (nu * B + b) * 2), v = cld(V + (nu * B + b) * 2);
  return csub(cmul(cmul(gi, cconj(gj)), m), v);
}

/* L(g) = sum_nu sum_{i>j} |R_ij,nu|^2.  Returns the loss. */
double oracle_calib_loss(const double *V, const double *M, const double *g, int n_inputs,
                         int n_chan) {
  const int64_t N = n_inputs, B = N * (N + 1) / 2;
  double L = 0.0;
  for (int64_t nu = 0; nu < n_chan; ++nu)
    for (int64_t i = 0; i < N; ++i)
      for (int64_t j = 0; j < i; ++j) {
        cplx r = resid(V, M, g, B, nu, i, j);
        L += r.re * r.re + r.im * r.im;
      }
  return L;
}

typedef struct {
  const double *V, *M, *g;
  int n_inputs, n_chan;
  double *grad;
  int tid, n_threads;
} grad_job;

static void *grad_worker(void *arg) {
  grad_job *q = (grad_job *)arg;
  const int64_t N = q->n_inputs, B = N * (N + 1) / 2;
  for (int64_t k = q->tid; k < N; k += q->n_threads) {
    cplx acc = {0.0, 0.0};
    for (int64_t nu = 0; nu < q->n_chan; ++nu)
      for (int64_t j = 0; j < N; ++j) {
        if (j == k) continue;
        cplx r_kj, m_kj;
        if (k > j) {
          r_kj = resid(q->V, q->M, q->g, B, nu, k, j);
          m_kj = cld(q->M + (nu * B + k * (k + 1) / 2 + j) * 2);
        } else {
          r_kj = cconj(resid(q->V, q->M, q->g, B, nu, j, k));
          m_kj = cconj(cld(q->M + (nu * B + j * (j + 1) / 2 + k) * 2));
        }
        cplx t = cmul(cmul(r_kj, cld(q->g + 2 * j)), cconj(m_kj));
        acc.re += t.re;
        acc.im += t.im;
      }
    q->grad[2 * k] = 2.0 * acc.re;
    q->grad[2 * k + 1] = 2.0 * acc.im;
  }
  return NULL;
}

/* grad[k] = 2 dL/d conj(g_k), [n_inputs][2].  Returns 0, or 2 on thread failure. */
int oracle_calib_grad(const double *V, const double *M, const double *g, int n_inputs, int n_chan,
                      double *grad, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  grad_job jobs[256];
  int started = 0, rc = 0;
  for (int k = 0; k < n_threads; ++k) {
    jobs[k] = (grad_job){V, M, g, n_inputs, n_chan, grad, k, n_threads};
    if (pthread_create(&th[k], NULL, grad_worker, &jobs[k]) != 0) { rc = 2; break; }
    ++started;
  }
  for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
  return rc;
}

/* ---- alternating least-squares gain target (FP64) ----------------------- */

typedef struct {
  const double *V, *M, *g;
  int n_inputs, n_chan;
  double *h;
  int tid, n_threads;
} als_job;

/* V_kj and M_kj for any k != j, from the stored lower triangle. */
static void pair_vm(const double *V, const double *M, int64_t B, int64_t nu, int64_t k, int64_t j,
                    cplx *v, cplx *m) {
  if (k > j) {
    const int64_t b = k * (k + 1) / 2 + j;
    *v = cld(V + (nu * B + b) * 2);
    *m = cld(M + (nu * B + b) * 2);
  } else {
    const int64_t b = j * (j + 1) / 2 + k;
    *v = cconj(cld(V + (nu * B + b) * 2));
    *m = cconj(cld(M + (nu * B + b) * 2));
  }
}

static void *als_worker(void *arg) {
  als_job *q = (als_job *)arg;
  const int64_t N = q->n_inputs, B = N * (N + 1) / 2;
  for (int64_t k = q->tid; k < N; k += q->n_threads) {
    cplx num = {0.0, 0.0};
    double den = 0.0;
    for (int64_t nu = 0; nu < q->n_chan; ++nu)
      for (int64_t j = 0; j < N; ++j) {
        if (j == k) continue;
        cplx v, m;
        pair_vm(q->V, q->M, B, nu, k, j, &v, &m);
        const cplx gj = cld(q->g + 2 * j);
        const cplx t = cmul(cmul(v, gj), cconj(m));
        num.re += t.re;
        num.im += t.im;
        den += (gj.re * gj.re + gj.im * gj.im) * (m.re * m.re + m.im * m.im);
      }
    if (den > 0.0) {
      q->h[2 * k] = num.re / den;
      q->h[2 * k + 1] = num.im / den;
    } else {
      q->h[2 * k] = q->g[2 * k];
      q->h[2 * k + 1] = q->g[2 * k + 1];
    }
  }
  return NULL;
}

/* h[k] = argmin over g_k of L with the other gains fixed at g, [n_inputs][2].
 * Returns 0, or 2 on thread failure. */
int oracle_calib_als_target(const double *V, const double *M, const double *g, int n_inputs,
                            int n_chan, double *h, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  als_job jobs[256];
  int started = 0, rc = 0;
  for (int k = 0; k < n_threads; ++k) {
    jobs[k] = (als_job){V, M, g, n_inputs, n_chan, h, k, n_threads};
    if (pthread_create(&th[k], NULL, als_worker, &jobs[k]) != 0) { rc = 2; break; }
    ++started;
  }
  for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
  return rc;
}

/* ---- gridding (FP64) ------------------------------------------------------
 * Paper Sec. 2.1: the calibrated visibilities are convolved onto a regular
 * grid so that an FFT can form the images.  Definition used here:
 *   tiles a at (X_a, Y_a) metres; every tile baseline a > b and channel c
 *   (frequency nu_c = f0 + c df) is a point at
 *       u = (X_a - X_b) nu_c / c_light,  v = (Y_a - Y_b) nu_c / c_light
 *   in wavelengths, i.e. at continuous cell coordinates
 *       x = u / du + Ng / 2,  y = v / du + Ng / 2.
 *   Polarisation product (p, q) (0 = X, 1 = Y) of that baseline is the
 *   correlator output V[c][i(i+1)/2 + j] with i = 2a + p, j = 2b + q.  It is
 *   added to grid G_pq at every cell (r, s) with |s - x| < W/2 and
 *   |r - y| < W/2 with weight exp(-((s - x)^2 + (r - y)^2) / (2 sigma^2)).
 *   The reversed baseline (b, a) is the point (-u, -v) carrying
 *   conj(V of product (q, p) of (a, b)), gridded the same way.  Cells outside
 *   [0, Ng) are dropped.  Grids out[pol = 2p + q][r][s][re, im].
 */
static const double kCLight = 299792458.0;

typedef struct {
  const double *tile_xy;
  int n_tiles, n_chan;
  double f0, df, du, sigma;
  int Ng, W;
  const int32_t *vis;
} grid_geom;

static cplx vis_pol(const grid_geom *G, int64_t c, int64_t a, int64_t b, int p, int q) {
  const int64_t N = 2 * (int64_t)G->n_tiles, B = N * (N + 1) / 2;
  const int64_t i = 2 * a + p, j = 2 * b + q;
  const int32_t *v = G->vis + (c * B + i * (i + 1) / 2 + j) * 2;
  return (cplx){(double)v[0], (double)v[1]};
}

/* add point (x, y) carrying V[4] (indexed 2p + q) to the grids */
static void grid_point(const grid_geom *G, double x, double y, const cplx *V, double *out) {
  const int Ng = G->Ng;
  const double half = 0.5 * G->W, s2 = 2.0 * G->sigma * G->sigma;
  for (int r = (int)floor(y - half); r <= (int)ceil(y + half); ++r) {
    if (r < 0 || r >= Ng || !(fabs(r - y) < half)) continue;
    for (int s = (int)floor(x - half); s <= (int)ceil(x + half); ++s) {
      if (s < 0 || s >= Ng || !(fabs(s - x) < half)) continue;
      const double w = exp(-((s - x) * (s - x) + (r - y) * (r - y)) / s2);
      for (int pol = 0; pol < 4; ++pol) {
        double *o = out + (((int64_t)pol * Ng + r) * Ng + s) * 2;
        o[0] += w * V[pol].re;
        o[1] += w * V[pol].im;
      }
    }
  }
}

static void point_xy(const grid_geom *G, int64_t a, int64_t b, int64_t c, double *x, double *y) {
  const double nu = G->f0 + (double)c * G->df;
  const double u = (G->tile_xy[2 * a] - G->tile_xy[2 * b]) * nu / kCLight;
  const double v = (G->tile_xy[2 * a + 1] - G->tile_xy[2 * b + 1]) * nu / kCLight;
  *x = u / G->du + 0.5 * G->Ng;
  *y = v / G->du + 0.5 * G->Ng;
}

/* All four polarisation grids, out [4][Ng][Ng][2] (zeroed here).  vis:
 * [n_chan][N(N+1)/2][2] int32 with N = 2 n_tiles.  Returns 0. */
int oracle_grid(const double *tile_xy, int n_tiles, int n_chan, double f0, double df, int Ng,
                double du, int W, double sigma, const int32_t *vis, double *out) {
  grid_geom G = {tile_xy, n_tiles, n_chan, f0, df, du, sigma, Ng, W, vis};
  memset(out, 0, sizeof(double) * 2 * 4 * (size_t)Ng * Ng);
  for (int64_t c = 0; c < n_chan; ++c)
    for (int64_t a = 0; a < n_tiles; ++a)
      for (int64_t b = 0; b < a; ++b) {
        double x, y;
        point_xy(&G, a, b, c, &x, &y);
        cplx V[4], Vc[4];
        for (int p = 0; p < 2; ++p)
          for (int q = 0; q < 2; ++q) {
            V[2 * p + q] = vis_pol(&G, c, a, b, p, q);
            Vc[2 * p + q] = cconj(vis_pol(&G, c, a, b, q, p));  /* reversed baseline */
          }
        grid_point(&G, x, y, V, out);
        grid_point(&G, (double)Ng - x, (double)Ng - y, Vc, out);
      }
  return 0;
}

/* One cell (r, s) of grid `pol`, from every point directly: val[re, im]. */
int oracle_grid_cell(const double *tile_xy, int n_tiles, int n_chan, double f0, double df, int Ng,
                     double du, int W, double sigma, const int32_t *vis, int pol, int r, int s,
                     double *val) {
  grid_geom G = {tile_xy, n_tiles, n_chan, f0, df, du, sigma, Ng, W, vis};
  const int p = pol >> 1, q = pol & 1;
  const double half = 0.5 * W, s2 = 2.0 * sigma * sigma;
  double re = 0.0, im = 0.0;
  for (int64_t c = 0; c < n_chan; ++c)
    for (int64_t a = 0; a < n_tiles; ++a)
      for (int64_t b = 0; b < a; ++b) {
        double x, y;
        point_xy(&G, a, b, c, &x, &y);
        for (int side = 0; side < 2; ++side) {
          const double px = side ? (double)Ng - x : x, py = side ? (double)Ng - y : y;
          if (!(fabs(s - px) < half) || !(fabs(r - py) < half)) continue;
          const double w = exp(-((s - px) * (s - px) + (r - py) * (r - py)) / s2);
          const cplx v = side ? cconj(vis_pol(&G, c, a, b, q, p)) : vis_pol(&G, c, a, b, p, q);
          re += w * v.re;
          im += w * v.im;
        }
      }
  val[0] = re;
  val[1] = im;
  return 0;
}
