/*
 * synth.h -- seeded synthetic channelised voltages (inputs only).
 *
 * This header is the one piece of code shared by the CPU oracle side and
 * the CUDA side: it produces the *inputs* of the correlator (packed complex
 * voltage samples) and nothing else.  It contains none of the correlation,
 * integration or calibration arithmetic.
 *
 * Randomness: Philox4x64-10, the counter-based generator of Salmon, Moraes,
 * Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11),
 * written here from that definition (two 64x64->128 multiplies per round,
 * Weyl key schedule, 10 rounds).  It is pinned against numpy.random.Philox.
 *
 * Everything below is integer arithmetic so that gcc on the host and nvcc on
 * the device give bit-identical samples.  Gaussian values are Irwin-Hall
 * sums of twelve 16-bit uniforms (mean 0, variance ~1, in Q16 fixed point).
 * Sinusoids use a Q16 cosine table supplied by the caller (computed once in
 * Python and handed to both sides), indexed by the top 12 bits of a uint32
 * phase.
 *
 * Sample packing (the correlator input format):
 *   4+4-bit: one byte per complex sample, low nibble = re, high nibble = im,
 *            two's complement, values in [-7, 7].
 *   8+8-bit: two bytes per complex sample, byte 0 = re, byte 1 = im, int8,
 *            values in [-127, 127].
 *   Layout: voltages[chan][time][input].
 */
#ifndef MWAX_SYNTH_H
#define MWAX_SYNTH_H

#include <stdint.h>

#if defined(__CUDACC__)
#define SYNTH_FN __host__ __device__ __forceinline__
#else
#define SYNTH_FN static inline
#endif

#define SYNTH_TABLE_BITS 12
#define SYNTH_TABLE_SIZE (1 << SYNTH_TABLE_BITS)
#define SYNTH_MAX_SRC 32

/* Synthesis kinds. */
enum {
  SYNTH_NOISE_TONE = 0, /* Gaussian noise (sigma) + optional common tone      */
  SYNTH_SOURCES = 1,    /* noise + point sources with per-input phase        */
  SYNTH_CONST = 2,      /* every sample = (c_re, c_im)                        */
  SYNTH_BIGSMALL = 3,   /* (max,max) for t < t_split, then random +-1 signs   */
  SYNTH_RANDMAX = 4,    /* each component uniformly +-max                     */
  SYNTH_QUARTER = 5,    /* x_i(t) = c_i * i^t, c_i from the per-input table   */
};

/* Plain-old-data parameter block.  Tables are referenced by pointer so that
 * the host copy points at host arrays and the device copy at device arrays. */
typedef struct {
  uint64_t seed;
  int32_t kind;
  int32_t sample_bits; /* 4 or 8 */
  int32_t n_inputs;
  int32_t n_time;
  int32_t sigma;        /* noise standard deviation, sample units (integer) */
  int32_t tone_amp_q16; /* common tone amplitude, Q16 sample units          */
  int32_t n_src;        /* SYNTH_SOURCES: number of sources                 */
  int32_t chan_base;    /* added to the channel index in phase formulas     */
  int32_t c_re, c_im;   /* SYNTH_CONST                                      */
  int32_t t_split;      /* SYNTH_BIGSMALL                                   */
  int32_t pad_;
  const int32_t *cos_q16;     /* [SYNTH_TABLE_SIZE] round(65536 cos(2 pi k/4096)) */
  const int32_t *src_amp_q16; /* [n_src] source amplitude, Q16 sample units       */
  const uint32_t *src_rate;   /* [n_inputs][n_src] phase per channel, uint32 turns */
  const int32_t *ci;          /* SYNTH_QUARTER: [n_inputs][2] Gaussian integers    */
  const int32_t *gain_q16;    /* SYNTH_SOURCES: [n_inputs][2] complex gain on the
                                 source sum, Q16; NULL means unit gain           */
} synth_params;

/* ---- Philox4x64-10 ------------------------------------------------------ */

SYNTH_FN void synth_mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
#if defined(__CUDA_ARCH__)
  *lo = a * b;
  *hi = __umul64hi(a, b);
#else
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *lo = (uint64_t)p;
  *hi = (uint64_t)(p >> 64);
#endif
}

/* One Philox4x64-10 block: ctr[4], key[2] -> out[4]. */
SYNTH_FN void synth_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2],
                                  uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0, lo0, hi1, lo1;
    synth_mulhilo64(M0, c0, &hi0, &lo0);
    synth_mulhilo64(M1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Random block addressed by (a, b, c, stream) under (seed, domain). */
SYNTH_FN void synth_block(uint64_t seed, uint64_t domain, uint64_t a, uint64_t b, uint64_t c,
                          uint64_t stream, uint64_t out[4]) {
  uint64_t ctr[4] = {a, b, c, stream};
  uint64_t key[2] = {seed, domain};
  synth_philox4x64_10(ctr, key, out);
}

/* Irwin-Hall-12 Gaussian in Q16: sum of twelve 16-bit uniforms taken from
 * the 64-bit words w[0..2] (4 lanes each), minus the exact mean 393210. */
SYNTH_FN int32_t synth_ih12_q16(const uint64_t w[3]) {
  int32_t s = 0;
  for (int q = 0; q < 3; ++q)
    for (int l = 0; l < 4; ++l) s += (int32_t)((w[q] >> (16 * l)) & 0xFFFFu);
  return s - 393210;
}

/* Complex Gaussian (Q16, unit variance per component) for one address. */
SYNTH_FN void synth_cgauss_q16(uint64_t seed, uint64_t domain, uint64_t a, uint64_t b, uint64_t c,
                               int32_t *re, int32_t *im) {
  uint64_t r0[4], r1[4];
  synth_block(seed, domain, a, b, c, 0, r0);
  synth_block(seed, domain, a, b, c, 1, r1);
  uint64_t wr[3] = {r0[0], r0[1], r0[2]};
  uint64_t wi[3] = {r0[3], r1[0], r1[1]};
  *re = synth_ih12_q16(wr);
  *im = synth_ih12_q16(wi);
}

/* Arithmetic shift right with round-half-away-from-zero (x / 2^s). */
SYNTH_FN int64_t synth_rshift_rha(int64_t x, int s) {
  int64_t h = (int64_t)1 << (s - 1);
  return x >= 0 ? ((x + h) >> s) : -((-x + h) >> s);
}

SYNTH_FN int32_t synth_clip(int64_t v, int32_t m) {
  return (int32_t)(v > m ? m : (v < -m ? -m : v));
}

SYNTH_FN int32_t synth_cos_q16(const int32_t *tab, uint32_t phase) {
  return tab[phase >> (32 - SYNTH_TABLE_BITS)];
}
SYNTH_FN int32_t synth_sin_q16(const int32_t *tab, uint32_t phase) {
  /* sin(x) = cos(x - pi/2) */
  return tab[(phase - 0x40000000u) >> (32 - SYNTH_TABLE_BITS)];
}

/* Domains (second key word) separate the independent random streams. */
#define SYNTH_DOM_NOISE 0x6e6f697365ULL
#define SYNTH_DOM_TONE 0x746f6e65ULL
#define SYNTH_DOM_SRC 0x737263ULL
#define SYNTH_DOM_SIGN 0x7369676eULL

/* The complex sample (re, im) for (chan, t, input), already clipped to the
 * symmetric range [-max, max] of the sample width. */
SYNTH_FN void synth_sample(const synth_params *p, int64_t chan, int64_t t, int64_t input,
                           int32_t *out_re, int32_t *out_im) {
  const int32_t vmax = p->sample_bits == 4 ? 7 : 127;
  const uint64_t seed = p->seed;
  if (p->kind == SYNTH_CONST) {
    *out_re = synth_clip(p->c_re, vmax);
    *out_im = synth_clip(p->c_im, vmax);
    return;
  }
  if (p->kind == SYNTH_BIGSMALL || p->kind == SYNTH_RANDMAX) {
    if (p->kind == SYNTH_BIGSMALL && t < p->t_split) {
      *out_re = vmax;
      *out_im = vmax;
      return;
    }
    uint64_t r[4];
    synth_block(seed, SYNTH_DOM_SIGN, (uint64_t)chan, (uint64_t)t, (uint64_t)input, 0, r);
    int32_t mag = p->kind == SYNTH_BIGSMALL ? 1 : vmax;
    *out_re = (r[0] & 1) ? -mag : mag;
    *out_im = (r[1] & 1) ? -mag : mag;
    return;
  }
  if (p->kind == SYNTH_QUARTER) {
    int32_t cr = p->ci[2 * input], cim = p->ci[2 * input + 1];
    /* multiply by i^t: (a + ib) * i = -b + ia */
    switch ((int)(t & 3)) {
      case 0: *out_re = cr; *out_im = cim; break;
      case 1: *out_re = -cim; *out_im = cr; break;
      case 2: *out_re = -cr; *out_im = -cim; break;
      default: *out_re = cim; *out_im = -cr; break;
    }
    return;
  }
  /* Gaussian noise, Q16 sample units. */
  int32_t zr, zi;
  synth_cgauss_q16(seed, SYNTH_DOM_NOISE, (uint64_t)chan, (uint64_t)t, (uint64_t)input, &zr, &zi);
  int64_t vr = (int64_t)p->sigma * zr;
  int64_t vi = (int64_t)p->sigma * zi;
  if (p->tone_amp_q16 != 0) {
    /* common complex tone: per-channel start phase and rate, same for all inputs */
    uint64_t r[4];
    synth_block(seed, SYNTH_DOM_TONE, (uint64_t)chan, 0, 0, 0, r);
    uint32_t ph = (uint32_t)r[0] + (uint32_t)r[1] * (uint32_t)t;
    int64_t a = p->tone_amp_q16;
    vr += synth_rshift_rha(a * synth_cos_q16(p->cos_q16, ph), 16);
    vi += synth_rshift_rha(a * synth_sin_q16(p->cos_q16, ph), 16);
  }
  if (p->kind == SYNTH_SOURCES) {
    int64_t sr = 0, si = 0; /* source sum, Q16 */
    for (int s = 0; s < p->n_src; ++s) {
      int32_t nr, ni;
      synth_cgauss_q16(seed, SYNTH_DOM_SRC, (uint64_t)chan, (uint64_t)t, (uint64_t)s, &nr, &ni);
      uint32_t ph = p->src_rate[input * p->n_src + s] * (uint32_t)(chan + p->chan_base);
      int64_t c = synth_cos_q16(p->cos_q16, ph), sn = synth_sin_q16(p->cos_q16, ph);
      /* (nr + i ni)(c + i sn), Q16 * Q16 -> Q16 */
      int64_t rr = synth_rshift_rha((int64_t)nr * c - (int64_t)ni * sn, 16);
      int64_t ri = synth_rshift_rha((int64_t)nr * sn + (int64_t)ni * c, 16);
      int64_t a = p->src_amp_q16[s];
      sr += synth_rshift_rha(a * rr, 16);
      si += synth_rshift_rha(a * ri, 16);
    }
    if (p->gain_q16) {
      int64_t gr = p->gain_q16[2 * input], gi = p->gain_q16[2 * input + 1];
      int64_t tr = synth_rshift_rha(gr * sr - gi * si, 16);
      int64_t ti = synth_rshift_rha(gr * si + gi * sr, 16);
      sr = tr;
      si = ti;
    }
    vr += sr;
    vi += si;
  }
  *out_re = synth_clip(synth_rshift_rha(vr, 16), vmax);
  *out_im = synth_clip(synth_rshift_rha(vi, 16), vmax);
}

/* Bytes per complex sample. */
SYNTH_FN int synth_bytes_per_sample(int sample_bits) { return sample_bits == 4 ? 1 : 2; }

/* Pack one sample into dst (1 or 2 bytes). */
SYNTH_FN void synth_pack(int sample_bits, int32_t re, int32_t im, uint8_t *dst) {
  if (sample_bits == 4) {
    dst[0] = (uint8_t)(((uint32_t)re & 0xFu) | (((uint32_t)im & 0xFu) << 4));
  } else {
    dst[0] = (uint8_t)(int8_t)re;
    dst[1] = (uint8_t)(int8_t)im;
  }
}

#endif /* MWAX_SYNTH_H */
