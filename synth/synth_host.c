/*
 * synth_host.c -- host-side fill of synthetic voltages (inputs only).
 *
 * Regenerates any subset of channels bit-identically to the device fill in
 * synth_cuda.cu; both call synth_sample() from synth.h.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

#include "synth.h"

typedef struct {
  const synth_params *p;
  const int64_t *chans;
  int64_t n_chans, t0, n_time;
  uint8_t *out;
  int tid, n_threads;
} fill_job;

static void *fill_worker(void *arg) {
  fill_job *j = (fill_job *)arg;
  const synth_params *p = j->p;
  const int bps = synth_bytes_per_sample(p->sample_bits);
  const int64_t n_in = p->n_inputs;
  const int64_t rows = j->n_chans * j->n_time;
  for (int64_t r = j->tid; r < rows; r += j->n_threads) {
    int64_t ci = r / j->n_time, t = j->t0 + r % j->n_time;
    uint8_t *dst = j->out + r * n_in * bps;
    for (int64_t i = 0; i < n_in; ++i) {
      int32_t re, im;
      synth_sample(p, j->chans[ci], t, i, &re, &im);
      synth_pack(p->sample_bits, re, im, dst + i * bps);
    }
  }
  return NULL;
}

/* Fill out[n_chans][n_time][n_inputs] (packed) for channels chans[] and time
 * samples t0 .. t0+n_time-1.  Returns 0 on success. */
int synth_fill_host(const synth_params *p, const int64_t *chans, int64_t n_chans, int64_t t0,
                    int64_t n_time, uint8_t *out, int n_threads) {
  if (!p || !chans || !out || n_chans < 0 || n_time < 0) return 1;
  if (p->sample_bits != 4 && p->sample_bits != 8) return 1;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  fill_job jobs[256];
  for (int k = 0; k < n_threads; ++k) {
    jobs[k] = (fill_job){p, chans, n_chans, t0, n_time, out, k, n_threads};
    if (pthread_create(&th[k], NULL, fill_worker, &jobs[k]) != 0) {
      for (int q = 0; q < k; ++q) pthread_join(th[q], NULL);
      return 2;
    }
  }
  for (int k = 0; k < n_threads; ++k) pthread_join(th[k], NULL);
  return 0;
}

/* One Philox4x64-10 block, exported for the known-answer test. */
void synth_philox_host(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  synth_philox4x64_10(ctr, key, out);
}

/* Unpacked sample values, exported for statistics tests. */
void synth_sample_host(const synth_params *p, int64_t chan, int64_t t, int64_t input,
                       int32_t *re, int32_t *im) {
  synth_sample(p, chan, t, input, re, im);
}
