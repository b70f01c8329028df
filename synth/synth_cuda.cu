/*
 * synth_cuda.cu -- device-side fill of synthetic voltages (inputs only).
 *
 * Same samples as synth_host.c, bit for bit: both call synth_sample() from
 * synth.h.  Used to place multi-GB inputs directly in HBM.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "synth.h"

__global__ void synth_fill_kernel(synth_params p, int64_t chan0, int64_t n_chan, uint8_t *out) {
  const int bps = synth_bytes_per_sample(p.sample_bits);
  const int64_t n_in = p.n_inputs;
  const int64_t total = n_chan * (int64_t)p.n_time * n_in;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = k % n_in;
    int64_t rest = k / n_in;
    int64_t t = rest % p.n_time;
    int64_t c = rest / p.n_time;
    int32_t re, im;
    synth_sample(&p, chan0 + c, t, i, &re, &im);
    synth_pack(p.sample_bits, re, im, out + k * bps);
  }
}

/* Fill out[n_chan][n_time][n_inputs] for channels chan0 .. chan0+n_chan-1.
 * The table pointers inside *p must be device pointers.  Asynchronous on
 * `stream`; returns a cudaError_t value. */
extern "C" int synth_fill_device(const synth_params *p, int64_t chan0, int64_t n_chan, uint8_t *out,
                                 void *stream) {
  if (!p || !out || n_chan < 0) return (int)cudaErrorInvalidValue;
  if (p->sample_bits != 4 && p->sample_bits != 8) return (int)cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256;
  int blocks = sms > 0 ? sms * 8 : 1024;
  synth_fill_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(*p, chan0, n_chan, out);
  return (int)cudaGetLastError();
}
