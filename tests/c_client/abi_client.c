/* A plain C program against include/mwax.h and libmwax.so: no Python, no
 * torch.  It exercises the host-only entry points (no GPU needed) and, when a
 * GPU is present and a case file is given as argv[1], plans, correlates
 * (device buffers, then host buffers) and destroys a small job, comparing the
 * visibilities with the oracle's stored in the case file.  It prints one
 * "name value" line per check for the test that runs it. */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "mwax.h"

/* Case file: comment lines starting with '#', then "N C T bits", one line of
 * hex input bytes, then C lines of N(N+1) int32 values (re, im per baseline). */
static int device_case(const char *path) {
  FILE *f = fopen(path, "r");
  if (!f) {
    printf("case_file_missing 1\n");
    return 1;
  }
  char line[256];
  long pos = 0;
  int N = 0, C = 0, T = 0, bits = 0;
  while (fgets(line, sizeof line, f)) {
    if (line[0] != '#') {
      if (sscanf(line, "%d %d %d %d", &N, &C, &T, &bits) != 4) return 1;
      break;
    }
    pos = ftell(f);
  }
  (void)pos;
  const size_t in_bytes = (size_t)C * T * N * (bits == 4 ? 1 : 2);
  const size_t n_vis = (size_t)C * N * (N + 1);  /* int32 values */
  uint8_t *volt = (uint8_t *)malloc(in_bytes);
  int32_t *expect = (int32_t *)malloc(n_vis * sizeof(int32_t));
  int32_t *got = (int32_t *)malloc(n_vis * sizeof(int32_t));
  if (!volt || !expect || !got) return 1;
  for (size_t k = 0; k < in_bytes; ++k) {
    unsigned v = 0;
    if (fscanf(f, "%2x", &v) != 1) return 1;
    volt[k] = (uint8_t)v;
  }
  for (size_t k = 0; k < n_vis; ++k)
    if (fscanf(f, "%d", &expect[k]) != 1) return 1;
  fclose(f);

  mwax_job job;
  memset(&job, 0, sizeof job);
  job.n_inputs = N;
  job.n_chan = C;
  job.n_time = T;
  job.sample_bits = bits;
  mwax_plan_t plan = NULL;
  printf("plan_status %d\n", (int)mwax_plan(&plan, &job, NULL));
  void *dvolt = NULL, *dout = NULL;
  if (cudaMalloc(&dvolt, in_bytes) != cudaSuccess || cudaMalloc(&dout, n_vis * 4) != cudaSuccess ||
      cudaMemcpy(dvolt, volt, in_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
    return 1;
  printf("correlate_status %d\n", (int)mwax_correlate(plan, dvolt, N, C, T, dout));
  printf("plan_device_status %d\n", (int)mwax_plan_status(plan));
  if (cudaMemcpy(got, dout, n_vis * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  long bad = 0;
  for (size_t k = 0; k < n_vis; ++k) bad += got[k] != expect[k];
  printf("device_mismatches %ld\n", bad);
  memset(got, 0, n_vis * 4);
  printf("correlate_host_status %d\n", (int)mwax_correlate_host(plan, volt, N, C, T, got));
  bad = 0;
  for (size_t k = 0; k < n_vis; ++k) bad += got[k] != expect[k];
  printf("host_mismatches %ld\n", bad);
  printf("values_compared %ld\n", (long)n_vis);
  printf("destroy_status %d\n", (int)mwax_destroy(plan));
  cudaFree(dvolt);
  cudaFree(dout);
  free(volt);
  free(expect);
  free(got);
  return 0;
}

int main(int argc, char **argv) {
  int i = -1, j = -1;
  printf("n_baselines_512 %lld\n", (long long)mwax_n_baselines(512));
  printf("n_baselines_1024 %lld\n", (long long)mwax_n_baselines(1024));
  printf("baseline_index_5_3 %lld\n", (long long)mwax_baseline_index(5, 3));
  printf("baseline_pair_status %d\n", (int)mwax_baseline_pair(18, &i, &j));
  printf("baseline_pair_18 %d %d\n", i, j);
  printf("max_n_time_8 %lld\n", (long long)mwax_max_n_time(8));
  printf("max_n_time_4 %lld\n", (long long)mwax_max_n_time(4));
  /* a job whose integration overflows int32 is refused before any device call */
  mwax_job job = {0};
  job.n_inputs = 4;
  job.n_chan = 1;
  job.n_time = 66573;
  job.sample_bits = 8;
  mwax_plan_t plan = NULL;
  printf("plan_overflow_status %d\n", (int)mwax_plan(&plan, &job, NULL));
  printf("plan_overflow_string %s\n", mwax_status_string(MWAX_ERR_OVERFLOW_BOUND));
  /* the pair-mode work list of 8 tiles x 2 channels: 36 tile pairs per channel */
  const int64_t n = mwax_pair_work_list(8, 2, NULL, 0);
  int32_t *items = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * 7 * sizeof(int32_t));
  const int64_t m = mwax_pair_work_list(8, 2, items, n);
  long long pairs = 0;
  for (int64_t k = 0; k < m; ++k) pairs += items[7 * k] == 0 ? 1 : 2;
  printf("work_list_items %lld\n", (long long)m);
  printf("work_list_tile_pairs %lld\n", pairs);
  free(items);
  printf("calib_jones_ws_odd %lld\n", (long long)mwax_calib_jones_workspace_bytes(11, 4));
  int n_dev = 0;
  if (argc < 2 || cudaGetDeviceCount(&n_dev) != cudaSuccess || n_dev == 0) {
    printf("device_skipped 1\n");
    return 0;
  }
  return device_case(argv[1]);
}
