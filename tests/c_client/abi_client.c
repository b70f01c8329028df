/* A plain C program against include/mwax.h and libmwax.so: no Python, no
 * torch.  It exercises the host-only entry points (no GPU needed) and prints
 * one "name value" line per check for the test that runs it. */
#include <stdio.h>
#include <stdlib.h>

#include "mwax.h"

int main(void) {
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
  return 0;
}
