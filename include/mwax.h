/*
 * mwax.h -- C ABI of the GB300 X-engine correlator library (libmwax.so).
 *
 * The operation (paper Sec. 2): a correlator cross-correlates the
 * channelised voltages of every antenna input pair -- for the MWA, 512
 * antennas giving ~130,000 baselines, 768 channels and 4 polarisation
 * products -- and the products are integrated before calibration and
 * imaging.  For every fine channel c and input pair i >= j (the lower
 * triangle, autocorrelations included) this library computes
 *
 *     V_ij(c) = sum_{t < T} x_i(c, t) * conj(x_j(c, t))
 *     Re V_ij = sum_t xr_i xr_j + xi_i xi_j,   Im V_ij = sum_t xi_i xr_j - xr_i xi_j
 *
 * exactly, in integer arithmetic, and the gain-calibration loss that consumes
 * visibilities (Sec. 2: complex antenna gains by least squares):
 *
 *     L(g) = sum_c sum_{i > j} | g_i conj(g_j) M_ij(c) - V_ij(c) |^2
 *
 * with its gradient 2 dL/d conj(g) (PyTorch's convention for a complex
 * parameter: dL/dRe g + i dL/dIm g).
 *
 * Data layouts (all little-endian, all device memory unless stated):
 *   voltages  [n_chan][n_time][n_inputs] packed complex samples:
 *             sample_bits 4: one byte, low nibble = re, high nibble = im,
 *                            two's complement, values in [-7, 7];
 *             sample_bits 8: two bytes, re then im, int8 in [-127, 127].
 *             (-8 and -128 are outside the supported range: their negation
 *             does not fit the sample width.)
 *   input i   = 2 * tile + pol (pol 0 = X, 1 = Y); the four polarisation
 *             products of a tile pair are the four input pairs it contains.
 *   baseline  b = i (i + 1) / 2 + j for i >= j (row-major lower triangle).
 *   out       [n_chan][N(N+1)/2][2] int32 (re, im) for MWAX_KIND_EXACT,
 *             float32 (re, im) for MWAX_KIND_FP16.
 *   V, M      [n_chan][N(N+1)/2][2] float32 (re, im); g, grad [N][2] float32.
 *
 * Conventions: every function returns an mwax_status and never aborts or
 * exits.  Device work is asynchronous on the stream given to the plan (or to
 * the call); results are valid once that stream is synchronised.  The caller
 * owns every buffer it passes; a plan owns its scratch, its work list, its
 * device status word and its CUDA graph, and releases them in mwax_destroy.
 */
#ifndef MWAX_H
#define MWAX_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MWAX_OK = 0,
  MWAX_ERR_INVALID_ARG = 1,     /* null pointer, bad size, host pointer where device is required */
  MWAX_ERR_SHAPE_MISMATCH = 2,  /* call shape differs from the planned shape                  */
  MWAX_ERR_OVERFLOW_BOUND = 3,  /* n_time * 2 * max|sample|^2 exceeds INT32_MAX              */
  MWAX_ERR_UNSUPPORTED = 4,     /* device is not sm_103 / option not available             */
  MWAX_ERR_OOM = 5,             /* a plan allocation failed                                 */
  MWAX_ERR_CUDA = 6,            /* a CUDA runtime call failed                               */
  MWAX_ERR_TIMEOUT = 7          /* a bounded device-side wait gave up (see mwax_plan_status) */
} mwax_status;

typedef enum {
  MWAX_KIND_EXACT = 0, /* integer-exact visibilities, int32 output                     */
  MWAX_KIND_FP16 = 1   /* 8-bit samples only: FP16 inputs, FP32 accumulation, no integer
                          flush; float32 output (reported with its error vs FP64)     */
} mwax_kind;

typedef enum {
  MWAX_ENGINE_TENSOR = 0, /* unpack + tcgen05 tensor-core correlator + dump (default)   */
  MWAX_ENGINE_PLAIN = 1   /* CUDA-core int32 correlator, one launch per channel         */
} mwax_engine;
/* The plain engine's launch of a channel with too few 64x64 (32x32 up to 256
 * inputs) tile pairs to fill the GPU cuts the integration into ranges whose
 * partial sums are added with integer atomics; the channel's output is then
 * zeroed first with a memset on the same stream. */

/* One correlation job.  Zero-initialise, then set the shape fields; the
 * tuning fields may stay 0 (= chosen by the plan / autotuner). */
typedef struct {
  int32_t n_inputs;    /* N >= 1                                               */
  int32_t n_chan;      /* C >= 1                                               */
  int32_t n_time;      /* T >= 1 samples per integration                       */
  int32_t sample_bits; /* 4 or 8                                               */
  int32_t kind;        /* mwax_kind                                            */
  int32_t engine;      /* mwax_engine                                          */
  int32_t flush_blocks;    /* tuning: K-blocks per exact FP32 segment (0 = largest safe) */
  int32_t chan_group;      /* tuning: channels unpacked per pass (0 = auto)              */
  int32_t stages;          /* tuning: shared-memory stages: 2 narrow (3 K blocks each),
                              2..4 wide, 2 pair (2 K blocks each) (0 = auto)               */
  int32_t prefetch;        /* tuning: K-blocks of L2 prefetch ahead, 1..64 (0 = auto,
                              which is none; -1 = none); narrow and wide shapes only      */
  int32_t mma_shape;       /* tuning: 1 = M128xN128 MMAs (Re, Im separately), 2 = M128xN256
                              MMAs with [Re | Im] at once, 3 = two tile pairs (I, J),
                              (I, J+1) per work item with M128xN256 MMAs against the
                              tiles of J and J+1 (only when the whole integration is one
                              exact FP32 segment: 4-bit samples with n_time <= 171,136,
                              the FP16 kind, or flush_blocks >= the time blocks; or,
                              for longer exact single-job plans with flush_blocks 0,
                              one checked segment, see mwax_plan_info.checked_segment;
                              else MWAX_ERR_UNSUPPORTED), 4 = the same work items with
                              the unpack folded into the correlate: converter warps
                              read the packed samples and write the operand tiles into
                              shared memory, so no operand buffer and no unpack pass
                              (4-bit exact samples in one exact segment with n_inputs a
                              multiple of 16 -- every job of a batch plan --, else
                              MWAX_ERR_UNSUPPORTED); 0 = auto: 4 where it applies and
                              n_inputs <= 256 (every job), else 3 where it applies,
                              else 1                                                      */
  int32_t pipeline;        /* tuning: 1 = unpack then correlate each channel group on the
                              plan's stream, 2 = unpack the next group (second stream,
                              second scratch buffer) while the current group correlates,
                              see unpack_sms; 0 = auto (1)                               */
  int32_t timeout_ms;      /* limit of every device-side wait, ms (0 = 2000)              */
  int32_t test_fault;      /* failure-detection tests only, 0 = off: with k > 0 the
                              epilogue of the tensor correlator withholds the release of
                              its (k-1)-th accumulator segment, so the MMA warp's bounded
                              wait runs out; the call then completes with
                              MWAX_ERR_TIMEOUT in mwax_plan_status and the output is
                              invalid; the device stays usable                          */
  int32_t unpack_sms;      /* tuning, pipeline 2 only: 0 = the unpack runs as one small
                              CTA beside the correlate CTA on every SM (8-bit samples,
                              n_inputs a multiple of 8; other shapes use 20); k > 0 = k
                              SMs run the unpack while the correlate runs on the others */
  int32_t k_split;         /* tuning, exact kind in pair mode (mma_shape 3, or auto where it
                              applies) only: every work item's time blocks are cut into
                              k_split consecutive ranges, each a work item of its own
                              (the time-chunk depth of an item), whose partial int32
                              sums are added into the output with integer atomic adds
                              (exact: every partial is bounded by the whole integration's
                              int32 bound; the plan zeroes the output first).  For jobs
                              whose items alone cannot fill the SMs.  1..8 and at most
                              half the time blocks; 0 = auto: 1, or, when a launch has
                              at most half as many items as SMs, the largest k <= 8 with
                              items x k <= SMs and k <= time blocks / 2            */
} mwax_job;

/* Read-only description of a plan's choices. */
typedef struct {
  int32_t n_jobs;
  int32_t engine;
  int32_t samples_per_block; /* time samples per 128-byte operand row block           */
  int32_t flush_blocks;      /* K-blocks accumulated in FP32 before the int32 flush   */
  int32_t chan_group;        /* channels per unpack/correlate pass                     */
  int32_t grid;              /* persistent CTAs of the correlate kernel                */
  int32_t stages;            /* shared-memory pipeline stages                          */
  int32_t prefetch;          /* K-blocks of L2 prefetch ahead of the TMA loads         */
  int32_t mma_shape;         /* 1 = N128, 2 = N256 [Re | Im], 3 = two pairs per item   */
  int32_t pipeline;          /* 1 = sequential, 2 = overlapped unpack/correlate        */
  int64_t scratch_bytes;     /* device scratch owned by the plan                       */
  int64_t work_items;        /* work items per call: (job, channel, tile pair), or the
                                two-pair items of mma_shape 3                          */
  int32_t checked_segment;   /* 1: 8-bit exact job longer than one exact segment, run
                                in pair mode with each item accumulated in ONE FP32
                                segment; a check after each channel group finds every
                                channel whose largest auto-correlation Re V_ii reached
                                2^24 (by Cauchy-Schwarz no partial sum of any pair of a
                                channel exceeds that channel's largest V_ii, so all
                                other channels are exact) and a narrow launch
                                recomputes those channels with flush_blocks segments;
                                the output is exact either way.  After a call that
                                recomputed more than a quarter of its channels, the
                                next 8 calls run the narrow shape directly.  Chosen
                                when kind is exact and mma_shape and flush_blocks are
                                auto (0) or mma_shape is 3.  0 otherwise.               */
  int32_t k_split;           /* time ranges per pair-mode item (largest over the jobs) */
} mwax_plan_info;

typedef struct mwax_plan_s *mwax_plan_t;

/* ---- plans -------------------------------------------------------------- */

/* Create a plan for one job on `stream` (0 = the legacy default stream).
 * Checks the shape, the int32 bound (MWAX_ERR_OVERFLOW_BOUND when
 * n_time * 2 * max^2 > INT32_MAX, max = 7 or 127), the device
 * (MWAX_ERR_UNSUPPORTED unless compute capability 10.3), and allocates the
 * plan's scratch on the current device.  *plan is NULL on failure.
 * Test hook: with the environment variable MWAX_TEST_FAIL_ALLOC set to a
 * non-zero value, plan scratch allocations (here and in mwax_plan_batch)
 * fail with MWAX_ERR_OOM without allocating.  Every entry point of the
 * library opens an NVTX range named after itself. */
mwax_status mwax_plan(mwax_plan_t *plan, const mwax_job *job, cudaStream_t stream);

/* Plan several jobs (uneven N, C, T) that are correlated together by one
 * persistent launch per call.  On first use (and whenever the buffers
 * change) the calls are captured into two CUDA graphs: every job's unpack,
 * then the single persistent correlate launch over all jobs' work items. */
mwax_status mwax_plan_batch(mwax_plan_t *plan, const mwax_job *jobs, int n_jobs,
                            cudaStream_t stream);

/* Release everything the plan owns.  NULL is accepted. */
mwax_status mwax_destroy(mwax_plan_t plan);

mwax_status mwax_plan_get_info(mwax_plan_t plan, mwax_plan_info *info);

/* Device time of the kernels a plan launched while timing was enabled, and
 * of the host<->device copies of mwax_correlate_host. */
typedef struct {
  double unpack_ms;            /* summed device time of unpack launches            */
  double correlate_ms;         /* summed device time of correlate launches         */
  int64_t unpack_launches;
  int64_t correlate_launches;  /* tensor-core launches, or plain per-channel ones  */
  double h2d_ms;               /* summed duration of the host-path input copies    */
  double d2h_ms;               /* summed duration of the host-path output copies   */
  int64_t h2d_bytes;           /* bytes those copies moved                         */
  int64_t d2h_bytes;
  int64_t h2d_copies;
  int64_t d2h_copies;
} mwax_timing;

/* Record (enable != 0) or stop recording CUDA events on the plan's stream
 * around every kernel it launches (and, in mwax_correlate_host, on the copy
 * streams around every input and output copy).  A batch plan replays two
 * CUDA graphs per call -- all jobs' unpack launches, then the one persistent
 * correlate launch -- and times each graph launch as one unpack / correlate
 * launch. */
mwax_status mwax_plan_set_timing(mwax_plan_t plan, int enable);

/* Sums since the previous call; synchronises the plan's stream, then resets. */
mwax_status mwax_plan_get_timing(mwax_plan_t plan, mwax_timing *timing);

/* Device status word of the plan's last calls: MWAX_OK, or MWAX_ERR_TIMEOUT
 * if a bounded device wait gave up (the output is then invalid).  Reading it
 * synchronises the plan's stream; the word is cleared afterwards. */
mwax_status mwax_plan_status(mwax_plan_t plan);

/* Plans with checked_segment: the number of channels recomputed with exact
 * segments since the previous call (a measure of how often the input left
 * the one-segment window; 0 for other plans).  Synchronises the plan's
 * stream, then resets the count. */
mwax_status mwax_plan_recomputed_channels(mwax_plan_t plan, int64_t *n_channels);

/* The pair-mode work list (mma_shape 3) of one job of n_tiles x n_tiles tile
 * pairs and n_chan channels, for inspection (host only, no device use):
 * writes min(count, capacity) items of 7 int32 each, (type, c0, I0, J0, c1,
 * I1, J1) -- type 1: tile pairs (I0, J0) and (I0, J1 = J0 + 1) of channel c0;
 * type 2: the diagonal pairs (I0, I0) of channel c0 and (I1, I1) of channel
 * c1; type 0: the single pair (I0, J0) of channel c0 -- and returns the
 * count; -1 for bad arguments (n_tiles in [1, 255], n_chan >= 1). */
int64_t mwax_pair_work_list(int n_tiles, int n_chan, int32_t *items, int64_t capacity);

/* ---- autotuning ------------------------------------------------------------ */

typedef struct {
  int32_t candidates;  /* configurations timed                                        */
  int32_t from_cache;  /* 1 when the choice was read from the MWAX_TUNE_CACHE file     */
  double best_ms;      /* device time of one call with the chosen configuration        */
  double default_ms;   /* device time with the default configuration (first candidate) */
} mwax_tune_report;

/* Choose the tuning fields of a tensor-engine job (mma_shape, stages,
 * prefetch, pipeline, chan_group, k_split) by timing candidate configurations with
 * CUDA events on `voltages` / `out` (device buffers of the job's shape,
 * contents of `out` are overwritten) on `stream`.  Writes the choice into
 * *job and, when the environment variable MWAX_TUNE_CACHE names a file,
 * appends it there keyed by device name, SM count and job shape; a later
 * mwax_plan of a job whose tuning fields are all zero applies the cached
 * choice.  Synchronises `stream`.  Plain-engine jobs are left unchanged. */
mwax_status mwax_autotune(mwax_job *job, const void *voltages, void *out, cudaStream_t stream,
                          mwax_tune_report *report);

/* The same for a batch (voltages[k], out[k] as for mwax_correlate_batch):
 * first one choice of mma_shape, stages and prefetch for the launch (every
 * job runs in the one persistent kernel), then, job by job with the others
 * fixed, each job's k_split (1, 2, 4 or 8 time ranges per work item; a
 * setting replaces the automatic one only when the whole batch call is more
 * than 1 % faster).  default_ms is the batch plan's own default. */
mwax_status mwax_autotune_batch(mwax_job *jobs, int n_jobs, const void *const *voltages,
                                void *const *out, cudaStream_t stream, mwax_tune_report *report);

/* ---- correlation -------------------------------------------------------- */

/* Correlate one integration of a single-job plan.
 * voltages: device, [n_chan][n_time][n_inputs] packed samples (see above).
 * out:      device, [n_chan][N(N+1)/2][2], int32 (EXACT) or float32 (FP16).
 * Both must start on a 16-byte boundary (any cudaMalloc / torch allocation
 * does); otherwise MWAX_ERR_INVALID_ARG and nothing is launched.
 * The shape arguments must equal the planned ones (MWAX_ERR_SHAPE_MISMATCH). */
mwax_status mwax_correlate(mwax_plan_t plan, const void *voltages, int n_inputs, int n_chan,
                           int n_time, void *out);

/* Correlate every job of a batch plan: voltages[k] / out[k] are device
 * pointers for job k (16-byte aligned, as for mwax_correlate), passed in host
 * arrays of n_jobs entries. */
mwax_status mwax_correlate_batch(mwax_plan_t plan, const void *const *voltages,
                                 void *const *out);

/* Same as mwax_correlate with HOST buffers (pinned or pageable): channel
 * groups are copied in, correlated and copied out with copies overlapping
 * compute on the plan's stream and an internal copy stream.  Returns after
 * the output is complete in host memory. */
mwax_status mwax_correlate_host(mwax_plan_t plan, const void *voltages_host, int n_inputs,
                                int n_chan, int n_time, void *out_host);

/* ---- baseline triangle helpers (host) ------------------------------------ */

/* N(N+1)/2, or -1 for n_inputs < 0. */
int64_t mwax_n_baselines(int n_inputs);
/* i(i+1)/2 + j for i >= j >= 0; -1 otherwise. */
int64_t mwax_baseline_index(int i, int j);
/* Inverse of mwax_baseline_index for b >= 0. */
mwax_status mwax_baseline_pair(int64_t b, int *i, int *j);
/* Largest n_time whose visibilities fit int32 exactly: floor((2^31-1) / (2 max^2)). */
int64_t mwax_max_n_time(int sample_bits);
const char *mwax_status_string(mwax_status s);

/* ---- gain calibration (FP32) ------------------------------------------- */

/* Bytes of device workspace the calibration calls need for this shape. */
int64_t mwax_calib_workspace_bytes(int n_inputs, int n_chan);

/* L(g) into *loss (device float).  Deterministic: fixed-order reductions,
 * no floating-point atomics.  workspace: device, >= mwax_calib_workspace_bytes. */
mwax_status mwax_calib_loss(const float *V, const float *M, const float *g, int n_inputs,
                            int n_chan, void *workspace, float *loss, cudaStream_t stream);

/* grad[k] = 2 dL/d conj(g_k) into grad (device, [n_inputs][2]). */
mwax_status mwax_calib_grad(const float *V, const float *M, const float *g, int n_inputs,
                            int n_chan, void *workspace, float *grad, cudaStream_t stream);

/* Loss and gradient from one pass over V and M. */
mwax_status mwax_calib_loss_grad(const float *V, const float *M, const float *g, int n_inputs,
                                 int n_chan, void *workspace, float *loss, float *grad,
                                 cudaStream_t stream);

/* ---- gain solve (FP32) ---------------------------------------------------
 * Paper Sec. 2: the complex gain of every element comes from an iterative
 * least-squares fit of the data against a model of catalogue sources.  With
 * every gain but g_k fixed, the loss above is a linear least-squares problem
 * in g_k, minimised by
 *     h_k = sum V_kj g_j conj(M_kj) / sum |g_j|^2 |M_kj|^2   (j != k, all nu;
 *                                                             h_k = g_k if the
 *                                                             denominator is 0)
 * One sweep computes h for every input from the same g (one pass over V and
 * M, the loss/adjoint pass plus one accumulator) and then sets g = h on odd
 * sweeps and g = (g + h) / 2 on even sweeps (sweeps counted from 1; the
 * damping of Salvini & Wijnholds 2014).  The loss does not see a global phase
 * of g; the sweep keeps the phase of the starting point.
 *   g:         device [n_inputs][2], starting gains in, gains after n_iter
 *              sweeps out (updated in place).
 *   workspace: device, >= mwax_calib_solve_workspace_bytes(n_inputs, n_chan).
 *   loss_hist: device float[n_iter] or NULL; loss_hist[t] = L of the gains
 *              entering sweep t + 1 (computed by that sweep's pass).
 * V, M as in mwax_calib_loss.  Asynchronous on `stream`; deterministic (fixed
 * reduction order).  n_iter = 0 launches nothing.  Returns INVALID_ARG for
 * bad shapes, host or null pointers. */
int64_t mwax_calib_solve_workspace_bytes(int n_inputs, int n_chan);
mwax_status mwax_calib_solve(const float *V, const float *M, float *g, int n_inputs, int n_chan,
                             int n_iter, void *workspace, float *loss_hist, cudaStream_t stream);

/* ---- per-channel gains (FP32) ---------------------------------------------
 * The same fit with a complex gain for every input AND channel, g_k(nu):
 *     L(G) = sum_nu sum_{i>j} |g_i(nu) conj(g_j(nu)) M_ij(nu) - V_ij(nu)|^2.
 * The channels decouple: each channel's gradient and solve target are those
 * of the loss above restricted to that channel, with that channel's gains.
 *   G:         device float [n_chan][n_inputs][2] (re, im).
 *   grad:      device float [n_chan][n_inputs][2], grad[nu][k] = 2 dL/d conj(g_k(nu)).
 *   loss:      device float, the sum over all channels.
 *   workspace: device, >= mwax_calib_chan_workspace_bytes (loss/gradient) or
 *              mwax_calib_chan_solve_workspace_bytes (solve); partial sums per
 *              (32 x 32 input tile, channel): 0.21 GB (0.31 GB for the solve)
 *              at 1024 inputs x 768 channels.
 * mwax_calib_chan_loss_grad: loss and/or grad (one may be NULL) from one pass
 *   over V and M.
 * mwax_calib_chan_solve: n_iter sweeps of mwax_calib_solve's update
 *   (h from the same G for every input, G = h on odd sweeps, G = (G + h) / 2
 *   on even ones) applied to every channel separately; G updated in place;
 *   loss_hist (device float[n_iter] or NULL) as in mwax_calib_solve.
 * V, M as in mwax_calib_loss.  Asynchronous on `stream`; deterministic (fixed
 * reduction order, no floating-point atomics).  n_inputs in [2, 65536],
 * n_chan in [1, 524280]; INVALID_ARG otherwise or for host/null pointers.
 * The workspace-size calls return -1 for shapes outside those ranges. */
int64_t mwax_calib_chan_workspace_bytes(int n_inputs, int n_chan);
int64_t mwax_calib_chan_solve_workspace_bytes(int n_inputs, int n_chan);
mwax_status mwax_calib_chan_loss_grad(const float *V, const float *M, const float *G,
                                      int n_inputs, int n_chan, void *workspace, float *loss,
                                      float *grad, cudaStream_t stream);
mwax_status mwax_calib_chan_solve(const float *V, const float *M, float *G, int n_inputs,
                                  int n_chan, int n_iter, void *workspace, float *loss_hist,
                                  cudaStream_t stream);

/* ---- full 2x2 Jones matrices per tile (FP32) -------------------------------
 * Inputs 2a and 2a + 1 are the two polarisations of tile a.  With one 2x2
 * complex Jones matrix J_a per tile (frequency independent) the tile pair
 * a > b is the block V_ab[p][q] = V_{2a+p, 2b+q}, modelled as J_a M_ab J_b^H:
 *     L(J) = sum_nu sum_{a>b} ||J_a M_ab J_b^H - V_ab||_F^2
 * (a tile's block with itself, which holds autocorrelations, is left out).
 * Per-input gains are the diagonal case; the off-diagonal terms model
 * polarisation leakage.
 *   J:         device float [n_inputs / 2][2][2][2] (row-major 2x2, re/im).
 *   grad:      same layout, grad_a = 2 dL/d conj(J_a).
 *   workspace: device, >= mwax_calib_jones_workspace_bytes (10 MB at 1024
 *              inputs; the same for the solve).
 * mwax_calib_jones_loss_grad: loss and/or grad (one may be NULL), one pass.
 * mwax_calib_jones_solve: n_iter alternating least-squares sweeps: with the
 *   other matrices fixed, J_a's minimiser is H_a = (sum W B^H)(sum B B^H)^-1
 *   over (B, W) = (M_ab J_b^H, V_ab), b < a, and (M_ca^H J_c^H, V_ca^H),
 *   c > a, all channels; computed as H_a = J_a - (grad_a / 2) D_a^-1 with
 *   D_a = sum B B^H, J_a kept where det D_a <= 0.  J = H on odd sweeps,
 *   (J + H) / 2 on even ones; J updated in place; loss_hist as in
 *   mwax_calib_solve.
 * V, M as in mwax_calib_loss.  Asynchronous on `stream`; deterministic.
 * n_inputs even in [2, 65536], n_chan >= 1; INVALID_ARG otherwise or for
 * host/null pointers; the workspace-size call returns -1 for such shapes. */
int64_t mwax_calib_jones_workspace_bytes(int n_inputs, int n_chan);
mwax_status mwax_calib_jones_loss_grad(const float *V, const float *M, const float *J,
                                       int n_inputs, int n_chan, void *workspace, float *loss,
                                       float *grad, cudaStream_t stream);
mwax_status mwax_calib_jones_solve(const float *V, const float *M, float *J, int n_inputs,
                                   int n_chan, int n_iter, void *workspace, float *loss_hist,
                                   cudaStream_t stream);

/* ---- gridding (FP32) ------------------------------------------------------
 * Paper Sec. 2.1: the visibilities are convolved onto a regular grid so an
 * FFT can form the images; Sec. 3.2: each GPU thread gathers the values of
 * its own output cell (no floating-point atomics).  Definition (the paper
 * names no kernel or sizes): tiles a at tile_xy[a] = (X_a, Y_a) metres; every
 * tile baseline a > b and channel c (nu = f0 + c df) is a point at cell
 * coordinates x = (X_a - X_b) nu / c_light / du + Ng/2 (y likewise with Y),
 * carrying the four polarisation products V_pq (correlator inputs 2a+p and
 * 2b+q, p, q in {0 = X, 1 = Y}); the reversed baseline is the point
 * (Ng - x, Ng - y) carrying conj(V_qp).  Each point adds
 * V exp(-((s - x)^2 + (r - y)^2) / (2 sigma^2)) to cell (r, s) of grid 2p+q
 * for |s - x| < W/2, |r - y| < W/2; cells outside [0, Ng) are dropped.
 *
 * mwax_grid_plan: geometry only (host tile_xy [n_tiles][2] doubles, copied);
 *   bins the points by the first cell of their support on the GPU (counting
 *   sort, each bin in ascending point order), then stores the weights: the
 *   cells are cut into 4 x 8 patches, and for every point whose support can
 *   reach a patch (its candidates) the separable Gaussian's 8 column and 4
 *   row factors, computed in FP64 and kept in FP32 (0 outside the support):
 *   48 bytes per patch candidate, at most 12 patches per point at W = 7.  Blocks
 *   until done.  n_tiles in [2, 4096], Ng even in [8, 16384], W in [1, 31];
 *   INVALID_ARG otherwise; UNSUPPORTED when the candidates exceed 2^31; OOM /
 *   CUDA on device failures.
 * mwax_grid: vis = device correlator output [n_chan][N(N+1)/2][2] int32,
 *   N = 2 n_tiles (the layout mwax_correlate writes); grids = device float
 *   [4][Ng][Ng][2] (re, im), every cell written.  Both 8-byte aligned.
 *   Asynchronous on the plan's stream; deterministic (fixed summation order).
 * mwax_grid_plan_points: number of points that reach the grid.
 * mwax_grid_plan_entries: stored weight factors (12 per patch candidate). */
typedef struct mwax_grid_plan_s *mwax_grid_plan_t;
mwax_status mwax_grid_plan(mwax_grid_plan_t *plan, const double *tile_xy, int n_tiles, int n_chan,
                           double f0, double df, int Ng, double du, int W, double sigma,
                           cudaStream_t stream);
mwax_status mwax_grid(mwax_grid_plan_t plan, const int32_t *vis, float *grids);
int64_t mwax_grid_plan_points(mwax_grid_plan_t plan);
int64_t mwax_grid_plan_entries(mwax_grid_plan_t plan);
mwax_status mwax_grid_destroy(mwax_grid_plan_t plan);

/* ---- Stokes conversion (FP32) ----------------------------------------------
 * Paper Sec. 2.1: the instrumental polarisation images become Stokes
 * I, Q, U, V through a 4x4 matrix computed for every pixel from time and sky
 * position.  Definition (the paper gives no beam model): pixel (r, c) of an
 * n x n slant-orthographic image is at l = (c - n/2) dl, m = (r - n/2) dl;
 * above the horizon (l^2 + m^2 < 1) the ideal crossed-dipole response at
 * zenith angle theta = asin(sqrt(l^2 + m^2)) and azimuth
 * phi = atan2(m, l) + chi (chi: parallactic rotation, radians) is
 * J = [[cos th cos ph, -sin ph], [cos th sin ph, cos ph]], the sky brightness
 * is B = J^-1 C J^-T for C = [[XX, XY], [YX, YY]], and
 * (I, Q, U, V) = (B00 + B11, B00 - B11, B01 + B10, -i (B01 - B10)).
 * Pixels on or below the horizon are zero.
 *   inst:   device float [4][n][n][2] (XX, XY, YX, YY; re, im)
 *   stokes: device float [4][n][n][2] (I, Q, U, V); the two ranges of
 *           4 n^2 complex values must not overlap at all (INVALID_ARG)
 * Both 8-byte aligned; n even in [2, 65536], dl > 0; INVALID_ARG otherwise.
 * Asynchronous on `stream`. */
mwax_status mwax_stokes(const float *inst, int n, double dl, double chi, float *stokes,
                        cudaStream_t stream);

/* ---- allocation-free calibration -------------------------------------------
 * No counterpart in the paper.  For callers that must not allocate device
 * memory when they evaluate the loss -- a real-time loop in which
 * cudaMalloc/cudaFree would synchronise the device and add unbounded latency
 * to every integration, or an application whose device memory all belongs
 * to another allocator.  Same result as mwax_calib_loss_grad, but the
 * partial sums go to a fixed array of mwax_calib_static_workspace_bytes()
 * (4 MiB) inside the library that every GPU which loads it keeps until the
 * process exits; this call allocates nothing.
 *   - Shapes whose mwax_calib_workspace_bytes(n_inputs, n_chan) exceeds the
 *     array are rejected with MWAX_ERR_INVALID_ARG before any launch
 *     (1024 inputs need about 3.3 MB, for any n_chan; up to about 1150 inputs fit).
 *   - Outside stream capture every call looks up the array's device address
 *     with the current device (no allocation), so the call stays valid after
 *     a cudaDeviceReset.  A call made while `stream` is being captured uses
 *     the address from the device's last uncaptured call: make one call on
 *     each device before capturing (a captured first call returns
 *     MWAX_ERR_CUDA).
 *   - All calls on a device share the array: calls that overlap on the GPU
 *     (different streams without ordering between them) race and give wrong
 *     results.  The array keeps the last call's contents; each call writes
 *     every slot it reads, so nothing needs clearing between calls.
 * loss and/or grad (device; one may be NULL) as in mwax_calib_loss_grad. */
int64_t mwax_calib_static_workspace_bytes(void);
mwax_status mwax_calib_loss_grad_static(const float *V, const float *M, const float *g,
                                        int n_inputs, int n_chan, float *loss, float *grad,
                                        cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* MWAX_H */
