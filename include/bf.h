/*
 * bf.h — C ABI of the GB300 (sm_103a) frequency-domain coherent beamformer.
 *
 * The library computes, for every beam b, channel c and integration window j,
 *
 *     P[b][c][j] = sum_{t = j*T_int}^{(j+1)*T_int - 1} | sum_n W[c][b][n] X[n][c][t] |^2
 *     W[c][b][n] = exp(-i 2 pi f_c (r_n . s_b) / c0),   c0 = 299 792 458 m/s
 *
 * from channelised complex antenna voltages X (Section 2.1 of "GPU-Powered
 * Coherent Beamforming", Magro, Zarb Adami & Hickish: beamforming as a
 * per-channel matrix-vector product with power detection inside the kernel;
 * the weights are the phase terms of Eq. 1).  A partial last window
 * (T mod T_int samples) is dropped.
 *
 * Conventions for every call:
 *  - Host pointers ("h_" or documented as host) are read during the call only
 *    and never retained.  Device pointers ("d_") are caller-owned global memory
 *    of the current device; the library never frees them.
 *  - The plan owns its weights, tuning choice and scratch; bf_destroy frees
 *    them.  Nothing allocated by the library is handed to the caller.
 *  - Calls that take a stream enqueue work on it and return without waiting
 *    (stream-ordered, asynchronous) unless documented as synchronous.  A NULL
 *    stream means the plan's stream given to bf_plan_create.
 *  - Every call returns a bf_status.  On failure nothing observable has been
 *    enqueued, and bf_last_error() returns a thread-local message.  No call
 *    throws across the ABI.
 *  - Device-side waits are bounded; a wait that gives up records
 *    BF_ERR_TIMEOUT in the plan, reported by the next bf_sync.
 *  - A plan may be used by one host thread at a time, and its executes run
 *    one after another on the device: they share the plan's scratch, so
 *    executes of one plan on different streams must be ordered (events) by
 *    the caller.
 */
#ifndef BF_H
#define BF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bf_status {
    BF_OK = 0,
    BF_ERR_ARG = 1,          /* invalid argument, shape or dtype mismatch */
    BF_ERR_NOMEM = 2,        /* device or pinned host allocation failed */
    BF_ERR_CUDA = 3,         /* a CUDA runtime or driver call failed */
    BF_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    BF_ERR_UNSUPPORTED = 5,  /* well-formed request this build cannot run */
    BF_ERR_STATE = 6         /* call not valid in the plan's current state */
} bf_status;

/* Storage of one complex voltage sample (Section 2.1 uses 4-bit complex;
 * the reduced-precision tensor-core modes are this library's).  Samples
 * are stored as interleaved (re, im) pairs except BF_CI4. */
typedef enum bf_dtype {
    BF_C32 = 0,     /* 2 x float32; IEEE FP32 FFMA path, relative error <= 1e-5 */
    BF_C16F = 1,    /* 2 x float16; FP16 tensor cores, FP32 accumulation */
    BF_C16BF = 2,   /* 2 x bfloat16; BF16 tensor cores, FP32 accumulation */
    BF_C8E4M3 = 3,  /* 2 x FP8 E4M3FN; FP8 tensor cores, per-beam weight scale */
    BF_CI8 = 4,     /* 2 x int8; exact products (int8 -> FP16), per-beam weight scale */
    BF_CI4 = 5      /* 1 byte: re in the high nibble, im in the low nibble,
                       two's complement -8..7 (the F-engine format of Section 2.1) */
} bf_dtype;

/* Order of the voltage array. */
typedef enum bf_layout {
    BF_LAYOUT_CTN = 0,  /* X[c][t][n]: channel, sample, antenna fastest (the
                           packet order of Section 3); no corner turn */
    BF_LAYOUT_NCT = 1   /* X[n][c][t]: antenna-major; a corner-turn kernel
                           re-lays it as [c][t][n] in plan scratch first */
} bf_layout;

/* Kernel family choice for bf_plan_set_kernel. */
typedef enum bf_kernel {
    BF_KERNEL_AUTO = 0, /* FP32 -> SIMT FFMA kernel; other dtypes -> tensor cores */
    BF_KERNEL_SIMT = 1, /* CUDA-core FP32 kernel (BF_C32 only) */
    BF_KERNEL_TC = 2    /* tcgen05/TMEM kernel (all dtypes except BF_C32) */
} bf_kernel;

typedef struct bf_plan bf_plan;

/*
 * bf_plan_create — validate the geometry and allocate a plan on the current
 * device, then generate the weights (as bf_weights(plan, NULL)).
 *
 *  out       [out] receives the plan handle (NULL on failure).
 *  n_ant     N >= 1 antennas.
 *  pos_m     host, [N][3] doubles: antenna positions r_n in metres (any origin;
 *            integrated powers do not depend on it).
 *  mask      host, [N] bytes or NULL: antenna n is used iff mask[n] != 0
 *            (sub-arraying with an antenna mask, Section 3.1).  Masked antennas
 *            get zero weight.
 *  n_chan    C >= 1 channels.  freqs_hz: host, [C] doubles, channel centre
 *            frequencies f_c in Hz (> 0).
 *  n_beam    B >= 1 beams.  dirs: host, [B][3] doubles, unit pointing vectors s_b
 *            (|s_b| = 1 within 1e-6).
 *  dtype     bf_dtype of the voltages (and of the tensor-core operands).
 *  t_int     T_int >= 1 samples per integration window.
 *  layout    bf_layout of the voltages passed to the execute calls.
 *  stream    cudaStream_t for plan work (NULL = the legacy default stream).
 *
 * Errors: BF_ERR_ARG for a NULL required pointer, a non-positive size, a
 * non-finite position or frequency, or a non-unit direction;
 * BF_ERR_UNSUPPORTED for a dtype/shape the kernels cannot run (e.g. a
 * tensor-core mode whose antenna count does not fill 16-byte rows);
 * BF_ERR_NOMEM / BF_ERR_CUDA from the device.
 */
bf_status bf_plan_create(bf_plan **out, int n_ant, const double *pos_m,
                         const uint8_t *mask, int n_chan, const double *freqs_hz,
                         int n_beam, const double *dirs, int dtype, int t_int,
                         int layout, void *stream);

/*
 * bf_weights — (re)generate the plan's weights on the device (Eq. 1; the
 * phase argument f_c (r_n . s_b) / c0 is formed and reduced modulo one cycle
 * in FP64, then sin/cos are taken in FP32 and the result is stored in the
 * plan's operand format).  dirs: host [B][3] new pointing vectors (tracking
 * beams, Section 3.1) or NULL to regenerate the current ones.  Asynchronous
 * on the plan stream.  Errors: BF_ERR_ARG for a non-unit direction.
 */
bf_status bf_weights(bf_plan *plan, const double *dirs);

/*
 * bf_execute — integrated beam powers.
 *  d_voltages  device, n_samp samples per channel in the plan's dtype and
 *              layout: CTN -> [C][n_samp][N] samples, NCT -> [N][C][n_samp].
 *              16-byte aligned.
 *  n_samp      T >= 0 samples per channel.
 *  d_power     device, float [B][C][T / T_int] (T / T_int rounded down).
 *  stream      cudaStream_t or NULL for the plan stream.
 * Powers are in units of |weight|^2 |voltage|^2 (unit-modulus weights, no
 * normalisation); per-beam weight scales of the FP8/int8 modes are applied.
 * 8- and 4-bit integer samples are widened to FP16 inside the beamforming
 * kernel when the weights stay resident (K <= 3 blocks of 128 bytes per
 * weight row, e.g. up to 96 antennas) and a sample row is a multiple of 16
 * bytes (N % 8 == 0 for 8-bit, N % 16 == 0 for 4-bit); other plans widen
 * them into plan scratch first (4 bytes per sample).
 * Errors: BF_ERR_ARG (NULL pointer, n_samp < 0, misaligned pointer).
 */
bf_status bf_execute(bf_plan *plan, const void *d_voltages, int n_samp,
                     float *d_power, void *stream);

/*
 * bf_execute_complex — beam voltages without detection (the S-engine style
 * complex beam output of Section 1.1; also a test hook for the raw sums).
 *  d_beams  device, float [B][C][n_samp][2] (re, im), 8-byte aligned.
 * Same arguments and errors as bf_execute (BF_ERR_ARG also for d_beams not
 * 8-byte aligned).
 */
bf_status bf_execute_complex(bf_plan *plan, const void *d_voltages, int n_samp,
                             float *d_beams, void *stream);

/*
 * bf_execute_incoherent — incoherent beam (square, then add; Section 1):
 *  d_power  device, float [C][T / T_int], sum over the window of sum_n |X|^2
 *           over the unmasked antennas.
 */
bf_status bf_execute_incoherent(bf_plan *plan, const void *d_voltages, int n_samp,
                                float *d_power, void *stream);

/*
 * bf_execute_host — bf_execute from and to HOST memory, SYNCHRONOUS: copies
 * the voltages to plan-owned device memory (pipelined over channel blocks on
 * two streams so copies overlap the kernels, Section 2.2), runs the kernels
 * and copies the powers back before returning.  Pinned host memory gives the
 * full link rate; pageable memory works but is slower.
 *  h_voltages  host, same layout as bf_execute's d_voltages (CTN only).
 *  h_power     host, float [B][C][T / T_int].
 * Errors: as bf_execute; BF_ERR_UNSUPPORTED for the NCT layout.
 */
bf_status bf_execute_host(bf_plan *plan, const void *h_voltages, int n_samp,
                          float *h_power);

/*
 * bf_sync — wait for all work the plan enqueued on its streams and report any
 * device-side timeout recorded since the last bf_sync (BF_ERR_TIMEOUT), or a
 * CUDA error (BF_ERR_CUDA).  Clears the recorded timeout.
 */
bf_status bf_sync(bf_plan *plan);

/* bf_destroy — free everything the plan owns (synchronises its streams first).
 * NULL is accepted. */
bf_status bf_destroy(bf_plan *plan);

/* Thread-local message for the last failing call on this thread ("" if none).
 * Valid until the next library call on the same thread. */
const char *bf_last_error(void);

/*
 * bf_plan_set_kernel — choose the kernel family and the time-tile width.
 *  kernel  bf_kernel.  tile_t: samples per tile (0 = automatic).  For the
 *  tensor-core kernel a multiple of 16 in [16, 256] and of T_int (or of
 *  2*T_int); for the SIMT kernel ignored.
 * Errors: BF_ERR_UNSUPPORTED if the family cannot run the plan's dtype.
 */
bf_status bf_plan_set_kernel(bf_plan *plan, int kernel, int tile_t);

/*
 * bf_plan_set_tiles — tensor-core tiling (each 0 = automatic):
 *  tile_t       samples per tile (MMA N), as in bf_plan_set_kernel;
 *  group_tiles  128-row weight tiles (64 beams each) kept resident in shared
 *               memory while a CTA walks along time (1..16);
 *  x_stages     voltage tiles in flight (2..4).
 * The autotuner (paper_1412_4907_gb300.tune) searches these.  No effect on
 * BF_C32 plans.  Errors: BF_ERR_ARG for out-of-range values,
 * BF_ERR_UNSUPPORTED if the combination does not fit in shared memory.
 */
bf_status bf_plan_set_tiles(bf_plan *plan, int tile_t, int group_tiles, int x_stages);

/* bf_plan_query_tiles — the tiling in use (any output may be NULL): tile_t,
 * group_tiles, x_stages and the number of weight groups per channel.
 * x_stages is 0 for plans whose weights are streamed (K >= 4 blocks of 128
 * bytes per weight row): those run the batched kernel's pipeline, which sizes
 * its own stages; set_tiles' group_tiles and x_stages do not apply to them. */
bf_status bf_plan_query_tiles(const bf_plan *plan, int *tile_t, int *group_tiles,
                              int *x_stages, int *n_groups);

/*
 * bf_plan_set_input_order — the antenna order of the voltage stream differs
 * from the array order of pos_m/mask (the F-engine lookup table of Section 3):
 * array antenna n arrives in input slot perm[n] (host [N] ints, a permutation
 * of 0..N-1; NULL restores the identity).  Applied to the weights, so the
 * voltages are never gathered.  Synchronises the plan stream, then
 * regenerates the weights.  Errors: BF_ERR_ARG if perm is not a permutation.
 */
bf_status bf_plan_set_input_order(bf_plan *plan, const int *perm);

/*
 * bf_plan_set_weight_buffers — n = 2: the plan keeps two weight buffers, and
 * bf_weights (tracking: re-pointing every chunk, Section 3) regenerates into
 * the one not in use on a plan-owned stream, after the last execute that
 * read it, then makes it current; executes on any stream wait for the latest
 * refresh (stream-ordered, no host synchronisation).  So the refresh for the
 * next chunk overlaps the beamforming of the current one.  Costs one more
 * copy of the weights in device memory.  n = 1 (the default) frees it.
 * Synchronises the plan's streams.  A plan with two buffers cannot join a
 * batch or a server.  Errors: BF_ERR_ARG, BF_ERR_NOMEM.
 */
bf_status bf_plan_set_weight_buffers(bf_plan *plan, int n);

/*
 * bf_plan_query — report the plan's choices (any output pointer may be NULL):
 *  kernel (bf_kernel actually used), tile_t, beams per weight group resident
 *  in shared memory (tensor-core kernel), and bytes of device memory owned.
 */
bf_status bf_plan_query(const bf_plan *plan, int *kernel, int *tile_t,
                        int *group_tiles, size_t *device_bytes);

/*
 * bf_export_weights — copy the plan's weights, decoded from the operand
 * format to complex float32 without the per-beam scale, into
 *  d_w      device, float [C][B][N][2]
 *  d_scale  device, float [C][B] per-beam scale sigma_b (1 for FP32/FP16/BF16),
 *           or NULL.
 * The effective weight is sigma_b * d_w.  Asynchronous on the plan stream.
 */
bf_status bf_export_weights(bf_plan *plan, float *d_w, float *d_scale);

/*
 * bf_corner_turn — stand-alone corner turn (Section 3 antenna reorder):
 * antenna-major d_in[N][C][T] (complex samples of in_dtype) ->
 * d_out[C][T][N] (out_dtype), output antenna n taken from input row perm[n]
 * (host [N] ints, or NULL for identity).  Converting BF_C32 to a reduced
 * dtype rounds to nearest even (FP8 saturates at +-448, int8 clips at +-127);
 * other conversions are BF_ERR_UNSUPPORTED.  Asynchronous on `stream`.
 */
bf_status bf_corner_turn(const void *d_in, int in_dtype, void *d_out, int out_dtype,
                         int n_ant, int n_chan, int n_samp, const int *perm,
                         void *stream);

/*
 * Batched execution: the jobs of several plans in one step.
 *
 * A batch groups plans that differ in antennas, beams, channels and sample
 * counts (sub-arrays, beam sets, observing modes sharing a GPU) so that a
 * step over all of them is one call (and one CUDA graph replay), scheduled
 * by job size instead of one launch per plan:
 *  - jobs of fewer than 4 K blocks of 64 operand elements (fewer than 128
 *    antennas at 16 bits) run their plan's resident-weight kernel, several
 *    at a time on streams forked from the step's stream;
 *  - the others run the streamed-weight persistent kernel: a job of at least
 *    64 tiles per SM gets a launch to itself, and the smaller ones share one
 *    launch whose CTAs take tiles from a work counter.  Section 4 measures one beamformer configuration at a time; this is
 * the same computation (Eq. 1 weights, Section 2.1 fused power detection)
 * applied to many configurations at once.
 *
 * Every plan of a batch must be a tensor-core plan (not BF_C32) in the CTN
 * layout, on one device, with the same operand format (BF_C16F, BF_CI8 and
 * BF_CI4 share the FP16 format; BF_C16BF and BF_C8E4M3 stand alone) and the
 * same T_int.  The batch keeps pointers to the plans: they must outlive it,
 * and their weights are read at execution time (bf_weights on a member plan
 * takes effect at the next batch step, stream-ordered as usual).
 */
typedef struct bf_batch bf_batch;

/*
 * bf_batch_create — batch over plans[0 .. n_plans-1] (host array, read
 * during the call).  tile_t = 0 chooses the widest tile (samples per MMA, a
 * multiple of 16 and of T_int, at most 256 and 16 windows); otherwise that
 * width (of the persistent launch; resident-weight jobs keep their plan's
 * tiling).  Allocates the device job table (one entry per plan), a pinned
 * host copy, and the fork streams.  Errors: BF_ERR_ARG (NULL or empty), BF_ERR_UNSUPPORTED
 * (plans that cannot share a launch, no tile width fits), BF_ERR_NOMEM /
 * BF_ERR_CUDA.
 */
bf_status bf_batch_create(bf_batch **out, bf_plan *const *plans, int n_plans, int tile_t);

/*
 * bf_batch_set — bind job `job` (index into the plans given at creation) to
 *  d_voltages  device, CTN [C][n_samp][N] complex samples of the plan's dtype,
 *              16-byte aligned (N * sample bytes a multiple of 16 for TMA);
 *  n_samp      samples per channel (0 = the job contributes nothing);
 *  d_power     device, float [B][C][n_samp / T_int], 16-byte aligned.
 * Waits for the batch's last step to finish (the job table it read is
 * rewritten) and discards a captured graph.  Errors: BF_ERR_ARG.
 */
bf_status bf_batch_set(bf_batch *batch, int job, const void *d_voltages, int n_samp, float *d_power);

/*
 * bf_batch_execute — one step over every job on `stream` (NULL = the legacy
 * default stream): the resident-weight jobs run on streams that wait for
 * `stream` and that `stream` then waits for (8/4-bit inputs are widened in
 * their kernel when TMA can read the rows, else in a batch-owned buffer);
 * the other jobs' integer inputs are widened to FP16 in batch-owned buffers
 * and persistent launches compute their powers.  Asynchronous: when
 * `stream` has reached the step's end, every output is written.  Errors:
 * BF_ERR_STATE if a job was never set.
 */
bf_status bf_batch_execute(bf_batch *batch, void *stream);

/*
 * bf_batch_capture / bf_batch_replay — record one bf_batch_execute on
 * `stream` (non-NULL, not already capturing) into a CUDA graph, then launch
 * that graph on any stream.  Replays read the inputs and write the outputs
 * bound by bf_batch_set at capture time; a later bf_batch_set drops the
 * graph (BF_ERR_STATE from replay until captured again).
 */
bf_status bf_batch_capture(bf_batch *batch, void *stream);
bf_status bf_batch_replay(bf_batch *batch, void *stream);

/* bf_batch_sync — wait for the batch's last step; BF_ERR_TIMEOUT if a
 * device-side wait of that step gave up (the flag is then cleared). */
bf_status bf_batch_sync(bf_batch *batch);

/* bf_batch_query — tile width and work units (channel x time tile x 64-beam
 * block) of the persistent launch, and useful FLOPs per step over all jobs
 * (8 N B C n_samp summed); any output may be NULL. */
bf_status bf_batch_query(const bf_batch *batch, int *tile_t, long long *units, double *flops);

/* bf_batch_destroy — wait for the last step and free the batch (not the
 * plans).  NULL is a no-op. */
bf_status bf_batch_destroy(bf_batch *batch);

/*
 * Serving: a real-time loop over voltage chunks of several streams.
 *
 * Each stream is one configuration (a plan: sub-array, beams, channels,
 * dtype); its chunks are consecutive pieces of one voltage stream [C][T][N]
 * (CTN, the plan's dtype) of any length.  Chunks are submitted from host
 * memory as they arrive; a scheduler thread admits them into a device arena
 * of fixed size as memory frees up, runs each step (at most one chunk per
 * stream, any mix of streams) as one batched tensor-core launch, and copies
 * the powers back into host memory.  A chunk's copy to the device starts as
 * soon as it is admitted, so copies overlap the launches of earlier chunks.  The weights (in the plans) and the open integration
 * window of every stream stay on the device: a chunk completes the window the
 * previous chunk of its stream left open (Section 2.1 integration across
 * buffer boundaries, Section 3 real-time operation), so a stream integrates
 * the same whatever its cut into chunks.
 *
 * The plans must satisfy the bf_batch_create rules; additionally N * 2 *
 * (bytes per MMA operand element: 2 for 16-bit and widened integer inputs,
 * 1 for FP8) must be a multiple of 16.  The server keeps pointers to the
 * plans; they must outlive it and must not be re-pointed while it runs.
 */
typedef struct bf_server bf_server;

/* One finished chunk.  Times are seconds on the host steady clock
 * (bf_server_now). */
typedef struct bf_completion {
    long long id;        /* as returned by bf_server_submit */
    int config;          /* stream index */
    int status;          /* bf_status of the chunk */
    int n_windows;       /* windows completed by this chunk: h_power holds [B][C][n_windows] */
    int step;            /* scheduler step that computed it */
    int n_samp;          /* samples per channel in the chunk */
    double t_submit;     /* bf_server_submit returned */
    double t_start;      /* admitted: its copy to the device was enqueued */
    double t_done;       /* its powers were in host memory */
} bf_completion;

typedef struct bf_server_counters {
    long long submitted, completed, steps;
    int max_jobs_per_step;
    int tile_t;
    double flops;        /* 8 N B C T summed over completed chunks */
    double kernel_ms;    /* device time of the batched launches (CUDA events) */
    double copy_in_ms;   /* span of each step's host-to-device chunk copies, summed */
    double copy_in_bytes;
    size_t arena_bytes, arena_peak;
} bf_server_counters;

/*
 * bf_server_create — server over plans[0 .. n_configs-1] (host array, read
 * during the call; at most 16 streams).  mem_bytes: device arena for admitted chunks (voltages,
 * FP16 widening of integer inputs, powers); a chunk waits until its block
 * fits.  max_steps (1..8): steps in flight at once.  tile_t as
 * bf_batch_create.  Waits for the plans' weights, allocates the arena and
 * two [B][C] float accumulators per stream, starts the scheduler thread.
 */
bf_status bf_server_create(bf_server **out, bf_plan *const *plans, int n_configs, size_t mem_bytes,
                           int max_steps, int tile_t);

/*
 * bf_server_submit — queue a chunk of stream `config`:
 *  h_voltages  host, [C][n_samp][N] samples of the plan's dtype (page-locked
 *              memory lets the copy run asynchronously), read until the chunk
 *              completes;
 *  h_power     host, room for [B][C][ceil(n_samp / T_int)] floats, written
 *              before the completion is reported;
 *  id          out (may be NULL): the chunk's id.
 * Thread-safe.  Errors: BF_ERR_ARG (bad config, n_samp < 1, a chunk that
 * could never fit the arena), BF_ERR_STATE (shutting down).
 */
bf_status bf_server_submit(bf_server *server, int config, const void *h_voltages, int n_samp,
                           float *h_power, long long *id);

/* bf_server_pause — paused != 0: admit and dispatch nothing until resumed
 * (submitted chunks queue; steps already enqueued finish), for instance to
 * hold dispatch while the caller prepares a burst.  bf_server_destroy
 * resumes. */
bf_status bf_server_pause(bf_server *server, int paused);

/* bf_server_poll — move up to `max` completions (oldest first) into out[],
 * their count into *n_out; waits up to timeout_ms for the first one. */
bf_status bf_server_poll(bf_server *server, bf_completion *out, int max, int *n_out, int timeout_ms);

/* bf_server_drain — wait up to timeout_ms until every submitted chunk has
 * completed.  BF_ERR_TIMEOUT if some have not; BF_ERR_CUDA if the scheduler
 * met a CUDA error (the chunks concerned complete with that status). */
bf_status bf_server_drain(bf_server *server, int timeout_ms);

/* bf_server_stats — counters since creation (chunks, steps, FLOPs, device
 * time, arena use). */
bf_status bf_server_stats(bf_server *server, bf_server_counters *out);

/* bf_server_destroy — finish every queued chunk, stop the scheduler, free
 * the server (not the plans).  Completions not polled are discarded. */
bf_status bf_server_destroy(bf_server *server);

/* bf_server_now — the host steady clock of bf_completion, in seconds. */
double bf_server_now(void);

/*
 * bf_detect — a consumer of the integrated powers that keeps them on the
 * device (the transient-detection stages after the beamformer, Section 3,
 * Table 3: detrending and thresholding; the paper gives no formulas, so this
 * is the library's reading): for every beam b and channel c over the n_win
 * windows of d_power [B][C][n_win] (device, float),
 *   mu = mean_j P,  sigma = sqrt(mean_j (P - mu)^2)   (FP32, two passes,
 *   fixed reduction order),  z[b][c][j] = (P - mu) / sigma   (0 where sigma = 0),
 * written to d_z (device, float [B][C][n_win], or NULL), and every (b, c, j)
 * with z > k_sigma appended to d_hits (device, int [max_hits][3], in no
 * particular order); *d_n_hits (device int) receives the number of hits,
 * which may exceed max_hits (only the first max_hits are stored).
 * Asynchronous on `stream`.  Errors: BF_ERR_ARG.
 */
bf_status bf_detect(const float *d_power, int n_beam, int n_chan, int n_win, float k_sigma,
                    float *d_z, int *d_hits, int max_hits, int *d_n_hits, void *stream);

/*
 * bf_selftest_timeout — diagnostic of the failure path: launches a one-warp
 * kernel that waits, with the bounded wait every pipelined kernel of the
 * library uses, on an mbarrier that nothing arrives at.  After limit_ms
 * (0 < limit_ms <= 10000) the wait gives up, records the timeout in a status
 * word and the kernel returns; the context stays usable.  Synchronous on
 * `stream`.  Returns BF_ERR_TIMEOUT when the path works as designed,
 * BF_ERR_CUDA if the wait did not report, BF_ERR_ARG for a bad limit.
 */
bf_status bf_selftest_timeout(double limit_ms, void *stream);

/*
 * bf_measure_ffma — measurement aid, not part of the paper's method: the FP32
 * FFMA rate of the current GPU (independent FFMA chains on every SM for about
 * `seconds`), the peak the plain FP32 form (BF_C32) is held against.
 *  seconds  in (0, 60];  tflops  host, receives FLOP/s / 1e12 (2 FLOP per FFMA).
 * Synchronous; allocates and frees a small device buffer.  Errors: BF_ERR_ARG.
 */
bf_status bf_measure_ffma(double seconds, double *tflops, void *stream);

/*
 * bf_execute_nct_static — bf_execute for an antenna-major (BF_LAYOUT_NCT)
 * tensor-core plan that allocates nothing.  The paper has no counterpart: it
 * exists for callers that cannot allocate device memory when they execute
 * (allocators that forbid cudaMalloc after set-up, real-time loops that must
 * not pay for an allocation or the synchronisation of freeing one, processes
 * with a fixed memory budget).  bf_execute lays the corner-turned voltages out
 * in plan scratch that it allocates (and grows) on first use; this call uses
 * a fixed 64 MiB array in device memory instead, which every GPU that loads
 * the library holds until the process exits.
 *  d_voltages, n_samp, d_power, stream: as bf_execute.  The corner-turned
 *  input, C * n_samp * N samples of the plan's dtype (plus 4 bytes per sample
 *  for BF_CI8 / BF_CI4 plans that bf_execute widens in scratch, see there),
 *  must fit in the 64 MiB; larger inputs return BF_ERR_ARG without doing
 *  anything.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the one array and it keeps the last call's
 * contents: calls whose work overlaps on the GPU (other streams, other plans,
 * other threads) race on it and must be serialised by the caller.  Nothing in
 * it needs to start at zero.  Errors: BF_ERR_UNSUPPORTED for a CTN or FP32
 * plan; otherwise as bf_execute.
 */
bf_status bf_execute_nct_static(bf_plan *plan, const void *d_voltages, int n_samp,
                                float *d_power, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BF_H */
