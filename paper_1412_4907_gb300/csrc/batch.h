// Internal interface of the batched tensor-core launch, shared by the
// bf_batch_* calls and the serving loop (bf_server_*).
//
// A launch walks a table of jobs.  Each job is one chunk of one plan: its
// voltages [C][T][2N] (TMA tensor map), the plan's weight rows (tensor map),
// per-beam scales and the output powers.  A job may continue an integration
// that the previous chunk of the same stream left open: the first t_shift
// samples of its first window belong to that chunk and their partial sum
// arrives in acc_in; a window that this chunk leaves open is written, as a
// partial sum, to acc_out instead of the output (Section 2.1 integration,
// carried across chunk boundaries).
#pragma once
#include <cudaTypedefs.h>

#include "bf_internal.h"

namespace bfi {

struct __align__(128) BatchJob {
    CUtensorMap xmap;   // voltages [C][T][2N]
    CUtensorMap wmap;   // weight rows [C][M_pad][K_pad]
    long long unit0;    // first global unit of the job
    long long units;    // C x t_tiles x mt
    int C, t_tiles, mt, kb, ke;
    int c_base, c_total;   // weight / output channel of the job's channel 0; output channel count
    int T, T_o, B, b_pad;
    int t_shift;        // samples of window 0 that precede this chunk (0..T_int-1)
    int ks_last;        // MMA k-steps (of 4) holding antennas in the last K block
    uint32_t idesc;
    const float *wscale;   // [C][b_pad] sigma^2, or NULL (unscaled formats)
    const float *wsig;
    float *out;            // [B][C][T_o]
    const float *acc_in;   // [B][C] partial sum of window 0 carried in, or NULL
    float *acc_out;        // [B][C] partial sum of window T_o carried out, or NULL
};

static_assert(sizeof(BatchJob) == 384, "job table rows are 384 bytes (64 fit in the launch parameters)");

// Launch-wide choices: tile width and the pipeline depths that follow.
struct BatchCore {
    int nt = 256, nsplit = 2, wpt = 4, t_int = 64, xst = 2, nacc = 2, smem = 0;
    bool f8 = false;
    bool cpx = false;   // complex beams [B][C][T][2] instead of powers (single plans only)
    bool direct = false; // power epilogue stores windows itself (256-sample tiles, T_int 16/32/64)
    int num_sms = 1;
};

// Checks that the plans can share one launch (tensor-core, one operand
// format, one T_int, one device) and picks the tile width (tile_t = 0: the
// widest that fits).  Sets the kernels' shared-memory attribute.  The kernel
// reads [C][T][2N] operand voltages: callers with antenna-major input corner
// turn it first (bf_batch_create and bf_server_create accept CTN plans only).
bf_status batch_core_init(BatchCore *core, bf_plan *const *plans, int n, int tile_t);

// Fills one job.  x_mma: the voltages as the MMA reads them (the FP16
// widening for 8/4-bit integer inputs), [c_count][T][2N] for the plan's
// channels c_base .. c_base + c_count - 1 (c_count < 0: all channels).  T_o,
// t_tiles and units follow from T, t_shift and whether acc_out is given.
bf_status batch_fill_job(const BatchCore &core, BatchJob *J, const bf_plan *p, const void *x_mma, int T,
                         float *out, int t_shift, const float *acc_in, float *acc_out, int c_base = 0,
                         int c_count = -1);

// Numbers the units of jobs[0..n) in order; returns the total.
long long batch_index(BatchJob *jobs, int n);

// One persistent launch over the table (already in device memory).  d_err:
// status word of the device-side waits.  d_next: the launch's work counter
// (device, 8 bytes), zeroed on `s` before the launch, so launches sharing a
// counter must be ordered on the device; NULL: CTA i takes units i, i + G,
// ... (G = grid size).  The counter keeps the CTAs of a launch over several
// jobs on neighbouring units; one job alone runs faster on the fixed stride
// (46.9 against 48.8 ms for the 20 sub-array jobs of 128 and 256 antennas of
// the uneven-batch workload launched one at a time).
cudaError_t batch_core_launch(const BatchCore &core, const BatchJob *d_jobs, int n, long long total_units,
                              unsigned *d_err, unsigned long long *d_next, cudaStream_t s);

// Jobs a launch can take by value in its parameters (64 x 384 bytes = 24 KB,
// within the 32 KB parameter space of current CUDA): no table copy, so nothing
// of the launch waits behind other host-to-device copies, and the tensor maps
// are read from the parameter bank.  On the 20 sub-array jobs of 128 and 256
// antennas of the uneven-batch workload a step took 48.6 ms with the table in
// the parameters against 50.7 ms with it in device memory.
constexpr int kParamJobs = 64;
struct ParamJobs {
    BatchJob j[kParamJobs];
};

// One persistent launch over jobs[0 .. n-1] (n <= kParamJobs) passed by
// value.  Used by single plans with large antenna counts (n = 1), the serving
// loop and small batches.
cudaError_t batch_core_launch_params(const BatchCore &core, const BatchJob *jobs, int n, long long total_units,
                                     unsigned *d_err, unsigned long long *d_next, cudaStream_t s);
// One job alone, on the fixed stride.
cudaError_t batch_core_launch_one(const BatchCore &core, const BatchJob &job, unsigned *d_err, cudaStream_t s);

}  // namespace bfi
