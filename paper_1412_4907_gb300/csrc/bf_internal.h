// Internal declarations shared by the host API and the kernel files.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "bf.h"

namespace bfi {
struct BatchCore;

constexpr double kC0 = 299792458.0;      // m/s
constexpr int kRowsPerMTile = 128;       // tensor-core tile rows (MMA M)
constexpr int kBeamsPerMTile = 64;       // each beam owns a re row and an im row
constexpr int kKBlockBytes = 128;        // one swizzled K block = 128-byte rows
constexpr int kSmemLimit = 227 * 1024;   // dynamic shared memory per CTA

// Operand element formats of the tensor-core kernel.
enum OpFmt { kOpF16 = 0, kOpBF16 = 1, kOpE4M3 = 2 };

// Weight storage chosen for a plan.
struct WeightFormat {
    bool simt = false;   // float2 [C][B][N]
    int op = kOpF16;     // tensor-core rows [C][M_pad][K_pad] of this format
    int es = 2;          // bytes per operand element
    int ke = 64;         // elements per 128-byte K block
    int kb = 1;          // K blocks per row
    int k_pad = 64;      // elements per row
    int m_pad = 128;     // rows per channel
    int b_pad = 64;      // beams per channel (multiple of 64)
    float qmax = 0.f;    // > 0: per-beam scale sigma_b = max|component| / qmax
};

// Requested tensor-core tiling (0 = choose automatically).
struct TcRequest {
    int tile_t = 0;      // samples per tile (MMA N)
    int group_tiles = 0; // M tiles whose weights stay resident
    int x_stages = 0;    // voltage tiles in flight
};

// Tensor-core launch configuration.
struct TcConfig {
    int nt = 256;        // time-tile (MMA N)
    int xst = 2;         // voltage stages in flight (streamed: weight+voltage K-block stages)
    bool stream = false; // weights streamed per K block instead of resident
    int nsplit = 2;      // epilogue column halves
    int group = 1;       // M tiles whose weights stay resident per work unit
    int n_groups = 1;
    int smem = 0;
    bool fast_windows = true;   // T_int % 16 == 0
    // 8/4-bit inputs widened inside the resident-weight kernel: raw bytes of one
    // 128-byte FP16 K block per sample row (64 for int8, 32 for 4-bit), else 0
    // (FP16/BF16/FP8 inputs, or integer rows whose stride TMA cannot read)
    int raw_kb = 0;
};

struct TcArgs {
    const void *x;       // [C_launch][T][2N] operand voltages
    int c_base, c_launch, c_total;
    int T, T_o, t_int;
    int complex_out;
    float *out;          // power [B][C_total][T_o] or beams [B][C_total][T][2]
    unsigned *err = nullptr;   // status word of the device-side waits (NULL: the plan's)
};

bf_status set_error(bf_status s, const std::string &msg);
void clear_error();   // every entry point starts with this: bf_last_error() then describes this call only
bf_status cuda_error(cudaError_t e, const char *what);

}  // namespace bfi

struct bf_plan {
    int N = 0, C = 0, B = 0, dtype = 0, t_int = 1, layout = 0;
    int kernel = BF_KERNEL_AUTO;
    bfi::TcRequest tc_req;
    int num_sms = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t stream2 = nullptr;   // host-to-device copies of bf_execute_host
    cudaStream_t stream3 = nullptr;   // device-to-host copies of bf_execute_host
    static constexpr int kEvents = 16;
    cudaEvent_t ev[kEvents] = {};

    std::vector<double> pos, freqs, dirs;
    std::vector<uint8_t> mask;
    std::vector<int> perm;            // input slot of each array antenna (empty = identity)

    double *d_pos = nullptr, *d_freqs = nullptr, *d_dirs = nullptr;
    uint8_t *d_mask = nullptr;
    double *d_tau = nullptr;          // [B][N] geometric delays (s)
    unsigned long long *d_ab = nullptr;   // [B][N][2] frac(f0 tau), frac(df tau) in 2^-64 cycles
    bool uniform_freqs = false;       // f_c = f0 + c df within 1 uHz
    double f0 = 0.0, df = 0.0;

    bfi::WeightFormat wf;
    void *d_w = nullptr;              // weights in the format above
    size_t w_bytes = 0;
    float *d_wscale = nullptr;        // [C][b_pad] power scale sigma_b^2
    float *d_wsig = nullptr;          // [C][b_pad] sigma_b

    bfi::TcConfig tc;
    bfi::BatchCore *bcore = nullptr;  // streamed power path (large K): the batched kernel, one job

    void *d_scratch = nullptr;        // corner-turn / expansion output
    size_t scratch_bytes = 0;
    void *d_hx = nullptr;             // bf_execute_host staging (voltages)
    size_t hx_bytes = 0;
    float *d_hp = nullptr;            // bf_execute_host staging (powers)
    size_t hp_bytes = 0;

    // double-buffered weights (bf_plan_set_weight_buffers): the refresh fills
    // the other buffer on wstream while executes read the current one
    int wbufs = 1, wcur = 0;
    void *wbuf[2] = {nullptr, nullptr};
    float *wscale_buf[2] = {nullptr, nullptr}, *wsig_buf[2] = {nullptr, nullptr};
    cudaStream_t wstream = nullptr;
    cudaEvent_t ev_wready = nullptr;                  // the latest refresh is complete
    cudaEvent_t ev_wused[2] = {nullptr, nullptr};     // the last execute that read buffer i

    unsigned *d_err = nullptr;        // device-side status word
    size_t dev_bytes = 0;
};

namespace bfi {

// k_weights.cu
cudaError_t launch_delays(bf_plan *p, cudaStream_t s);
cudaError_t launch_weights(bf_plan *p, cudaStream_t s);
cudaError_t launch_export_weights(bf_plan *p, float *d_w, float *d_scale, cudaStream_t s);

// k_simt.cu
cudaError_t launch_simt(bf_plan *p, const void *x, int T, float *out, int complex_out, cudaStream_t s);
cudaError_t launch_simt_range(bf_plan *p, const void *x, int c_base, int c_launch, int T, float *out,
                              int complex_out, cudaStream_t s);

// k_tc.cu
bool tc_choose(bf_plan *p, const TcRequest &req, TcConfig *cfg, std::string *why);
cudaError_t launch_tc(bf_plan *p, const TcArgs &a, cudaStream_t s, std::string *why);

// k_aux.cu
cudaError_t launch_corner_turn(const void *in, int in_dtype, void *out, int out_dtype, int N, int C, int T,
                               const int *d_perm, cudaStream_t s);
cudaError_t launch_expand_to_f16(const void *in, int in_dtype, void *out, long long n_samples, int N,
                                 cudaStream_t s);
cudaError_t launch_incoherent(const void *x, int dtype, int layout, const uint8_t *d_mask, int N, int C,
                              int T, int t_int, float *out, cudaStream_t s);

size_t dtype_sample_bytes(int dtype);

}  // namespace bfi
