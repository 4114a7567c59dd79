// Downstream consumer of the integrated powers, kept on the device: per beam
// and channel, detrend the chunk's windows (subtract their mean), normalise
// by their standard deviation and list the windows above a threshold.  This
// is the library's reading of the detrending and RFI-thresholding stages that
// follow the beamformer in the transient pipeline of Section 3 (Table 3);
// the paper names the stages without formulas.
//
// One warp per (beam, channel) row, three passes over the row (in registers
// for rows of up to 256 windows, else re-read from L1), all in FP32 with a
// fixed reduction order (lane-strided partial sums, then a butterfly), so
// the result does not depend on the launch shape: the mean, then the
// population variance as the mean of the squared deviations from it (two
// passes: no cancellation), then z = (P - mu) / sigma compared with k.
// GB300's FP64 rate is a small fraction of its FP32 rate, so FP64 here
// would make the kernel arithmetic-bound; the FP32 statistics agree with
// the FP64 oracle to ~1e-6 relative.
#include "bf_internal.h"

namespace bfi {

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kRowRegs = 8;   // rows of up to 256 windows are held in registers

__global__ void k_detect(const float *__restrict__ P, int rows, int n_win, float k_sigma, float *__restrict__ z_out,
                         int *__restrict__ hits, int max_hits, int *__restrict__ n_hits, int n_chan)
{
    const int lane = threadIdx.x & 31;
    const long long row = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    const float *p = P + row * n_win;
    const int b = (int)(row / n_chan), c = (int)(row % n_chan);
    auto hit = [&](float z, int j) {
        if (z > k_sigma) {
            const int k = atomicAdd(n_hits, 1);
            if (k < max_hits) {
                hits[3 * k] = b;
                hits[3 * k + 1] = c;
                hits[3 * k + 2] = j;
            }
        }
    };
    if (n_win <= 32 * kRowRegs) {
        // the row in registers: every load issued before any is used (indices
        // clamped to the row, the surplus masked), then the three passes run
        // on registers in the same per-lane order as the loops below
        float r[kRowRegs];
#pragma unroll
        for (int k = 0; k < kRowRegs; ++k) r[k] = __ldcs(p + min(lane + 32 * k, n_win - 1));
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kRowRegs; ++k)
            if (lane + 32 * k < n_win) s += r[k];
        const float mu_f = warp_sum(s) / (float)n_win;
        float v = 0.f;
#pragma unroll
        for (int k = 0; k < kRowRegs; ++k)
            if (lane + 32 * k < n_win) {
                const float d = r[k] - mu_f;
                v = fmaf(d, d, v);
            }
        const float var = warp_sum(v) / (float)n_win;
        const float inv = var > 0.f ? 1.f / sqrtf(var) : 0.f;
#pragma unroll
        for (int k = 0; k < kRowRegs; ++k) {
            const int j = lane + 32 * k;
            if (j < n_win) {
                const float z = (r[k] - mu_f) * inv;
                if (z_out) __stcs(z_out + row * n_win + j, z);
                hit(z, j);
            }
        }
        return;
    }
    float s = 0.f;
    for (int j = lane; j < n_win; j += 32) s += p[j];
    const float mu_f = warp_sum(s) / (float)n_win;
    float v = 0.f;
    for (int j = lane; j < n_win; j += 32) {
        const float d = p[j] - mu_f;
        v = fmaf(d, d, v);
    }
    const float var = warp_sum(v) / (float)n_win;
    const float inv = var > 0.f ? 1.f / sqrtf(var) : 0.f;
    for (int j = lane; j < n_win; j += 32) {
        const float z = (p[j] - mu_f) * inv;
        if (z_out) z_out[row * n_win + j] = z;
        hit(z, j);
    }
}

}  // namespace bfi

using namespace bfi;

extern "C" bf_status bf_detect(const float *d_power, int n_beam, int n_chan, int n_win, float k_sigma, float *d_z,
                               int *d_hits, int max_hits, int *d_n_hits, void *stream)
{
    clear_error();
    if (n_beam < 0 || n_chan < 0 || n_win < 0 || max_hits < 0) return set_error(BF_ERR_ARG, "negative size");
    if (!d_n_hits) return set_error(BF_ERR_ARG, "d_n_hits is NULL");
    if (max_hits > 0 && !d_hits) return set_error(BF_ERR_ARG, "d_hits is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_n_hits, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_error(e, "hit counter");
    const long long rows = (long long)n_beam * n_chan;
    if (rows == 0 || n_win == 0) return BF_OK;
    if (!d_power) return set_error(BF_ERR_ARG, "d_power is NULL");
    if (rows > (1ll << 31) - 1) return set_error(BF_ERR_ARG, "too many rows");
    const int warps = 8;
    const long long blocks = (rows + warps - 1) / warps;
    k_detect<<<(unsigned)blocks, warps * 32, 0, s>>>(d_power, (int)rows, n_win, k_sigma, d_z, d_hits, max_hits,
                                                      d_n_hits, n_chan);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "detection kernel");
    return BF_OK;
}
