// Downstream consumer of the integrated powers, kept on the device: per beam
// and channel, detrend the chunk's windows (subtract their mean), normalise
// by their standard deviation and list the windows above a threshold.  This
// is the library's reading of the detrending and RFI-thresholding stages that
// follow the beamformer in the transient pipeline of Section 3 (Table 3);
// the paper names the stages without formulas.
//
// One warp per (beam, channel) row, three passes over the row (it stays in
// L1 after the first): each lane sums its strided elements in FP32 (a few
// terms), the lanes' partial sums are combined in FP64 by a fixed butterfly,
// so the mean and the population variance (of the deviations from that mean)
// carry FP64 accuracy to within a few FP32 roundings, and do not depend on
// the launch shape; z is then formed in FP32 ((P - mu) * (1 / sigma)) and
// compared with k in FP32.  GB300's FP64 rate is low, so FP64 is kept to the
// per-row reductions.
#include "bf_internal.h"

namespace bfi {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void k_detect(const float *__restrict__ P, int rows, int n_win, float k_sigma, float *__restrict__ z_out,
                         int *__restrict__ hits, int max_hits, int *__restrict__ n_hits, int n_chan)
{
    const int lane = threadIdx.x & 31;
    const long long row = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    const float *p = P + row * n_win;
    float s = 0.f;
    for (int j = lane; j < n_win; j += 32) s += p[j];
    const double mu = warp_sum((double)s) / n_win;
    const float mu_f = (float)mu;
    float v = 0.f;
    for (int j = lane; j < n_win; j += 32) {
        const float d = p[j] - mu_f;
        v = fmaf(d, d, v);
    }
    const double var = warp_sum((double)v) / n_win;
    const float inv = var > 0.0 ? (float)(1.0 / sqrt(var)) : 0.f;
    const int b = (int)(row / n_chan), c = (int)(row % n_chan);
    for (int j = lane; j < n_win; j += 32) {
        const float z = (p[j] - mu_f) * inv;
        if (z_out) z_out[row * n_win + j] = z;
        if (z > k_sigma) {
            const int k = atomicAdd(n_hits, 1);
            if (k < max_hits) {
                hits[3 * k] = b;
                hits[3 * k + 1] = c;
                hits[3 * k + 2] = j;
            }
        }
    }
}

}  // namespace bfi

using namespace bfi;

extern "C" bf_status bf_detect(const float *d_power, int n_beam, int n_chan, int n_win, float k_sigma, float *d_z,
                               int *d_hits, int max_hits, int *d_n_hits, void *stream)
{
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
