// FP32 beamformer on the CUDA cores (IEEE FFMA; no tensor cores, no TF32),
// the "plain FP32 form" of the method: per channel, beams = W (B x N) times
// voltages (N x T), then |.|^2 summed over each integration window
// (Section 2.1).  Weights are reused for every sample a block processes
// (the static-beam reuse of Section 2.1).
//
// Block: 64 beams x 64 samples of one channel, 256 threads, each thread a
// 4-beam x 4-sample register tile; antennas are staged through shared memory
// 16 at a time.  In power mode a block owns whole integration windows and
// sums |B|^2 of each window in ascending sample order (deterministic).
#include "bf_internal.h"

namespace bfi {

constexpr int kSB = 64;   // beams per block
constexpr int kST = 64;   // samples per sub-block
constexpr int kAK = 16;   // antennas per shared-memory stage
constexpr int kPad = 2;   // float2 padding per shared row (keeps 16-byte alignment)

template <bool NCT, bool COMPLEX>
__global__ void __launch_bounds__(256) k_simt(const float2 *__restrict__ X, const float2 *__restrict__ W,
                                              float *__restrict__ out, int N, int c_base, int c_in_stride,
                                              int c_total, int B, int b_pad, int T, int t_int, int T_o,
                                              int wins_per_block)
{
    __shared__ __align__(16) float2 sW[kAK][kSB + kPad];
    __shared__ __align__(16) float2 sX[kAK][kST + kPad];
    __shared__ float pw[kSB][kST + 1];
    extern __shared__ float sacc[];   // [kSB][wins_per_block]

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int c = blockIdx.z;                  // channel within this launch
    const int cg = c_base + c;                 // channel in the plan
    const int b0 = blockIdx.y * kSB;

    int t_begin, t_end, j0 = 0;
    if (COMPLEX) {
        t_begin = blockIdx.x * 128;
        t_end = min(T, t_begin + 128);
    } else {
        j0 = blockIdx.x * wins_per_block;
        t_begin = j0 * t_int;
        t_end = min(T_o, j0 + wins_per_block) * t_int;
        for (int i = tid; i < kSB * wins_per_block; i += 256) sacc[i] = 0.f;
    }
    const float2 *Wc = W + ((size_t)cg * b_pad + b0) * N;

    for (int ts = t_begin; ts < t_end; ts += kST) {
        float2 acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

        for (int a0 = 0; a0 < N; a0 += kAK) {
            for (int idx = tid; idx < kAK * kSB; idx += 256) {
                int bl = idx / kAK, a = idx % kAK;
                sW[a][bl] = (a0 + a < N) ? Wc[(size_t)bl * N + a0 + a] : make_float2(0.f, 0.f);
            }
            if (NCT) {
                for (int idx = tid; idx < kAK * kST; idx += 256) {
                    int a = idx / kST, tl = idx % kST;
                    int t = ts + tl;
                    sX[a][tl] = (a0 + a < N && t < t_end)
                                    ? X[((size_t)(a0 + a) * c_in_stride + c) * T + t]
                                    : make_float2(0.f, 0.f);
                }
            } else {
                for (int idx = tid; idx < kAK * kST; idx += 256) {
                    int tl = idx / kAK, a = idx % kAK;
                    int t = ts + tl;
                    sX[a][tl] = (a0 + a < N && t < t_end) ? X[((size_t)c * T + t) * N + a0 + a]
                                                          : make_float2(0.f, 0.f);
                }
            }
            __syncthreads();
#pragma unroll 4
            for (int a = 0; a < kAK; ++a) {
                const float4 w01 = *reinterpret_cast<const float4 *>(&sW[a][4 * ty]);
                const float4 w23 = *reinterpret_cast<const float4 *>(&sW[a][4 * ty + 2]);
                const float4 x01 = *reinterpret_cast<const float4 *>(&sX[a][4 * tx]);
                const float4 x23 = *reinterpret_cast<const float4 *>(&sX[a][4 * tx + 2]);
                const float2 w[4] = {make_float2(w01.x, w01.y), make_float2(w01.z, w01.w),
                                     make_float2(w23.x, w23.y), make_float2(w23.z, w23.w)};
                const float2 x[4] = {make_float2(x01.x, x01.y), make_float2(x01.z, x01.w),
                                     make_float2(x23.x, x23.y), make_float2(x23.z, x23.w)};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        acc[i][j].x = fmaf(w[i].x, x[j].x, acc[i][j].x);
                        acc[i][j].x = fmaf(-w[i].y, x[j].y, acc[i][j].x);
                        acc[i][j].y = fmaf(w[i].x, x[j].y, acc[i][j].y);
                        acc[i][j].y = fmaf(w[i].y, x[j].x, acc[i][j].y);
                    }
            }
            __syncthreads();
        }

        if (COMPLEX) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int b = b0 + 4 * ty + i;
                if (b >= B) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    int t = ts + 4 * tx + j;
                    if (t < t_end)
                        reinterpret_cast<float2 *>(out)[((size_t)b * c_total + cg) * T + t] = acc[i][j];
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    pw[4 * ty + i][4 * tx + j] = fmaf(acc[i][j].x, acc[i][j].x, acc[i][j].y * acc[i][j].y);
            __syncthreads();
            const int ts_end = min(ts + kST, t_end);
            for (int p = tid; p < kSB * wins_per_block; p += 256) {
                int bl = p / wins_per_block, wl = p % wins_per_block;
                int w_lo = max((j0 + wl) * t_int, ts), w_hi = min((j0 + wl + 1) * t_int, ts_end);
                float s = 0.f;
                for (int t = w_lo; t < w_hi; ++t) s += pw[bl][t - ts];
                sacc[p] += s;
            }
            __syncthreads();
        }
    }

    if (!COMPLEX) {
        for (int p = tid; p < kSB * wins_per_block; p += 256) {
            int bl = p / wins_per_block, wl = p % wins_per_block;
            int b = b0 + bl, j = j0 + wl;
            if (b < B && j < T_o) out[((size_t)b * c_total + cg) * T_o + j] = sacc[p];
        }
    }
}

cudaError_t launch_simt_range(bf_plan *p, const void *x, int c_base, int c_launch, int T, float *out,
                              int complex_out, cudaStream_t s)
{
    const bool nct = p->layout == BF_LAYOUT_NCT;
    const int T_o = T / p->t_int;
    const int wins = std::max(1, std::min(128, (128 + p->t_int - 1) / p->t_int));
    const int nx = complex_out ? (T + 127) / 128 : (T_o + wins - 1) / wins;
    if (nx == 0 || c_launch == 0) return cudaSuccess;
    dim3 grid(nx, p->wf.b_pad / kSB, c_launch);
    const size_t dyn = complex_out ? 0 : sizeof(float) * kSB * wins;
    const float2 *X = reinterpret_cast<const float2 *>(x);
    const float2 *W = reinterpret_cast<const float2 *>(p->d_w);
    const int c_in_stride = nct ? p->C : c_launch;
#define BF_SIMT_LAUNCH(NCTV, CPX)                                                                       \
    do {                                                                                                \
        cudaError_t e_ = cudaFuncSetAttribute(k_simt<NCTV, CPX>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                              (int)(sizeof(float) * kSB * 128));                        \
        if (e_ != cudaSuccess) return e_;                                                               \
        k_simt<NCTV, CPX><<<grid, 256, dyn, s>>>(X, W, out, p->N, c_base, c_in_stride, p->C, p->B,      \
                                                 p->wf.b_pad, T, p->t_int, T_o, wins);                   \
    } while (0)
    if (nct) {
        if (complex_out) BF_SIMT_LAUNCH(true, true);
        else BF_SIMT_LAUNCH(true, false);
    } else {
        if (complex_out) BF_SIMT_LAUNCH(false, true);
        else BF_SIMT_LAUNCH(false, false);
    }
#undef BF_SIMT_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_simt(bf_plan *p, const void *x, int T, float *out, int complex_out, cudaStream_t s)
{
    return launch_simt_range(p, x, 0, p->C, T, out, complex_out, s);
}

}  // namespace bfi
