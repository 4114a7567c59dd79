// FP32 beamformer on the CUDA cores (IEEE FFMA; no tensor cores, no TF32),
// the "plain FP32 form" of the method: per channel, beams = W (B x N) times
// voltages (N x T), then |.|^2 summed over each integration window
// (Section 2.1).  Weights are reused for every sample a block processes
// (the static-beam reuse of Section 2.1).
//
// Block: 64 beams x 64 samples of one channel, 256 threads, each thread a
// 4-beam x 4-sample register tile.  Two forms: a pipelined one (below) for
// complex beams and for windows of 16, 32 or 64 samples, and a general one
// for any other T_int, in which antennas are staged through shared memory 16
// at a time and a block owns whole integration windows, summing |B|^2 of
// each window in ascending sample order (deterministic).
#include <type_traits>

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

// ------------------------------------------------------------ pipelined form
// 128 beams x 64 samples per block, each thread an 8-beam x 4-sample register
// tile (6 shared-memory loads per 128 FFMA); a block walks a run of
// 64-sample sub-tiles of one channel and beam block, and its operands come in
// through a two-stage cp.async pipeline: antenna chunks of kKA (voltages, and
// weights unless the whole weight tile is resident, N <= kKA) for the next
// step land while the current one is multiplied.  Used for complex beams and
// for powers whose windows (T_int = WIN of 16, 32 or 64) divide a sub-tile:
// each thread squares its 4 samples of 4 beams and the window sums are
// reduced across the WIN / 4 lanes that hold the window, in a fixed order.
constexpr int kKA = 32;   // antennas per pipeline step
constexpr int kRun = 16;  // sub-tiles (1024 samples) per block; twice that with resident weights
constexpr int kPB = 128;  // beams per block of the pipelined form

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, bool valid)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gmem), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// RES (N <= kKA: the weights are loaded once and stay): four voltage stages,
// one barrier per step and runs of 32 sub-tiles per block; otherwise two
// stages of voltages and of weights, a second barrier that frees a stage
// for the step after next, and runs of 16 sub-tiles.
template <bool NCT, bool COMPLEX, int WIN, bool RES>
__global__ void __launch_bounds__(256, 2)
    k_simt_pipe(const float2 *__restrict__ X, const float2 *__restrict__ W, float *__restrict__ out, int N,
                int c_base, int c_in_stride, int c_total, int B, int b_pad, int T, int T_o, int t_end)
{
    // dynamic shared memory (100 KB either way): voltage stages, then weight stages
    constexpr int XS = RES ? 4 : 2;
    extern __shared__ __align__(16) float2 pipe_smem[];
    auto sX = reinterpret_cast<float2(*)[kKA][kST + kPad]>(pipe_smem);
    auto sW = reinterpret_cast<float2(*)[kKA][kPB + kPad]>(pipe_smem + XS * kKA * (kST + kPad));

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int c = blockIdx.z;
    const int cg = c_base + c;
    const int b0 = blockIdx.y * kPB;
    constexpr int RUN = RES ? 2 * kRun : kRun;
    const int sub0 = blockIdx.x * RUN;
    const int n_sub = min(RUN, (t_end - sub0 * kST + kST - 1) / kST);
    const int n_chunk = RES ? 1 : (N + kKA - 1) / kKA;
    const bool w_resident = n_chunk == 1;
    const int n_step = n_sub * n_chunk;
    const float2 *Wc = W + ((size_t)cg * b_pad + b0) * N;

    // issue the copies of step q (sub-tile q / n_chunk, antenna chunk q % n_chunk) into stage q % XS
    auto load = [&](int q) {
        const int st = q % XS;
        const int sub = sub0 + q / n_chunk, a0 = (q % n_chunk) * kKA;
        const int t0 = sub * kST;
        for (int i = tid; i < kKA * kST; i += 256) {
            int a, tl;
            if (NCT) {
                a = i / kST;
                tl = i % kST;
            } else {
                tl = i / kKA;
                a = i % kKA;
            }
            const int t = t0 + tl, an = a0 + a;
            const bool ok = an < N && t < t_end;
            const float2 *src = NCT ? X + ((size_t)(ok ? an : 0) * c_in_stride + c) * T + (ok ? t : 0)
                                    : X + ((size_t)c * T + (ok ? t : 0)) * N + (ok ? an : 0);
            cp_async8(&sX[st][a][tl], src, ok);
        }
        if (!w_resident || q == 0)
            for (int i = tid; i < kKA * kPB; i += 256) {
                const int bl = i / kKA, a = i % kKA;
                const bool ok = a0 + a < N && b0 + bl < b_pad;   // rows past the padded beams read zero
                cp_async8(&sW[RES ? 0 : st][a][bl], Wc + (ok ? (size_t)bl * N + a0 + a : 0), ok);
            }
        cp_async_commit();
    };

    float2 acc[8][4];
    load(0);
    if (RES && n_step > 1) load(1);
    if (RES && n_step > 2) load(2);
    for (int q = 0; q < n_step; ++q) {
        if (RES) {
            // steps q .. q + 2 are in flight; the barrier also tells that every
            // thread has finished step q - 1, whose stage load(q + 3) refills
            if (q + 2 < n_step) cp_async_wait2();
            else if (q + 1 < n_step) cp_async_wait1();
            else cp_async_wait0();
            __syncthreads();
            if (q + 3 < n_step) load(q + 3);
        } else {
            if (q + 1 < n_step) {
                load(q + 1);
                cp_async_wait1();
            } else {
                cp_async_wait0();
            }
            __syncthreads();
        }
        const int st = q % XS, k = q % n_chunk;
        const int ws = w_resident ? 0 : st;
        // one antenna: 8 beams x 4 samples of complex multiply-adds; the first
        // antenna of a sub-tile starts the sums with products (no zeroing)
        auto mac = [&](int a, auto first) {
            float2 w[8];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float4 v = *reinterpret_cast<const float4 *>(&sW[ws][a][8 * ty + 2 * h]);
                w[2 * h] = make_float2(v.x, v.y);
                w[2 * h + 1] = make_float2(v.z, v.w);
            }
            const float4 x01 = *reinterpret_cast<const float4 *>(&sX[st][a][4 * tx]);
            const float4 x23 = *reinterpret_cast<const float4 *>(&sX[st][a][4 * tx + 2]);
            const float2 x[4] = {make_float2(x01.x, x01.y), make_float2(x01.z, x01.w), make_float2(x23.x, x23.y),
                                 make_float2(x23.z, x23.w)};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if constexpr (decltype(first)::value) {
                        acc[i][j].x = __fmul_rn(w[i].x, x[j].x);
                        acc[i][j].y = __fmul_rn(w[i].x, x[j].y);
                    } else {
                        acc[i][j].x = fmaf(w[i].x, x[j].x, acc[i][j].x);
                        acc[i][j].y = fmaf(w[i].x, x[j].y, acc[i][j].y);
                    }
                    acc[i][j].x = fmaf(-w[i].y, x[j].y, acc[i][j].x);
                    acc[i][j].y = fmaf(w[i].y, x[j].x, acc[i][j].y);
                }
        };
        int a_first = 0;
        if (k == 0) {
            mac(0, std::true_type{});
            a_first = 1;
        }
#pragma unroll 1
        for (int a = a_first; a < kKA; ++a) mac(a, std::false_type{});
        if (k == n_chunk - 1) {
            const int t_sub = (sub0 + q / n_chunk) * kST;
            if (COMPLEX) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int b = b0 + 8 * ty + i;
                    if (b >= B) continue;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int t = t_sub + 4 * tx + j;
                        if (t < t_end) reinterpret_cast<float2 *>(out)[((size_t)b * c_total + cg) * T + t] = acc[i][j];
                    }
                }
            } else {
                constexpr int L = WIN / 4;   // lanes per window
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float pw = 0.f;
#pragma unroll
                    for (int j = 0; j < 4; ++j) pw = fmaf(acc[i][j].x, acc[i][j].x, fmaf(acc[i][j].y, acc[i][j].y, pw));
#pragma unroll
                    for (int m = 1; m < L; m <<= 1) pw += __shfl_xor_sync(0xffffffffu, pw, m);
                    const int b = b0 + 8 * ty + i, j = (t_sub + 4 * tx) / WIN;
                    if ((tx % L) == 0 && b < B && j < T_o) out[((size_t)b * c_total + cg) * T_o + j] = pw;
                }
            }
        }
        if (!RES) __syncthreads();   // the stage is free for step q + 2
    }
}

cudaError_t launch_simt_range(bf_plan *p, const void *x, int c_base, int c_launch, int T, float *out,
                              int complex_out, cudaStream_t s)
{
    const bool nct = p->layout == BF_LAYOUT_NCT;
    const int T_o = T / p->t_int;
    const int t_int = p->t_int;
    if (complex_out || t_int == 16 || t_int == 32 || t_int == 64) {
        // pipelined form: complex beams (every sample) or powers of whole windows
        const int t_end = complex_out ? T : T_o * t_int;
        const int n_sub = (t_end + kST - 1) / kST;
        if (n_sub == 0 || c_launch == 0) return cudaSuccess;
        const int run = p->N <= kKA ? 2 * kRun : kRun;   // sub-tiles per block (the kernel's RUN)
        dim3 grid((n_sub + run - 1) / run, (p->wf.b_pad + kPB - 1) / kPB, c_launch);
        const float2 *X = reinterpret_cast<const float2 *>(x);
        const float2 *W = reinterpret_cast<const float2 *>(p->d_w);
        const int c_in_stride = nct ? p->C : c_launch;
        // up to kKA antennas the weights stay resident: three voltage stages, one weight stage
        const bool res = p->N <= kKA;
        const int pipe_smem = res ? (int)(sizeof(float2) * kKA * (4 * (kST + kPad) + (kPB + kPad)))
                                  : (int)(sizeof(float2) * 2 * kKA * ((kST + kPad) + (kPB + kPad)));
#define BF_SIMT_PIPE(NCTV, CPX, WV)                                                                             \
    do {                                                                                                        \
        auto k_ = res ? k_simt_pipe<NCTV, CPX, WV, true> : k_simt_pipe<NCTV, CPX, WV, false>;                   \
        cudaError_t e_ = cudaFuncSetAttribute(k_, cudaFuncAttributeMaxDynamicSharedMemorySize, pipe_smem);      \
        if (e_ != cudaSuccess) return e_;                                                                       \
        k_<<<grid, 256, pipe_smem, s>>>(X, W, out, p->N, c_base, c_in_stride, p->C, p->B, p->wf.b_pad, T, T_o,  \
                                        t_end);                                                                 \
    } while (0)
#define BF_SIMT_PIPE_W(NCTV)                          \
    do {                                              \
        if (complex_out) BF_SIMT_PIPE(NCTV, true, 64); \
        else if (t_int == 64) BF_SIMT_PIPE(NCTV, false, 64); \
        else if (t_int == 32) BF_SIMT_PIPE(NCTV, false, 32); \
        else BF_SIMT_PIPE(NCTV, false, 16);           \
    } while (0)
        if (nct) BF_SIMT_PIPE_W(true);
        else BF_SIMT_PIPE_W(false);
#undef BF_SIMT_PIPE_W
#undef BF_SIMT_PIPE
        return cudaGetLastError();
    }
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
