// Data-movement kernels around the beamformer:
//  - corner turn [n][c][t] -> [c][t][n] with the antenna reorder lookup of
//    Section 3 and optional FP32 -> reduced-format quantisation (round to
//    nearest even; FP8 saturating; int8/int4 clipped);
//  - expansion of 8-bit / 4-bit integer samples to FP16 (exact: |v| <= 127);
//  - the incoherent beam (square, then add; Section 1).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "bf_internal.h"

namespace bfi {

size_t dtype_sample_bytes(int dtype)
{
    switch (dtype) {
    case BF_C32: return 8;
    case BF_C16F:
    case BF_C16BF: return 4;
    case BF_C8E4M3:
    case BF_CI8: return 2;
    case BF_CI4: return 1;
    default: return 0;
    }
}

// ------------------------------------------------------------ corner turn
template <typename T>
struct Raw {
    __device__ static T conv(T v) { return v; }
};

__device__ __forceinline__ uint32_t q_f16(float2 v)
{
    __half2 h = __floats2half2_rn(v.x, v.y);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t q_bf16(float2 v)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ uint16_t q_e4m3(float2 v)
{
    return (uint16_t)__nv_cvt_float2_to_fp8x2(v, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ uint16_t q_i8(float2 v)
{
    int re = max(-127, min(127, __float2int_rn(v.x)));
    int im = max(-127, min(127, __float2int_rn(v.y)));
    return (uint16_t)((re & 0xFF) | ((im & 0xFF) << 8));
}
__device__ __forceinline__ uint8_t q_i4(float2 v)
{
    int re = max(-8, min(7, __float2int_rn(v.x)));
    int im = max(-8, min(7, __float2int_rn(v.y)));
    return (uint8_t)(((re & 0xF) << 4) | (im & 0xF));
}

template <typename Tin, typename Tout, int CONV>
__global__ void k_corner(const Tin *__restrict__ in, Tout *__restrict__ out, int N, int C, int T,
                         const int *__restrict__ perm)
{
    __shared__ Tin tile[32][33];
    const int t0 = blockIdx.x * 32, n0 = blockIdx.y * 32, c = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int j = ty; j < 32; j += 8) {
        const int n = n0 + j, t = t0 + tx;
        if (n < N && t < T) {
            const int src = perm ? perm[n] : n;
            tile[j][tx] = in[((size_t)src * C + c) * T + t];
        }
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int t = t0 + j, n = n0 + tx;
        if (n < N && t < T) {
            Tout v;
            if constexpr (CONV == 0) v = tile[tx][j];
            else if constexpr (CONV == 1) v = q_f16(tile[tx][j]);
            else if constexpr (CONV == 2) v = q_bf16(tile[tx][j]);
            else if constexpr (CONV == 3) v = q_e4m3(tile[tx][j]);
            else if constexpr (CONV == 4) v = q_i8(tile[tx][j]);
            else v = q_i4(tile[tx][j]);
            out[((size_t)c * T + t) * N + n] = v;
        }
    }
}

// 4-byte samples (FP16 / BF16 complex), 16-byte accesses on both sides: a
// block turns 32 antennas x 64 samples of one channel.  Needs T % 4 == 0,
// N % 4 == 0 and 16-byte aligned buffers (every row then starts aligned).
__global__ void k_corner4v(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int N, int C, int T,
                           const int *__restrict__ perm)
{
    __shared__ uint32_t tile[32][65];   // [antenna][sample], padded
    const int t0 = blockIdx.x * 64, n0 = blockIdx.y * 32, c = blockIdx.z;
    for (int v = threadIdx.x; v < 512; v += blockDim.x) {
        const int j = v >> 4, q = v & 15;   // antenna row j, samples 4q .. 4q+3
        const int n = n0 + j, t = t0 + 4 * q;
        if (n < N && t < T) {   // T % 4 == 0: the whole vector is in range
            const int src = perm ? perm[n] : n;
            const uint4 x = *reinterpret_cast<const uint4 *>(in + ((size_t)src * C + c) * T + t);
            tile[j][4 * q] = x.x;
            tile[j][4 * q + 1] = x.y;
            tile[j][4 * q + 2] = x.z;
            tile[j][4 * q + 3] = x.w;
        }
    }
    __syncthreads();
    for (int v = threadIdx.x; v < 512; v += blockDim.x) {
        const int i = v >> 3, q = v & 7;    // sample t0 + i, antennas 4q .. 4q+3
        const int t = t0 + i, n = n0 + 4 * q;
        if (t < T && n < N) {   // N % 4 == 0
            uint4 y;
            y.x = tile[4 * q][i];
            y.y = tile[4 * q + 1][i];
            y.z = tile[4 * q + 2][i];
            y.w = tile[4 * q + 3][i];
            *reinterpret_cast<uint4 *>(out + ((size_t)c * T + t) * N + n) = y;
        }
    }
}

// 4-byte samples with any T: 32 antennas x 128 samples per block, 4-byte
// loads (a warp reads 128 contiguous bytes of one antenna row) and 16-byte
// stores (4 antennas of one sample); needs N % 4 == 0 and a 16-byte aligned
// output.  16 loads per thread in flight.
__global__ void k_corner4s(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int N, int C, int T,
                           const int *__restrict__ perm)
{
    __shared__ uint32_t tile[32][129];   // [antenna][sample], padded
    const int t0 = blockIdx.x * 128, n0 = blockIdx.y * 32, c = blockIdx.z;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;   // 8 warps
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
        const int idx = wid * 16 + k;         // 128 (antenna, 32-sample segment) pairs
        const int j = idx >> 2, seg = idx & 3;
        const int n = n0 + j, t = t0 + seg * 32 + lane;
        if (n < N && t < T) {
            const int src = perm ? perm[n] : n;
            tile[j][seg * 32 + lane] = in[((size_t)src * C + c) * T + t];
        }
    }
    __syncthreads();
    for (int v = threadIdx.x; v < 1024; v += blockDim.x) {
        const int i = v >> 3, q = v & 7;      // sample t0 + i, antennas 4q .. 4q+3
        const int t = t0 + i, n = n0 + 4 * q;
        if (t < T && n < N) {                 // N % 4 == 0
            uint4 y;
            y.x = tile[4 * q][i];
            y.y = tile[4 * q + 1][i];
            y.z = tile[4 * q + 2][i];
            y.w = tile[4 * q + 3][i];
            *reinterpret_cast<uint4 *>(out + ((size_t)c * T + t) * N + n) = y;
        }
    }
}

cudaError_t launch_corner_turn(const void *in, int in_dtype, void *out, int out_dtype, int N, int C, int T,
                               const int *d_perm, cudaStream_t s)
{
    if ((long long)N * C * T == 0) return cudaSuccess;
    dim3 grid((T + 31) / 32, (N + 31) / 32, C), block(32, 8);
    if (in_dtype == out_dtype && dtype_sample_bytes(in_dtype) == 4 && T % 4 == 0 && N % 4 == 0 &&
        ((uintptr_t)in & 15) == 0 && ((uintptr_t)out & 15) == 0) {
        dim3 g4((T + 63) / 64, (N + 31) / 32, C);
        k_corner4v<<<g4, 256, 0, s>>>((const uint32_t *)in, (uint32_t *)out, N, C, T, d_perm);
        return cudaGetLastError();
    }
    if (in_dtype == out_dtype && dtype_sample_bytes(in_dtype) == 4 && N % 4 == 0 && ((uintptr_t)out & 15) == 0) {
        dim3 g4((T + 127) / 128, (N + 31) / 32, C);
        k_corner4s<<<g4, 256, 0, s>>>((const uint32_t *)in, (uint32_t *)out, N, C, T, d_perm);
        return cudaGetLastError();
    }
    if (in_dtype == out_dtype) {
        switch (dtype_sample_bytes(in_dtype)) {
        case 8: k_corner<uint2, uint2, 0><<<grid, block, 0, s>>>((const uint2 *)in, (uint2 *)out, N, C, T, d_perm); break;
        case 4: k_corner<uint32_t, uint32_t, 0><<<grid, block, 0, s>>>((const uint32_t *)in, (uint32_t *)out, N, C, T, d_perm); break;
        case 2: k_corner<uint16_t, uint16_t, 0><<<grid, block, 0, s>>>((const uint16_t *)in, (uint16_t *)out, N, C, T, d_perm); break;
        default: k_corner<uint8_t, uint8_t, 0><<<grid, block, 0, s>>>((const uint8_t *)in, (uint8_t *)out, N, C, T, d_perm); break;
        }
        return cudaGetLastError();
    }
    if (in_dtype != BF_C32) return cudaErrorInvalidValue;
    const float2 *fi = (const float2 *)in;
    switch (out_dtype) {
    case BF_C16F: k_corner<float2, uint32_t, 1><<<grid, block, 0, s>>>(fi, (uint32_t *)out, N, C, T, d_perm); break;
    case BF_C16BF: k_corner<float2, uint32_t, 2><<<grid, block, 0, s>>>(fi, (uint32_t *)out, N, C, T, d_perm); break;
    case BF_C8E4M3: k_corner<float2, uint16_t, 3><<<grid, block, 0, s>>>(fi, (uint16_t *)out, N, C, T, d_perm); break;
    case BF_CI8: k_corner<float2, uint16_t, 4><<<grid, block, 0, s>>>(fi, (uint16_t *)out, N, C, T, d_perm); break;
    case BF_CI4: k_corner<float2, uint8_t, 5><<<grid, block, 0, s>>>(fi, (uint8_t *)out, N, C, T, d_perm); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------- integer -> FP16 expand
__global__ void k_expand_i8(const char2 *__restrict__ in, __half2 *__restrict__ out, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) {
        char2 v = in[i];
        out[i] = __halves2half2(__int2half_rn(v.x), __int2half_rn(v.y));
    }
}

__global__ void k_expand_i4(const uint8_t *__restrict__ in, __half2 *__restrict__ out, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) {
        int b = in[i];
        int re = (b >> 4) & 0xF, im = b & 0xF;
        re = re >= 8 ? re - 16 : re;
        im = im >= 8 ? im - 16 : im;
        out[i] = __halves2half2(__int2half_rn(re), __int2half_rn(im));
    }
}

cudaError_t launch_expand_to_f16(const void *in, int in_dtype, void *out, long long n_samples, int, cudaStream_t s)
{
    if (n_samples == 0) return cudaSuccess;
    int blocks = (int)std::min<long long>(4096, (n_samples + 255) / 256);
    if (in_dtype == BF_CI8) k_expand_i8<<<blocks, 256, 0, s>>>((const char2 *)in, (__half2 *)out, n_samples);
    else if (in_dtype == BF_CI4) k_expand_i4<<<blocks, 256, 0, s>>>((const uint8_t *)in, (__half2 *)out, n_samples);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ------------------------------------------------------------ incoherent beam
template <int DT>
__device__ __forceinline__ float2 load_sample(const void *base, size_t i)
{
    if constexpr (DT == BF_C32) {
        return reinterpret_cast<const float2 *>(base)[i];
    } else if constexpr (DT == BF_C16F) {
        __half2 h = reinterpret_cast<const __half2 *>(base)[i];
        return __half22float2(h);
    } else if constexpr (DT == BF_C16BF) {
        __nv_bfloat162 h = reinterpret_cast<const __nv_bfloat162 *>(base)[i];
        return __bfloat1622float2(h);
    } else if constexpr (DT == BF_C8E4M3) {
        __nv_fp8x2_storage_t v = reinterpret_cast<const __nv_fp8x2_storage_t *>(base)[i];
        __half2 h = __half2(__nv_cvt_fp8x2_to_halfraw2(v, __NV_E4M3));
        return __half22float2(h);
    } else if constexpr (DT == BF_CI8) {
        char2 v = reinterpret_cast<const char2 *>(base)[i];
        return make_float2((float)v.x, (float)v.y);
    } else {
        int b = reinterpret_cast<const uint8_t *>(base)[i];
        int re = (b >> 4) & 0xF, im = b & 0xF;
        return make_float2((float)(re >= 8 ? re - 16 : re), (float)(im >= 8 ? im - 16 : im));
    }
}

template <int DT, bool NCT>
__global__ void k_incoherent(const void *__restrict__ x, const uint8_t *__restrict__ mask, int N, int C, int T,
                             int t_int, int T_o, float *__restrict__ out)
{
    // one warp per (channel, window): the window's t_int x N samples, 32-bit
    // index arithmetic (t_int * N < 2^31 is checked on the host), the antenna
    // of each element tracked incrementally, two accumulators per lane
    const int lane = threadIdx.x & 31;
    const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= (long long)C * T_o) return;
    const int c = (int)(wid / T_o), j = (int)(wid % T_o);
    const int n_el = t_int * N;
    float s0 = 0.f, s1 = 0.f;
    if (NCT) {
        // element i = n * t_int + tt: a warp reads consecutive samples of one antenna row
        for (int i = lane; i < n_el; i += 32) {
            const int n = i / t_int, tt = i - n * t_int;
            if (mask && !mask[n]) continue;
            const float2 v = load_sample<DT>(x, ((size_t)n * C + c) * T + (size_t)j * t_int + tt);
            s0 = fmaf(v.x, v.x, s0);
            s1 = fmaf(v.y, v.y, s1);
        }
    } else if ((DT == BF_C16F || DT == BF_C16BF) && !mask && (n_el & 3) == 0 && ((uintptr_t)x & 15) == 0 &&
               ((((size_t)c * T + (size_t)j * t_int) * N) & 3) == 0) {
        // 16-bit samples, no mask, aligned window: 16-byte loads of 4 samples,
        // eight loads in flight per lane (issued unconditionally before any is
        // used: past the window's end they re-read its last 16 bytes and are
        // replaced by zeros), summed in the same per-lane order as one load at
        // a time
        const uint4 *w4 = reinterpret_cast<const uint4 *>(x) + (((size_t)c * T + (size_t)j * t_int) * N >> 2);
        const int n4 = n_el >> 2;
        constexpr int kDepth = 8;
        for (int i0 = lane; i0 < n4; i0 += 32 * kDepth) {
            uint4 q[kDepth];
#pragma unroll
            for (int k = 0; k < kDepth; ++k) q[k] = __ldcs(w4 + min(i0 + 32 * k, n4 - 1));   // unconditional
#pragma unroll
            for (int k = 0; k < kDepth; ++k)
                if (i0 + 32 * k >= n4) q[k] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int k = 0; k < kDepth; ++k) {
                const uint32_t w[4] = {q[k].x, q[k].y, q[k].z, q[k].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float2 v;
                    if constexpr (DT == BF_C16F) {
                        v = __half22float2(*reinterpret_cast<const __half2 *>(&w[e]));
                    } else {
                        v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[e]));
                    }
                    s0 = fmaf(v.x, v.x, s0);
                    s1 = fmaf(v.y, v.y, s1);
                }
            }
        }
    } else {
        // the window is contiguous: [t_int][N] samples from (c, j * t_int)
        const size_t base = ((size_t)c * T + (size_t)j * t_int) * N;
        int n = lane % N;
        const int step = 32 % N;
        for (int i = lane; i < n_el; i += 32) {
            if (!mask || mask[n]) {
                const float2 v = load_sample<DT>(x, base + i);
                s0 = fmaf(v.x, v.x, s0);
                s1 = fmaf(v.y, v.y, s1);
            }
            n += step;
            if (n >= N) n -= N;
        }
    }
    float s = s0 + s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[(size_t)c * T_o + j] = s;
}

template <int DT>
static void inc_launch(const void *x, int layout, const uint8_t *mask, int N, int C, int T, int t_int, float *out,
                       cudaStream_t s)
{
    const int T_o = T / t_int;
    const long long warps = (long long)C * T_o;
    const unsigned blocks = (unsigned)((warps + 7) / 8);
    if (layout == BF_LAYOUT_NCT) k_incoherent<DT, true><<<blocks, 256, 0, s>>>(x, mask, N, C, T, t_int, T_o, out);
    else k_incoherent<DT, false><<<blocks, 256, 0, s>>>(x, mask, N, C, T, t_int, T_o, out);
}

cudaError_t launch_incoherent(const void *x, int dtype, int layout, const uint8_t *d_mask, int N, int C, int T,
                              int t_int, float *out, cudaStream_t s)
{
    if ((long long)C * (T / t_int) == 0) return cudaSuccess;
    if ((long long)t_int * N >= (1ll << 31)) return cudaErrorInvalidValue;
    switch (dtype) {
    case BF_C32: inc_launch<BF_C32>(x, layout, d_mask, N, C, T, t_int, out, s); break;
    case BF_C16F: inc_launch<BF_C16F>(x, layout, d_mask, N, C, T, t_int, out, s); break;
    case BF_C16BF: inc_launch<BF_C16BF>(x, layout, d_mask, N, C, T, t_int, out, s); break;
    case BF_C8E4M3: inc_launch<BF_C8E4M3>(x, layout, d_mask, N, C, T, t_int, out, s); break;
    case BF_CI8: inc_launch<BF_CI8>(x, layout, d_mask, N, C, T, t_int, out, s); break;
    case BF_CI4: inc_launch<BF_CI4>(x, layout, d_mask, N, C, T, t_int, out, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace bfi
