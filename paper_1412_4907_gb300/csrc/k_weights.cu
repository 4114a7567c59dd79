// Weight generation (Eq. 1): W[c][b][n] = exp(-i 2 pi f_c (r_n . s_b) / c0).
//
// The phase in cycles, f_c * tau[b][n] with tau = (r_n . s_b) / c0, is
// reduced modulo one cycle before sin/cos: a 200 m baseline at 416 MHz spans
// ~277 cycles, and FP32 would keep only ~1.7e-5 cycle of the fraction.
// Two exact ways of doing the reduction:
//  - any channel list: per weight, f_c * tau and its fractional part in FP64;
//  - uniformly spaced channels f_c = f_0 + c df (checked on the host to
//    1 uHz): per (beam, antenna), alpha = frac(f_0 tau) and beta =
//    frac(df tau) are formed in FP64 and kept as 64-bit fixed-point
//    fractions of a cycle; the phase of channel c is alpha + c beta modulo
//    2^64, exact in integer arithmetic, so no per-weight FP64 work remains.
// The reduced phase is then exact in FP32 to 2^-25 cycle and sin/cos are
// taken in FP32 (sincospif).  The weights are computed once per plan or
// pointing update and reused for every sample of every chunk (Section 2.1).
//
// Tensor-core storage: each beam owns two operand rows of K = 2N real
// elements against voltages stored as interleaved (Re X, Im X) pairs:
//   re row: (Re W, -Im W) per antenna  -> row . x = Re(W X)
//   im row: (Im W,  Re W) per antenna  -> row . x = Im(W X)
// Within a 128-row tile (64 beams) rows are grouped by 32: beams 16g..16g+15
// take rows 32g..32g+15 (re) and 32g+16..32g+31 (im), so the two rows of a
// beam land in the same warp of the epilogue, 16 lanes apart.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <type_traits>

#include "bf_internal.h"

namespace bfi {

__global__ void k_delays(const double *__restrict__ pos, const double *__restrict__ dirs, int N, int B,
                         double f0, double df, double *__restrict__ tau, unsigned long long *__restrict__ ab)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * B) return;
    int b = i / N, n = i % N;
    double rs = pos[3 * n] * dirs[3 * b] + pos[3 * n + 1] * dirs[3 * b + 1] + pos[3 * n + 2] * dirs[3 * b + 2];
    double t = rs / kC0;
    tau[i] = t;
    // fractional cycles as 64-bit fixed point (2^64 = one cycle)
    const double two64 = 18446744073709551616.0;
    double a = f0 * t, d = df * t;
    a -= floor(a);
    d -= floor(d);
    ab[2 * i] = __double2ull_rz(a * two64);
    ab[2 * i + 1] = __double2ull_rz(d * two64);
}

// Phase source of one channel: per-weight FP64 (any channel list) or the
// fixed-point recurrence (uniform channels).
template <bool FIXED>
struct Phase {
    const double *tau;
    const unsigned long long *ab;
    double f;
    unsigned long long c;
    int N;

    // twice the reduced phase, in [-1, 1], rounded to FP32
    __device__ __forceinline__ float x32(int b, int n) const
    {
        if (FIXED) {
            const size_t i = (size_t)b * N + n;
            const unsigned long long ph = ab[2 * i] + c * ab[2 * i + 1];   // modulo 2^64
            // top 32 bits as a signed value times 2^-31, without an integer
            // conversion instruction: the two 16-bit halves become floats
            // exactly through the 1.5 * 2^23 bias, and one FMA rounds once
            const int hi = (int)(ph >> 32);
            const float m = 12582912.0f;
            const float h16 = __int_as_float(0x4B400000 + (hi >> 16)) - m;        // exact, signed
            const float l16 = __int_as_float(0x4B400000 + (hi & 0xFFFF)) - m;     // exact, 0..65535
            return __fmaf_rn(h16, 3.0517578125e-05f, l16 * 4.656612873077393e-10f);  // 2^-15, 2^-31
        }
        double ph = f * tau[(size_t)b * N + n];   // cycles
        double r = ph - rint(ph);                 // [-1/2, 1/2]
        return static_cast<float>(2.0 * r);
    }
    __device__ __forceinline__ double x64(int b, int n) const
    {
        if (FIXED) {
            const size_t i = (size_t)b * N + n;
            const unsigned long long ph = ab[2 * i] + c * ab[2 * i + 1];
            return (double)(long long)ph * 1.0842021724855044e-19;        // x 2^-63
        }
        double ph = f * tau[(size_t)b * N + n];
        return 2.0 * (ph - rint(ph));
    }
};

template <bool FIXED>
__device__ __forceinline__ float2 weight_at(const Phase<FIXED> &ph, const uint8_t *mask, int b, int n, int N, int B)
{
    if (b >= B || n >= N || (mask && !mask[n])) return make_float2(0.f, 0.f);
    float s, c;
    sincospif(ph.x32(b, n), &s, &c);
    return make_float2(c, -s);   // exp(-i 2 pi phase)
}

// The same weight with sin/cos in FP64 (used only near rounding boundaries).
template <bool FIXED>
__device__ __forceinline__ double2 weight_at64(const Phase<FIXED> &ph, const uint8_t *mask, int b, int n, int N,
                                               int B)
{
    if (b >= B || n >= N || (mask && !mask[n])) return make_double2(0.0, 0.0);
    double s, c;
    sincospi(ph.x64(b, n), &s, &c);
    return make_double2(c, -s);
}

// Storage formats of the tensor-core weight rows.  Every format rounds to
// nearest, ties to even; FP8 saturates; the int8 reading keeps integers
// |q| <= 127 (exact in FP16).
enum { kFmtSimt = 0, kFmtF16 = 1, kFmtBF16 = 2, kFmtE4M3 = 3, kFmtI8 = 4 };

template <int FMT>
struct Quant;
template <>
struct Quant<kFmtF16> {
    using T = uint16_t;
    static constexpr float qmax = 0.f;
    static constexpr T mag = 0x7FFF;
    __device__ static T q(double x) { return __half_as_ushort(__double2half(x)); }
    __device__ static uint32_t q2(float a, float b)
    {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
};
template <>
struct Quant<kFmtBF16> {
    using T = uint16_t;
    static constexpr float qmax = 0.f;
    static constexpr T mag = 0x7FFF;
    __device__ static T q(double x) { return __bfloat16_as_ushort(__double2bfloat16(x)); }
    __device__ static uint32_t q2(float a, float b)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
};
template <>
struct Quant<kFmtE4M3> {
    using T = uint8_t;
    static constexpr float qmax = 448.f;
    static constexpr T mag = 0x7F;
    __device__ static T q(double x) { return (T)__nv_cvt_double_to_fp8(x, __NV_SATFINITE, __NV_E4M3); }
    __device__ static uint16_t q2(float a, float b)
    {
        return (uint16_t)__nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    }
};
template <>
struct Quant<kFmtI8> {
    using T = uint16_t;   // stored as FP16 integers
    static constexpr float qmax = 127.f;
    static constexpr T mag = 0x7FFF;
    __device__ static T q(double x) { return __half_as_ushort(__double2half(fmin(fmax(rint(x), -127.0), 127.0))); }
    // round to the nearest integer, ties to even, with two FP32 adds
    // (exact for |x| < 2^22), clip, then pack to FP16 (exact for integers)
    __device__ static float rnd(float x)
    {
        const float m = 12582912.0f;   // 1.5 * 2^23
        return fminf(fmaxf(__fsub_rn(__fadd_rn(x, m), m), -127.f), 127.f);
    }
    __device__ static uint32_t q2(float a, float b)
    {
        __half2 h = __floats2half2_rn(rnd(a), rnd(b));
        return *reinterpret_cast<uint32_t *>(&h);
    }
};

// Do the two codes packed in `pair` (low, high) store the same value?
// (+0 and -0 count as equal)
template <class Q>
__device__ __forceinline__ bool pair_same(uint32_t pair)
{
    constexpr int bits = 8 * sizeof(typename Q::T);
    constexpr uint32_t one = (1u << bits) - 1u;
    const uint32_t a = pair & one, b = (pair >> bits) & one;
    return a == b || ((a & Q::mag) == 0 && (b & Q::mag) == 0);
}

// One warp per (channel, beam slot).
template <bool FIXED>
__global__ void k_weights_simt(const double *__restrict__ freqs, const double *__restrict__ tau,
                               const unsigned long long *__restrict__ ab, const uint8_t *__restrict__ mask, int N,
                               int B, int b_pad, float2 *__restrict__ w, float *__restrict__ wscale,
                               float *__restrict__ wsig)
{
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int c = blockIdx.y;
    if (b >= b_pad) return;
    const Phase<FIXED> ph{tau, ab, freqs[c], (unsigned long long)c, N};
    if (lane == 0) {
        wscale[(size_t)c * b_pad + b] = 1.f;
        wsig[(size_t)c * b_pad + b] = 1.f;
    }
    float2 *row = w + ((size_t)c * b_pad + b) * N;
    for (int n = lane; n < N; n += 32) row[n] = weight_at(ph, mask, b, n, N, B);
}

// Tensor-core rows.  Each stored component is first rounded from the FP32
// weight; when that value lies within the FP32 error (4e-7, in weight units)
// of a rounding boundary of the format, the component (unscaled formats) or
// the whole beam (scaled formats, whose scale depends on every antenna) is
// recomputed in FP64 and rounded once from double, so the stored value is
// the format's rounding of the exact weight.
template <int FMT, bool FIXED>
__global__ void k_weights_tc(const double *__restrict__ freqs, const double *__restrict__ tau,
                             const unsigned long long *__restrict__ ab, const uint8_t *__restrict__ mask, int N,
                             int B, int b_pad, int k_pad, void *__restrict__ w, float *__restrict__ wscale,
                             float *__restrict__ wsig)
{
    using Q = Quant<FMT>;
    using T = typename Q::T;
    constexpr bool scaled = Q::qmax > 0.f;
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int c = blockIdx.y;
    if (b >= b_pad) return;
    const Phase<FIXED> ph{tau, ab, freqs[c], (unsigned long long)c, N};
    const int n_cols = k_pad / 2;

    float sig = 1.f;
    if (scaled) {
        float mx = 0.f;
        for (int n = lane; n < N; n += 32) {
            float2 v = weight_at(ph, mask, b, n, N, B);
            mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (mx > 0.f) sig = mx / Q::qmax;
    }
    const float delta = 4e-7f / sig;   // FP32 weight error bound in stored units

    const int mt = b / kBeamsPerMTile, bi = b % kBeamsPerMTile;
    const int row_re = mt * kRowsPerMTile + (bi >> 4) * 32 + (bi & 15);
    const size_t m_pad = (size_t)(b_pad / kBeamsPerMTile) * kRowsPerMTile;
    T *p_re = reinterpret_cast<T *>(w) + ((size_t)c * m_pad + row_re) * k_pad;
    T *p_im = p_re + (size_t)16 * k_pad;   // the im row sits 16 rows below
    // re row: (Re W, -Im W); im row: (Im W, Re W) -- one packed conversion and
    // one store per row pair (packed conversions run on the FP32 pipes)
    using T2 = typename std::conditional<sizeof(T) == 2, uint32_t, uint16_t>::type;
    auto put = [&](int n, T qre, T qim, T qim_neg) {
        reinterpret_cast<T2 *>(p_re)[n] = (T2)qre | ((T2)qim_neg << (8 * sizeof(T)));
        reinterpret_cast<T2 *>(p_im)[n] = (T2)qim | ((T2)qre << (8 * sizeof(T)));
    };
    bool redo = false;
    uint32_t near_bits = 0;   // antennas lane + 32k of this lane near a boundary (k < 32)
    for (int n = lane, k = 0; n < n_cols; n += 32, ++k) {
        float2 v = weight_at(ph, mask, b, n, N, B);
        if (v.x == 0.f && v.y == 0.f) {   // masked antenna, padding beam or padding column
            put(n, T(0), T(0), T(0));
            continue;
        }
        float re = v.x, im = v.y;
        if (scaled) {
            re /= sig;
            im /= sig;
        }
        const float dre = delta + 4e-7f * fabsf(re), dim = delta + 4e-7f * fabsf(im);
        const bool near = !pair_same<Q>(Q::q2(re - dre, re + dre)) || !pair_same<Q>(Q::q2(im - dim, im + dim));
        reinterpret_cast<T2 *>(p_re)[n] = (T2)Q::q2(re, -im);
        reinterpret_cast<T2 *>(p_im)[n] = (T2)Q::q2(im, re);
        if (near) near_bits |= 1u << (k & 31);
        redo |= near;
    }
    // FP64 recomputation of the few components near a boundary, in a separate
    // warp-uniform pass so the FP64 code is branched around, not predicated
    if (!scaled && __any_sync(0xffffffffu, near_bits != 0)) {
        for (int n = lane, k = 0; n < n_cols; n += 32, ++k)
            if (near_bits & (1u << (k & 31))) {
                double2 d = weight_at64(ph, mask, b, n, N, B);
                put(n, Q::q(d.x), Q::q(d.y), Q::q(-d.y));
            }
    }
    if (scaled && __any_sync(0xffffffffu, redo)) {
        double mx = 0.0;
        for (int n = lane; n < N; n += 32) {
            double2 d = weight_at64(ph, mask, b, n, N, B);
            mx = fmax(mx, fmax(fabs(d.x), fabs(d.y)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const double sig64 = mx > 0.0 ? mx / (double)Q::qmax : 1.0;
        for (int n = lane; n < n_cols; n += 32) {
            double2 d = weight_at64(ph, mask, b, n, N, B);
            const double re = d.x / sig64, im = d.y / sig64;
            put(n, Q::q(re), Q::q(im), Q::q(-im));
        }
        sig = (float)sig64;
    }
    if (lane == 0) {
        wscale[(size_t)c * b_pad + b] = sig * sig;
        wsig[(size_t)c * b_pad + b] = sig;
    }
}

// Decode the stored weights back to complex float32 [C][B][N] (without scale).
template <int FMT>
__global__ void k_export(const void *__restrict__ w, const float *__restrict__ wsig, int C, int N, int B,
                         int b_pad, int k_pad, float *__restrict__ out, float *__restrict__ scale)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)C * B * N;
    if (i >= total) return;
    int n = (int)(i % N);
    int b = (int)((i / N) % B);
    int c = (int)(i / ((size_t)N * B));
    float2 v;
    if (FMT == 0) {
        v = reinterpret_cast<const float2 *>(w)[((size_t)c * b_pad + b) * N + n];
    } else {
        const int mt = b / kBeamsPerMTile, bi = b % kBeamsPerMTile;
        const int row_re = mt * kRowsPerMTile + (bi >> 4) * 32 + (bi & 15);
        const size_t m_pad = (size_t)(b_pad / kBeamsPerMTile) * kRowsPerMTile;
        const size_t e = ((size_t)c * m_pad + row_re) * k_pad + 2 * n;
        float a0, a1;
        if (FMT == kFmtF16 || FMT == kFmtI8) {
            __half2 h = reinterpret_cast<const __half2 *>(w)[e / 2];
            a0 = __low2float(h);
            a1 = __high2float(h);
        } else if (FMT == kFmtBF16) {
            __nv_bfloat162 h = reinterpret_cast<const __nv_bfloat162 *>(w)[e / 2];
            a0 = __low2float(h);
            a1 = __high2float(h);
        } else {
            const __nv_fp8_storage_t *p = reinterpret_cast<const __nv_fp8_storage_t *>(w);
            a0 = __half2float(__half(__nv_cvt_fp8_to_halfraw(p[e], __NV_E4M3)));
            a1 = __half2float(__half(__nv_cvt_fp8_to_halfraw(p[e + 1], __NV_E4M3)));
        }
        v = make_float2(a0, -a1);
    }
    out[2 * i] = v.x;
    out[2 * i + 1] = v.y;
    if (scale && n == 0) scale[(size_t)c * B + b] = wsig[(size_t)c * b_pad + b];
}

static int fmt_code(const bf_plan *p)
{
    if (p->wf.simt) return kFmtSimt;
    if (p->wf.op == kOpBF16) return kFmtBF16;
    if (p->wf.op == kOpE4M3) return kFmtE4M3;
    if (p->wf.qmax == 127.f) return kFmtI8;
    return kFmtF16;
}

cudaError_t launch_delays(bf_plan *p, cudaStream_t s)
{
    int total = p->N * p->B;
    k_delays<<<(total + 255) / 256, 256, 0, s>>>(p->d_pos, p->d_dirs, p->N, p->B, p->f0, p->df, p->d_tau,
                                                 p->d_ab);
    return cudaGetLastError();
}

template <bool FIXED>
static void weights_launch(bf_plan *p, cudaStream_t s)
{
    dim3 grid((p->wf.b_pad + 7) / 8, p->C);
    const WeightFormat &f = p->wf;
#define BF_W_LAUNCH(F)                                                                                      \
    k_weights_tc<F, FIXED><<<grid, 256, 0, s>>>(p->d_freqs, p->d_tau, p->d_ab, p->d_mask, p->N, p->B, f.b_pad, \
                                                f.k_pad, p->d_w, p->d_wscale, p->d_wsig)
    switch (fmt_code(p)) {
    case kFmtSimt:
        k_weights_simt<FIXED><<<grid, 256, 0, s>>>(p->d_freqs, p->d_tau, p->d_ab, p->d_mask, p->N, p->B,
                                                   f.b_pad, (float2 *)p->d_w, p->d_wscale, p->d_wsig);
        break;
    case kFmtF16: BF_W_LAUNCH(kFmtF16); break;
    case kFmtBF16: BF_W_LAUNCH(kFmtBF16); break;
    case kFmtE4M3: BF_W_LAUNCH(kFmtE4M3); break;
    default: BF_W_LAUNCH(kFmtI8); break;
    }
#undef BF_W_LAUNCH
}

cudaError_t launch_weights(bf_plan *p, cudaStream_t s)
{
    if (p->uniform_freqs) weights_launch<true>(p, s);
    else weights_launch<false>(p, s);
    return cudaGetLastError();
}

cudaError_t launch_export_weights(bf_plan *p, float *d_w, float *d_scale, cudaStream_t s)
{
    size_t total = (size_t)p->C * p->B * p->N;
    unsigned blocks = (unsigned)((total + 255) / 256);
    const WeightFormat &f = p->wf;
#define BF_E_LAUNCH(F)                                                                                       \
    k_export<F><<<blocks, 256, 0, s>>>(p->d_w, p->d_wsig, p->C, p->N, p->B, f.b_pad, f.k_pad, d_w, d_scale)
    switch (fmt_code(p)) {
    case kFmtSimt: BF_E_LAUNCH(kFmtSimt); break;
    case kFmtF16: BF_E_LAUNCH(kFmtF16); break;
    case kFmtBF16: BF_E_LAUNCH(kFmtBF16); break;
    case kFmtE4M3: BF_E_LAUNCH(kFmtE4M3); break;
    default: BF_E_LAUNCH(kFmtI8); break;
    }
#undef BF_E_LAUNCH
    return cudaGetLastError();
}

}  // namespace bfi
