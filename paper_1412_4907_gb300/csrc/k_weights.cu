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
        if (mx > 0.f) sig = mx / (Q::qmax > 0.f ? Q::qmax : 1.f);
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
        const double sig64 = mx > 0.0 ? mx / (double)(Q::qmax > 0.f ? Q::qmax : 1.f) : 1.0;
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

// ---------------------------------------------------------------------------
// Channel-looping weight kernel.  One thread per (beam, antenna column); a
// block covers whole beams (32..256 threads per beam, up to two columns per
// thread) and a run of channels.  On the fixed-point path the phase of each
// (beam, antenna) advances by one exact 64-bit addition per channel, so the
// per-(beam, antenna) table is read once per run of channels.  The reduced
// phase is split into a 23-bit head (exact in FP32) and a 23-bit tail, and
// the tail is applied as a first-order correction after sincospif, so the
// FP32 weight is accurate to a few ulps relative to each component; the
// near-boundary test then uses a relative window (1e-6) and the FP64
// recomputation is rare.
struct WGeom {
    int N, B, b_pad, k_pad, n_cols;   // n_cols: stored antenna columns (K_pad / 2 or N)
    int tpb, bpb, apt, cc;            // threads per beam, beams per block, columns per thread, channels per block
    long long m_pad;
};

// twice the reduced phase as head + tail (head exact, |tail| <= 2^-22)
__device__ __forceinline__ void split_fixed(unsigned long long ph, float &xh, float &xl)
{
    const long long sp = (long long)ph;
    const int t = (int)(sp >> 41);                          // [-2^22, 2^22)
    const unsigned u = (unsigned)(ph >> 18) & 0x7FFFFFu;   // next 23 bits
    xh = (__int_as_float(0x4B400000 + t) - 12582912.0f) * 2.384185791015625e-07f;   // x 2^-22
    xl = (__int_as_float(0x4B000000 | u) - 8388608.0f) * 2.842170943040401e-14f;    // x 2^-45
}

__device__ __forceinline__ void split_double(double x, float &xh, float &xl)
{
    xh = (float)x;
    xl = (float)(x - (double)xh);
}

// exp(-i pi (xh + xl)) to a few FP32 ulps per component
__device__ __forceinline__ float2 cis_neg(float xh, float xl)
{
    float s, c;
    sincospif(xh, &s, &c);
    const float d = 3.14159265358979f * xl;
    return make_float2(fmaf(-d, s, c), -fmaf(d, c, s));
}

__device__ __noinline__ double2 cis_neg64(double x)
{
    double s, c;
    sincospi(x, &s, &c);
    return make_double2(c, -s);
}

template <int FMT>
__device__ __forceinline__ void store_pair(void *w, const WGeom &g, int c, int b, int n, uint32_t qre_row,
                                           uint32_t qim_row)
{
    using T2 = typename std::conditional<FMT == kFmtE4M3, uint16_t, uint32_t>::type;
    const int mt = b / kBeamsPerMTile, bi = b % kBeamsPerMTile;
    const long long row_re = (long long)mt * kRowsPerMTile + (bi >> 4) * 32 + (bi & 15);
    T2 *base = reinterpret_cast<T2 *>(w);
    const long long e_re = (((long long)c * g.m_pad + row_re) * g.k_pad) / 2 + n;
    base[e_re] = (T2)qre_row;
    base[e_re + (long long)16 * g.k_pad / 2] = (T2)qim_row;
}

template <int FMT, bool FIXED>
__global__ void __launch_bounds__(256) k_weights2(const double *__restrict__ freqs, const double *__restrict__ tau,
                                                  const unsigned long long *__restrict__ ab,
                                                  const uint8_t *__restrict__ mask, WGeom g, int C,
                                                  void *__restrict__ w, float *__restrict__ wscale,
                                                  float *__restrict__ wsig)
{
    using Q = Quant<FMT>;
    constexpr bool scaled = Q::qmax > 0.f;
    __shared__ float red[8];
    __shared__ int vote[8];
    const int tid = threadIdx.x;
    const int bl = tid / g.tpb, lt = tid % g.tpb;
    const int warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.x * g.bpb + bl;
    const int c0 = blockIdx.y * g.cc, c1 = min(C, c0 + g.cc);
    const bool in_block = bl < g.bpb && b < g.b_pad;
    unsigned long long ph[2] = {0ull, 0ull}, dph[2] = {0ull, 0ull};
    bool live[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int n = lt + a * g.tpb;
        live[a] = in_block && a < g.apt && n < g.N && b < g.B && !(mask && !mask[n]);
        if (FIXED && live[a]) {
            const size_t i = (size_t)b * g.N + n;
            dph[a] = ab[2 * i + 1];
            ph[a] = ab[2 * i] + (unsigned long long)c0 * dph[a];
        }
    }
    for (int c = c0; c < c1; ++c) {
        float2 v[2];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            v[a] = make_float2(0.f, 0.f);
            if (live[a]) {
                float xh, xl;
                if (FIXED) split_fixed(ph[a], xh, xl);
                else {
                    const double p2 = freqs[c] * tau[(size_t)b * g.N + lt + a * g.tpb];
                    split_double(2.0 * (p2 - rint(p2)), xh, xl);
                }
                v[a] = cis_neg(xh, xl);
            }
        }
        float sig = 1.f;
        if (scaled) {
            float mx = 0.f;
#pragma unroll
            for (int a = 0; a < 2; ++a) mx = fmaxf(mx, fmaxf(fabsf(v[a].x), fabsf(v[a].y)));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (g.tpb > 32) {   // beams span several warps
                if (lane == 0) red[warp] = mx;
                __syncthreads();
                const int w0 = (bl * g.tpb) >> 5, nw = g.tpb >> 5;
                for (int k = 0; k < nw; ++k) mx = fmaxf(mx, red[w0 + k]);
                __syncthreads();
            }
            if (mx > 0.f) sig = mx / (Q::qmax > 0.f ? Q::qmax : 1.f);
        }
        // quantise, store, note components within the FP32 error of a boundary
        bool near_any = false;
        uint32_t near_bits = 0;
        if (in_block) {
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int n = lt + a * g.tpb;
                if (a >= g.apt || n >= g.n_cols) continue;
                float re = v[a].x, im = v[a].y;
                if (scaled) {
                    re /= sig;
                    im /= sig;
                }
                bool near = false;
                if (live[a]) {
                    const float dre = 1e-6f * fabsf(re) + 1e-12f, dim = 1e-6f * fabsf(im) + 1e-12f;
                    near = !pair_same<Q>(Q::q2(re - dre, re + dre)) || !pair_same<Q>(Q::q2(im - dim, im + dim));
                }
                store_pair<FMT>(w, g, c, b, n, Q::q2(re, -im), Q::q2(im, re));
                near_bits |= (uint32_t)near << a;
                near_any |= near;
            }
        }
        if (!scaled) {
            // unscaled formats: recompute just the flagged components in FP64
#pragma unroll
            for (int a = 0; a < 2; ++a)
                if (near_bits & (1u << a)) {
                    const int n = lt + a * g.tpb;
                    double x;
                    if (FIXED) {
                        x = (double)(long long)ph[a] * 1.0842021724855044e-19;   // x 2^-63
                    } else {
                        const double p2 = freqs[c] * tau[(size_t)b * g.N + n];
                        x = 2.0 * (p2 - rint(p2));
                    }
                    const double2 d = cis_neg64(x);
                    const uint32_t lo = Q::q(d.x), hi = Q::q(-d.y), lo2 = Q::q(d.y);
                    constexpr int sh = 8 * sizeof(typename Q::T);
                    store_pair<FMT>(w, g, c, b, n, lo | (hi << sh), lo2 | (lo << sh));
                }
        } else {
            // scaled formats: the scale depends on every antenna of the beam, so a
            // flagged beam is recomputed whole in FP64
            bool redo = __any_sync(0xffffffffu, near_any);
            if (g.tpb > 32) {
                if (lane == 0) vote[warp] = redo;
                __syncthreads();
                const int w0 = (bl * g.tpb) >> 5, nw = g.tpb >> 5;
                redo = false;
                for (int k = 0; k < nw; ++k) redo |= vote[w0 + k] != 0;
                __syncthreads();
            }
            if (redo) {   // uniform across the beam (and across the warp when tpb <= 32)
                double2 d[2];
                double mx = 0.0;
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    d[a] = make_double2(0.0, 0.0);
                    if (live[a]) {
                        double x;
                        if (FIXED) {
                            x = (double)(long long)ph[a] * 1.0842021724855044e-19;
                        } else {
                            const double p2 = freqs[c] * tau[(size_t)b * g.N + lt + a * g.tpb];
                            x = 2.0 * (p2 - rint(p2));
                        }
                        d[a] = cis_neg64(x);
                    }
                    mx = fmax(mx, fmax(fabs(d[a].x), fabs(d[a].y)));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                // tpb > 32 with a redo is handled below through shared memory
                __shared__ double redd[8];
                if (g.tpb > 32) {
                    if (lane == 0) redd[warp] = mx;
                    __syncwarp();
                }
                if (g.tpb > 32) {
                    // only warps of redo beams reach here; they synchronise among
                    // themselves through a named barrier of the beam's threads
                    asm volatile("bar.sync %0, %1;" ::"r"(1 + bl), "r"(g.tpb) : "memory");
                    const int w0 = (bl * g.tpb) >> 5, nw = g.tpb >> 5;
                    for (int k = 0; k < nw; ++k) mx = fmax(mx, redd[w0 + k]);
                    asm volatile("bar.sync %0, %1;" ::"r"(1 + bl), "r"(g.tpb) : "memory");
                }
                const double sig64 = mx > 0.0 ? mx / (double)(Q::qmax > 0.f ? Q::qmax : 1.f) : 1.0;
                if (in_block) {
#pragma unroll
                    for (int a = 0; a < 2; ++a) {
                        const int n = lt + a * g.tpb;
                        if (a >= g.apt || n >= g.n_cols) continue;
                        const double re = d[a].x / sig64, im = d[a].y / sig64;
                        const uint32_t qre = Q::q(re), qim = Q::q(im), qimn = Q::q(-im);
                        constexpr int sh = 8 * sizeof(typename Q::T);
                        store_pair<FMT>(w, g, c, b, n, qre | (qimn << sh), qim | (qre << sh));
                    }
                }
                sig = (float)sig64;
            }
        }
        if (in_block && lt == 0) {
            wscale[(size_t)c * g.b_pad + b] = sig * sig;
            wsig[(size_t)c * g.b_pad + b] = sig;
        }
#pragma unroll
        for (int a = 0; a < 2; ++a) ph[a] += dph[a];
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
static bool weights2_launch(bf_plan *p, cudaStream_t s)
{
    const WeightFormat &f = p->wf;
    if (f.simt) return false;
    WGeom g;
    g.N = p->N;
    g.B = p->B;
    g.b_pad = f.b_pad;
    g.k_pad = f.k_pad;
    g.n_cols = f.k_pad / 2;
    g.m_pad = f.m_pad;
    if (g.n_cols > 512) return false;
    g.tpb = g.n_cols <= 32 ? 32 : g.n_cols <= 64 ? 64 : g.n_cols <= 128 ? 128 : 256;
    // 128-thread blocks where a beam fits (5K registers a block), so a refresh
    // on a side stream can share SMs with a running beamformer launch
    const int wt = g.tpb <= 128 ? 128 : 256;
    g.bpb = wt / g.tpb;
    g.apt = (g.n_cols + g.tpb - 1) / g.tpb;
    const int beam_blocks = (g.b_pad + g.bpb - 1) / g.bpb;
    // enough blocks to fill the GPU a few times over, each running many channels
    const int target = 8 * p->num_sms * (2048 / wt);
    int chunks = std::max(1, std::min(p->C, (target + beam_blocks - 1) / beam_blocks));
    g.cc = (p->C + chunks - 1) / chunks;
    chunks = (p->C + g.cc - 1) / g.cc;
    dim3 grid(beam_blocks, chunks);
#define BF_W2(F) k_weights2<F, FIXED><<<grid, wt, 0, s>>>(p->d_freqs, p->d_tau, p->d_ab, p->d_mask, g, p->C, \
                                                           p->d_w, p->d_wscale, p->d_wsig)
    switch (fmt_code(p)) {
    case kFmtF16: BF_W2(kFmtF16); break;
    case kFmtBF16: BF_W2(kFmtBF16); break;
    case kFmtE4M3: BF_W2(kFmtE4M3); break;
    default: BF_W2(kFmtI8); break;
    }
#undef BF_W2
    return true;
}

template <bool FIXED>
static void weights_launch(bf_plan *p, cudaStream_t s)
{
    if (weights2_launch<FIXED>(p, s)) return;
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
