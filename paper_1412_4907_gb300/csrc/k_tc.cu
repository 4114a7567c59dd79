// Tensor-core beamformer (tcgen05 + TMEM + TMA) with fused power detection
// and time integration.
//
// Per channel the beams are a complex matrix product (Section 2.1): beams
// (B x N complex weights) times voltages (N x T complex samples).  It runs as
// one real GEMM with K = 2N: each beam contributes a "re" and an "im" weight
// row (see k_weights.cu) against the interleaved (Re X, Im X) sample rows,
// so D[row][t] holds Re B or Im B, computed in FP32 from FP16/BF16/FP8
// operands.  The epilogue forms |B|^2 = D_re^2 + D_im^2 and sums it over each
// integration window, so only integrated powers reach HBM (the fusion of
// Section 2.1); the per-beam weight scale of the FP8/int8 modes is applied
// there.
//
// Structure (one CTA per SM, persistent):
//   warp 0      TMA producer: voltage tiles [NT samples x K] double-buffered,
//               and the weight rows of a group of M tiles kept resident in
//               shared memory while the CTA walks along time (weights are
//               reused for every sample, Section 2.1)
//   warp 1      allocates 512 TMEM columns; one thread issues tcgen05.mma,
//               128 x NT x 16 (or x32 for FP8) per instruction, into two
//               NT-column FP32 accumulators (the epilogue drains one while
//               the next tile accumulates)
//   warps 2-9   epilogue: tcgen05.ld of the accumulator, squares, window
//               sums in a fixed order, re+im combination via one shuffle
//               (the two rows of a beam are 16 lanes apart), store.
// Work unit = (channel, M-tile group, time tile); each CTA takes a
// contiguous, equal share of units, so consecutive units share a channel and
// group and the resident weights are reloaded only when they change.
// Every wait is bounded (2 s); a timeout raises the plan's error word, all
// roles leave their loops, in-flight copies and MMAs are drained and TMEM is
// freed before the CTA exits.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "bf_internal.h"
#include "ptx.cuh"

namespace bfi {

constexpr int kTcThreads = 320;
constexpr int kEpiWarps = 8;
constexpr int kTmemCols = 512;
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s

struct TcKernelArgs {
    long long units;
    int n_groups, g_base, g_rem, gmax;
    int t_tiles, nt, kb, ke, nsplit;
    int c_base, c_total, T, T_o, t_int, B, b_pad;
    uint32_t idesc;
    uint32_t x_stage_bytes, w_slot_bytes;
    const float *wscale;   // [C][b_pad] sigma^2
    const float *wsig;     // [C][b_pad] sigma
    float *out;
    unsigned *err;
};

struct Unit {
    int c, g, tt, m0, gs;
    long long cg;
};

__device__ __forceinline__ Unit decode_unit(const TcKernelArgs &a, long long u)
{
    Unit r;
    r.tt = (int)(u % a.t_tiles);
    long long q = u / a.t_tiles;
    r.g = (int)(q % a.n_groups);
    r.c = (int)(q / a.n_groups);
    r.cg = q;
    if (r.g < a.g_rem) {
        r.gs = a.g_base + 1;
        r.m0 = r.g * (a.g_base + 1);
    } else {
        r.gs = a.g_base;
        r.m0 = a.g_rem * (a.g_base + 1) + (r.g - a.g_rem) * a.g_base;
    }
    return r;
}

// Bounded wait that ignores the abort flag (used only to drain on abort).
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > 200000000ull) break;   // 0.2 s
}

template <bool F8, bool FASTWIN, bool COMPLEX>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap wmap, const TcKernelArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t sx = base;
    const uint32_t sw = sx + 2 * a.x_stage_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + 2 * a.x_stage_bytes + a.gmax * a.w_slot_bytes);
    const uint32_t b_xfull = smem_u32(bars + 0);
    const uint32_t b_xempty = smem_u32(bars + 2);
    const uint32_t b_tfull = smem_u32(bars + 4);
    const uint32_t b_tempty = smem_u32(bars + 6);
    const uint32_t b_drain = smem_u32(bars + 8);
    const uint32_t b_wfull = smem_u32(bars + 9);
    const uint32_t b_wempty = smem_u32(bars + 9 + a.gmax);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 9 + 2 * a.gmax);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(b_xfull + 8 * i, 1);
            mbar_init(b_xempty + 8 * i, 1);
            mbar_init(b_tfull + 8 * i, 1);
            mbar_init(b_tempty + 8 * i, kEpiWarps);
        }
        mbar_init(b_drain, 1);
        for (int s = 0; s < a.gmax; ++s) {
            mbar_init(b_wfull + 8 * s, 1);
            mbar_init(b_wempty + 8 * s, 1);
        }
        *abort_flag = 0;
        fence_mbar_init();
        prefetch_tensormap(&xmap);
        prefetch_tensormap(&wmap);
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_holder), kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    const long long u0 = a.units * blockIdx.x / gridDim.x;
    const long long u1 = a.units * (blockIdx.x + 1) / gridDim.x;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            uint32_t xcnt = 0, wcnt = 0, x_issued = 0, w_issued = 0;
            int xs = 0;
            long long prev = -1;
            for (long long u = u0; u < u1; ++u) {
                const Unit w = decode_unit(a, u);
                if (!mbar_wait(b_xempty + 8 * xs, ((xcnt >> xs) & 1u) ^ 1u, abort_flag, a.err, kWaitLimitNs))
                    break;
                xcnt ^= 1u << xs;
                x_issued |= 1u << xs;
                mbar_arrive_expect_tx(b_xfull + 8 * xs, a.x_stage_bytes);
                for (int kb = 0; kb < a.kb; ++kb)
                    tma_load_3d(sx + xs * a.x_stage_bytes + kb * a.nt * 128, &xmap, b_xfull + 8 * xs,
                                kb * a.ke, w.tt * a.nt, w.c);
                xs ^= 1;
                if (w.cg != prev) {
                    bool ok = true;
                    for (int s = 0; s < w.gs; ++s) {
                        if (!mbar_wait(b_wempty + 8 * s, ((wcnt >> s) & 1u) ^ 1u, abort_flag, a.err,
                                       kWaitLimitNs)) {
                            ok = false;
                            break;
                        }
                        wcnt ^= 1u << s;
                        w_issued |= 1u << s;
                        mbar_arrive_expect_tx(b_wfull + 8 * s, a.w_slot_bytes);
                        for (int kb = 0; kb < a.kb; ++kb)
                            tma_load_3d(sw + s * a.w_slot_bytes + kb * 16384, &wmap, b_wfull + 8 * s,
                                        kb * a.ke, (w.m0 + s) * kRowsPerMTile, a.c_base + w.c);
                    }
                    if (!ok) break;
                    prev = w.cg;
                }
            }
            if (*abort_flag) {   // let every issued copy land before the CTA exits
                for (int i = 0; i < 2; ++i)
                    if (x_issued & (1u << i)) drain_wait(b_xfull + 8 * i, ((xcnt >> i) & 1u) ^ 1u);
                for (int s = 0; s < a.gmax; ++s)
                    if (w_issued & (1u << s)) drain_wait(b_wfull + 8 * s, ((wcnt >> s) & 1u) ^ 1u);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ----------------------------------------------------------- MMA issuer
        if (lane == 0) {
            uint32_t xpar = 0, wpar = 0, tpar = 0;
            int xs = 0, acc = 0;
            long long prev = -1;
            const int ksteps = 4;   // 32-byte K steps per 128-byte block
            for (long long u = u0; u < u1; ++u) {
                const Unit w = decode_unit(a, u);
                const bool newg = w.cg != prev;
                prev = w.cg;
                const bool lastg = (u + 1 == u1) || decode_unit(a, u + 1).cg != w.cg;
                if (!mbar_wait(b_xfull + 8 * xs, (xpar >> xs) & 1u, abort_flag, a.err, kWaitLimitNs)) break;
                xpar ^= 1u << xs;
                bool ok = true;
                for (int s = 0; s < w.gs; ++s) {
                    if (newg) {
                        if (!mbar_wait(b_wfull + 8 * s, (wpar >> s) & 1u, abort_flag, a.err, kWaitLimitNs)) {
                            ok = false;
                            break;
                        }
                        wpar ^= 1u << s;
                    }
                    if (!mbar_wait(b_tempty + 8 * acc, ((tpar >> acc) & 1u) ^ 1u, abort_flag, a.err,
                                   kWaitLimitNs)) {
                        ok = false;
                        break;
                    }
                    tpar ^= 1u << acc;
                    tc_fence_after();
                    const uint32_t d = tmem + acc * a.nt;
                    for (int kb = 0; kb < a.kb; ++kb)
                        for (int ks = 0; ks < ksteps; ++ks) {
                            const uint64_t ad = sdesc_sw128(sw + s * a.w_slot_bytes + kb * 16384 + ks * 32);
                            const uint64_t bd = sdesc_sw128(sx + xs * a.x_stage_bytes + kb * a.nt * 128 + ks * 32);
                            if (F8) mma_f8(d, ad, bd, a.idesc, (kb | ks) != 0);
                            else mma_f16(d, ad, bd, a.idesc, (kb | ks) != 0);
                        }
                    mma_commit(b_tfull + 8 * acc);
                    if (lastg) mma_commit(b_wempty + 8 * s);
                    acc ^= 1;
                }
                if (!ok) break;
                mma_commit(b_xempty + 8 * xs);
                xs ^= 1;
            }
            mma_commit(b_drain);   // all issued MMAs complete before teardown
            drain_wait(b_drain, 0);
        }
        __syncwarp();
    } else {
        // -------------------------------------------------------------- epilogue
        const int e = warp - 2;
        const int q = warp & 3;               // TMEM lane quarter this warp may access
        const int h = e >> 2;                 // column half
        const int part = (lane >> 4) & 1;     // 0: re row, 1: im row
        const int bi = q * 16 + (lane & 15);  // beam within the M tile
        const int cols = a.nt / a.nsplit;
        const int col0 = h * cols;
        uint32_t tpar = 0;
        int acc = 0;
        for (long long u = u0; u < u1; ++u) {
            const Unit w = decode_unit(a, u);
            bool ok = true;
            for (int s = 0; s < w.gs; ++s) {
                if (!mbar_wait(b_tfull + 8 * acc, (tpar >> acc) & 1u, abort_flag, a.err, kWaitLimitNs)) {
                    ok = false;
                    break;
                }
                tpar ^= 1u << acc;
                tc_fence_after();
                if (h < a.nsplit) {
                    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + acc * a.nt + col0;
                    const int b = (w.m0 + s) * kBeamsPerMTile + bi;
                    const int cg = a.c_base + w.c;
                    const bool bvalid = b < a.B;
                    if (COMPLEX) {
                        const float sg = bvalid ? a.wsig[(size_t)cg * a.b_pad + b] : 0.f;
                        float2 *o2 = reinterpret_cast<float2 *>(a.out);
                        const size_t ob = ((size_t)b * a.c_total + cg) * a.T;
                        for (int ch = 0; ch < cols / 16; ++ch) {
                            float v[16], o[16];
                            tmem_ld16(taddr + ch * 16, v);
#pragma unroll
                            for (int i = 0; i < 16; ++i) o[i] = __shfl_xor_sync(0xffffffffu, v[i], 16);
                            const int t0 = w.tt * a.nt + col0 + ch * 16;
                            // lanes 0-15 hold the re row and store samples 0-7 of the
                            // chunk; lanes 16-31 hold the im row and store samples 8-15
                            if (bvalid && part == 0) {
#pragma unroll
                                for (int i = 0; i < 8; ++i)
                                    if (t0 + i < a.T) o2[ob + t0 + i] = make_float2(v[i] * sg, o[i] * sg);
                            } else if (bvalid) {
#pragma unroll
                                for (int i = 8; i < 16; ++i)
                                    if (t0 + i < a.T) o2[ob + t0 + i] = make_float2(o[i] * sg, v[i] * sg);
                            }
                        }
                    } else {
                        const float scale = bvalid ? a.wscale[(size_t)cg * a.b_pad + b] : 0.f;
                        const int nw = cols / a.t_int;
                        const int j_base = (w.tt * a.nt + col0) / a.t_int;
                        float *orow = a.out + ((size_t)b * a.c_total + cg) * a.T_o;
                        if (FASTWIN) {
                            const int nch = a.t_int / 16;
                            for (int wi = 0; wi < nw; ++wi) {
                                float ws = 0.f;
                                for (int ch = 0; ch < nch; ++ch) {
                                    float v[16];
                                    tmem_ld16(taddr + wi * a.t_int + ch * 16, v);
                                    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
                                    for (int i = 0; i < 16; i += 4) {
                                        s0 = fmaf(v[i], v[i], s0);
                                        s1 = fmaf(v[i + 1], v[i + 1], s1);
                                        s2 = fmaf(v[i + 2], v[i + 2], s2);
                                        s3 = fmaf(v[i + 3], v[i + 3], s3);
                                    }
                                    ws += (s0 + s1) + (s2 + s3);
                                }
                                const float pw = (ws + __shfl_xor_sync(0xffffffffu, ws, 16)) * scale;
                                const int j = j_base + wi;
                                const bool mine = (nw == 1) ? (part == 0) : ((wi & 1) == part);
                                if (mine && bvalid && j < a.T_o) orow[j] = pw;
                            }
                        } else {
                            float ws = 0.f;
                            int cnt = 0, wi = 0;
                            for (int ch = 0; ch < cols / 16; ++ch) {
                                float v[16];
                                tmem_ld16(taddr + ch * 16, v);
#pragma unroll
                                for (int i = 0; i < 16; ++i) {
                                    ws = fmaf(v[i], v[i], ws);
                                    if (++cnt == a.t_int) {
                                        const float pw = (ws + __shfl_xor_sync(0xffffffffu, ws, 16)) * scale;
                                        const int j = j_base + wi;
                                        const bool mine = (nw == 1) ? (part == 0) : ((wi & 1) == part);
                                        if (mine && bvalid && j < a.T_o) orow[j] = pw;
                                        ws = 0.f;
                                        cnt = 0;
                                        ++wi;
                                    }
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(b_tempty + 8 * acc);
                acc ^= 1;
            }
            if (!ok) break;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ----------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

static int gcd_i(int x, int y)
{
    while (y) {
        int t = x % y;
        x = y;
        y = t;
    }
    return x;
}

bool tc_choose(bf_plan *p, int tile_req, TcConfig *cfg, std::string *why)
{
    const WeightFormat &f = p->wf;
    const int t_int = p->t_int;
    const long long unit = 16LL / gcd_i(16, t_int) * t_int;   // lcm(16, T_int)
    if (unit > 256) {
        *why = "tensor-core kernel needs lcm(16, T_int) <= 256";
        return false;
    }
    const int mt = f.m_pad / kRowsPerMTile;
    for (int nt = 256; nt >= (int)unit; nt -= 16) {
        if (nt % unit) continue;
        if (tile_req && nt != tile_req) continue;
        TcConfig c;
        c.nt = nt;
        c.nsplit = ((nt / 2) % t_int == 0 && (nt / 2) % 16 == 0) ? 2 : 1;
        c.fast_windows = (t_int % 16) == 0;
        const int x_stage = f.kb * nt * 128;
        const int w_slot = f.kb * 16384;
        const int ctrl = 8 * (9 + 2 * 16) + 16;
        const int avail = kSmemLimit - 2 * x_stage - ctrl - 1024;
        if (avail < w_slot) continue;
        int g = std::min(mt, std::min(16, avail / w_slot));
        c.n_groups = (mt + g - 1) / g;
        const int g_base = mt / c.n_groups, g_rem = mt % c.n_groups;
        c.group = g_base + (g_rem ? 1 : 0);
        c.smem = 2 * x_stage + c.group * w_slot + ctrl + 1024;
        c.smem = std::max(c.smem, 116 * 1024);   // one CTA per SM: it owns all 512 TMEM columns
        *cfg = c;
        return true;
    }
    *why = tile_req ? "requested tile does not fit the tensor-core kernel"
                    : "antenna count too large for the resident-weight tensor-core kernel";
    return false;
}

template <bool F8, bool FW, bool CPX>
static cudaError_t launch_one(const CUtensorMap &xm, const CUtensorMap &wm, const TcKernelArgs &ka, int grid,
                              int smem, cudaStream_t s)
{
    auto kern = k_tc<F8, FW, CPX>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kTcThreads, smem, s>>>(xm, wm, ka);
    return cudaGetLastError();
}

cudaError_t launch_tc(bf_plan *p, const TcArgs &ta, cudaStream_t s, std::string *why)
{
    const WeightFormat &f = p->wf;
    const TcConfig &cfg = p->tc;
    auto enc = encode_fn();
    if (!enc) {
        *why = "cuTensorMapEncodeTiled unavailable";
        return cudaErrorNotSupported;
    }
    if (ta.T == 0 || ta.c_launch == 0) return cudaSuccess;
    const CUtensorMapDataType dt = f.es == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    CUtensorMap xm, wm;
    {
        cuuint64_t dims[3] = {(cuuint64_t)(2 * p->N), (cuuint64_t)ta.T, (cuuint64_t)ta.c_launch};
        cuuint64_t strides[2] = {(cuuint64_t)(2 * p->N * f.es), (cuuint64_t)ta.T * 2 * p->N * f.es};
        cuuint32_t box[3] = {(cuuint32_t)f.ke, (cuuint32_t)cfg.nt, 1};
        cuuint32_t es[3] = {1, 1, 1};
        CUresult r = enc(&xm, dt, 3, const_cast<void *>(ta.x), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            *why = "voltage tensor map rejected (pointer or row stride not 16-byte aligned?)";
            return cudaErrorInvalidValue;
        }
    }
    {
        cuuint64_t dims[3] = {(cuuint64_t)f.k_pad, (cuuint64_t)f.m_pad, (cuuint64_t)p->C};
        cuuint64_t strides[2] = {(cuuint64_t)f.k_pad * f.es, (cuuint64_t)f.m_pad * f.k_pad * f.es};
        cuuint32_t box[3] = {(cuuint32_t)f.ke, (cuuint32_t)kRowsPerMTile, 1};
        cuuint32_t es[3] = {1, 1, 1};
        CUresult r = enc(&wm, dt, 3, p->d_w, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            *why = "weight tensor map rejected";
            return cudaErrorInvalidValue;
        }
    }
    TcKernelArgs ka;
    const int mt = f.m_pad / kRowsPerMTile;
    ka.n_groups = cfg.n_groups;
    ka.g_base = mt / cfg.n_groups;
    ka.g_rem = mt % cfg.n_groups;
    ka.gmax = cfg.group;
    ka.t_tiles = (ta.T + cfg.nt - 1) / cfg.nt;
    ka.units = (long long)ta.c_launch * cfg.n_groups * ka.t_tiles;
    ka.nt = cfg.nt;
    ka.kb = f.kb;
    ka.ke = f.ke;
    ka.nsplit = cfg.nsplit;
    ka.c_base = ta.c_base;
    ka.c_total = ta.c_total;
    ka.T = ta.T;
    ka.T_o = ta.T_o;
    ka.t_int = ta.t_int;
    ka.B = p->B;
    ka.b_pad = f.b_pad;
    const uint32_t fmt = (f.op == kOpBF16) ? 1u : 0u;   // F16 = 0, BF16 = 1; E4M3 = 0 for f8f6f4
    ka.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(cfg.nt >> 3) << 17) |
               ((uint32_t)(kRowsPerMTile >> 4) << 24);
    ka.x_stage_bytes = (uint32_t)(f.kb * cfg.nt * 128);
    ka.w_slot_bytes = (uint32_t)(f.kb * 16384);
    ka.wscale = p->d_wscale;
    ka.wsig = p->d_wsig;
    ka.out = ta.out;
    ka.err = p->d_err;
    if (ka.units == 0) return cudaSuccess;
    const int grid = (int)std::min<long long>(p->num_sms, ka.units);
    const bool f8 = f.op == kOpE4M3;
    const bool fw = cfg.fast_windows;
    if (ta.complex_out) {
        if (f8) return launch_one<true, true, true>(xm, wm, ka, grid, cfg.smem, s);
        return launch_one<false, true, true>(xm, wm, ka, grid, cfg.smem, s);
    }
    if (f8) {
        if (fw) return launch_one<true, true, false>(xm, wm, ka, grid, cfg.smem, s);
        return launch_one<true, false, false>(xm, wm, ka, grid, cfg.smem, s);
    }
    if (fw) return launch_one<false, true, false>(xm, wm, ka, grid, cfg.smem, s);
    return launch_one<false, false, false>(xm, wm, ka, grid, cfg.smem, s);
}

}  // namespace bfi
