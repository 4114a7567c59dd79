// Pieces of the batched tensor-core kernel: constants, bounded drain wait,
// sums of squares, the per-tile epilogue (TMEM accumulator -> |B|^2 ->
// window powers staged in shared memory, or complex beams straight to HBM)
// and the store warp's per-tile write (with the carried integration window).
// The single-plan kernel (k_tc.cu) keeps the same steps inline: written as
// these shared functions it measured about 10% slower at 32 antennas.
#pragma once
#include <cudaTypedefs.h>

#include <cuda_fp16.h>

#include "bf_internal.h"
#include "ptx.cuh"
#include "tmap.h"

namespace bfi {

constexpr int kEpiWarps = 16;                      // two groups of 8 taking alternate tiles
constexpr int kStoreWarp = 2 + kEpiWarps;          // drains the staged window powers
constexpr int kTcThreads = (3 + kEpiWarps) * 32;
constexpr int kStageDepth = 4;                     // staged tiles in flight
constexpr int kTmemCols = 512;
constexpr int kMaxWinPerTile = 16;
constexpr int kMaxXStages = 8;
constexpr int kMaxAcc = 8;                         // TMEM accumulators (512 columns / tile)
constexpr uint64_t kWaitLimitCycles = 4000000000ull;   // SM cycles: about 2 s at the maximum clock

// Bounded wait that ignores the abort flag (used only to drain on abort).
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > 400000000ll) break;   // ~0.2 s
}

// Sum of squares of 16 values with four independent chains.
__device__ __forceinline__ float sumsq16(const float *v)
{
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
    for (int i = 0; i < 16; i += 4) {
        s0 = fmaf(v[i], v[i], s0);
        s1 = fmaf(v[i + 1], v[i + 1], s1);
        s2 = fmaf(v[i + 2], v[i + 2], s2);
        s3 = fmaf(v[i + 3], v[i + 3], s3);
    }
    return (s0 + s1) + (s2 + s3);
}

// Sum of squares of n (multiple of 8) raw FP32 values with packed FMAs in
// four independent chains, combined in a fixed order.
template <int n>
__device__ __forceinline__ float sumsq_pk(const uint32_t *r)
{
    unsigned long long acc[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
    for (int i = 0; i < n / 2; ++i) sq_acc2(acc[i & 3], r[2 * i], r[2 * i + 1]);
    return (sum2(acc[0]) + sum2(acc[1])) + (sum2(acc[2]) + sum2(acc[3]));
}

// ----------------------------------------------- 8- and 4-bit input widening
// Integer complex voltages are widened to the FP16 MMA operand in shared
// memory by converter warps, so the kernel reads each sample's 2 (int8) or
// 1 (4-bit) bytes from HBM once and nothing is written back (the unpacking
// of Section 2.1 done inside the beamformer).  Every value is exact in FP16.
//
// Bias trick, no integer-to-float instruction: a byte u in 0..255 placed as
// the low byte of the FP16 pattern 0x64uu is the number 1024 + u (FP16 has
// unit spacing in [1024, 2048)); so a signed 8-bit x becomes
// (1024 + (x ^ 0x80)) - 1152 = x, and a signed 4-bit v (nibble s, s ^ 8 =
// v + 8) becomes (1024 + (s ^ 8)) - 1032 = v; both subtractions are exact.
// One converter warp is added to the 19-warp kernels (an SM sub-partition's
// 16K registers hold five warps of 96 registers, so 20 warps is the most);
// where the store warp has no work it converts too.
constexpr int kConvWarps = 1;

// Four antennas of signed 8-bit (re, im) pairs (8 bytes) -> four FP16 pairs.
__device__ __forceinline__ uint4 widen_i8x4(uint2 w)
{
    const __half2 off = __float2half2_rn(1152.f);
    const uint32_t b0 = w.x ^ 0x80808080u, b1 = w.y ^ 0x80808080u;
    uint32_t r[4] = {__byte_perm(b0, 0x64646464u, 0x4140), __byte_perm(b0, 0x64646464u, 0x4342),
                     __byte_perm(b1, 0x64646464u, 0x4140), __byte_perm(b1, 0x64646464u, 0x4342)};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __half2 h = *reinterpret_cast<__half2 *>(&r[i]);
        h = __hsub2(h, off);
        r[i] = *reinterpret_cast<uint32_t *>(&h);
    }
    return make_uint4(r[0], r[1], r[2], r[3]);
}

// Four antennas of 4-bit pairs (one byte each: real part in the high nibble,
// two's complement) -> four FP16 pairs.
__device__ __forceinline__ uint4 widen_i4x4(uint32_t w)
{
    const __half2 off = __float2half2_rn(1032.f);
    const uint32_t hi = ((w >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;   // real parts, biased
    const uint32_t lo = (w & 0x0F0F0F0Fu) ^ 0x08080808u;          // imaginary parts, biased
    const uint32_t a01 = __byte_perm(hi, lo, 0x5140), a23 = __byte_perm(hi, lo, 0x7362);
    uint32_t r[4] = {__byte_perm(a01, 0x64646464u, 0x4140), __byte_perm(a01, 0x64646464u, 0x4342),
                     __byte_perm(a23, 0x64646464u, 0x4140), __byte_perm(a23, 0x64646464u, 0x4342)};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __half2 h = *reinterpret_cast<__half2 *>(&r[i]);
        h = __hsub2(h, off);
        r[i] = *reinterpret_cast<uint32_t *>(&h);
    }
    return make_uint4(r[0], r[1], r[2], r[3]);
}

// Widens one 128-byte K block of a voltage tile from its raw copy in shared
// memory (nt rows of RAW_KB bytes, as TMA lands them: out-of-range rows and
// antennas are zero bytes, which widen to 0) into nt swizzled FP16 rows of
// 128 bytes.  Each thread takes 16 raw bytes at a time: 8 antennas (int8) or
// 16 antennas (4-bit), i.e. 2 or 4 output chunks of 16 bytes.
template <int DT>
__device__ __forceinline__ void widen_block_smem(const uint8_t *raw, uint8_t *dst, int nt, int tid, int nthr)
{
    constexpr int kRawKb = DT == BF_CI8 ? 64 : 32;     // raw bytes per row of the K block
    constexpr int kPieces = kRawKb / 16;                // 16-byte raw pieces per row
    const int n_items = nt * kPieces;
    // four independent pieces per trip (loads first), so the byte permutes of
    // one piece overlap the loads and stores of the others
    for (int i0 = tid; i0 < n_items; i0 += 4 * nthr) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * nthr;
            if (i < n_items) v[u] = *reinterpret_cast<const uint4 *>(raw + (i / kPieces) * kRawKb + (i % kPieces) * 16);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * nthr;
            if (i >= n_items) break;
            const int row = i / kPieces, pc = i % kPieces;
            uint8_t *drow = dst + row * 128;
            const int sw = row & 7;
            if (DT == BF_CI8) {
                *reinterpret_cast<uint4 *>(drow + (((2 * pc) ^ sw) << 4)) = widen_i8x4(make_uint2(v[u].x, v[u].y));
                *reinterpret_cast<uint4 *>(drow + (((2 * pc + 1) ^ sw) << 4)) = widen_i8x4(make_uint2(v[u].z, v[u].w));
            } else {
                *reinterpret_cast<uint4 *>(drow + (((4 * pc) ^ sw) << 4)) = widen_i4x4(v[u].x);
                *reinterpret_cast<uint4 *>(drow + (((4 * pc + 1) ^ sw) << 4)) = widen_i4x4(v[u].y);
                *reinterpret_cast<uint4 *>(drow + (((4 * pc + 2) ^ sw) << 4)) = widen_i4x4(v[u].z);
                *reinterpret_cast<uint4 *>(drow + (((4 * pc + 3) ^ sw) << 4)) = widen_i4x4(v[u].w);
            }
        }
    }
}

// What the epilogue and the store warp need to know about the output of the
// batched job a tile belongs to (the functions are templates over it).
struct TileOut {
    int nt, nsplit, wpt, t_int, T, T_o, B, b_pad, c_total;
    const float *wscale;   // [C][b_pad] sigma^2, or NULL (unscaled)
    const float *wsig;     // [C][b_pad] sigma
    float *out;            // powers [B][C][T_o] or beams [B][C][T][2]
    const float *acc_in = nullptr;   // [B][C] partial sum added to window 0 (carried in)
    float *acc_out = nullptr;        // [B][C] receives window T_o, left open (carried out)
};

// Hand a TMEM accumulator back to the MMA issuer (after its loads completed).
__device__ __forceinline__ void tile_release(uint32_t b_tempty_acc, int lane)
{
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive_relaxed(b_tempty_acc);
}

// Power epilogue of one warp for one tile: read this warp's column slice of
// the accumulator (32 rows = 16 beams x re/im), release the accumulator, sum
// |B|^2 over each window in a fixed order, combine re and im rows with one
// shuffle, scale, and stage the window powers for the store warp.
// WIN: 16, 32 or 64 = T_int known at compile time; 0 = any multiple of 16;
// -1 = any T_int (per-column window counter).
template <int WIN, class O>
__device__ __forceinline__ void epi_power_tile(const O &o, uint32_t taddr, int cols, int h, int lane, int bq,
                                               int b, bool bvalid, int cg, float *stg, uint32_t b_tempty_acc,
                                               uint32_t b_sfull_sb)
{
    const int part = (lane >> 4) & 1;   // 0: re row, 1: im row
    const int wps = cols / o.t_int;     // windows per slice
    const float scale = bvalid ? (o.wscale ? o.wscale[(size_t)cg * o.b_pad + b] : 1.f) : 0.f;
    float ws = 0.f;
    int wi = 0, cnt = 0;
    auto emit = [&](float sum) {
        const float pw = (sum + __shfl_xor_sync(0xffffffffu, sum, 16)) * scale;
        if (part == 0) stg[bq * kMaxWinPerTile + h * wps + wi] = pw;
        ++wi;
    };
    auto add16 = [&](const float *v) {
        if (WIN >= 0) {
            ws += sumsq16(v);
            cnt += 16;
            if (cnt == o.t_int) {
                emit(ws);
                ws = 0.f;
                cnt = 0;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                ws = fmaf(v[i], v[i], ws);
                if (++cnt == o.t_int) {
                    emit(ws);
                    ws = 0.f;
                    cnt = 0;
                }
            }
        }
    };
    int col = 0;
    if (WIN > 0 && cols % 64 == 0) {
        // 64 columns per load (64 registers, leaving room for the walker state
        // of the batched kernel); the accumulator is released after the last
        // load, before the squares are summed
        for (; col < cols; col += 64) {
            uint32_t r[64];
            tmem_ld64r(taddr + col, r);
            if (col + 64 == cols) tile_release(b_tempty_acc, lane);
#pragma unroll
            for (int k = 0; k < 64 / (WIN > 0 ? WIN : 64); ++k)
                emit(sumsq_pk<(WIN > 0 ? WIN : 64)>(r + k * (WIN > 0 ? WIN : 64)));
        }
    }
    const int n64 = (cols - col) / 64, rem = (cols - col) % 64;   // rem is a multiple of 16
    for (int bt = 0; bt < n64; ++bt) {
        float v[64];
        tmem_ld64(taddr + col + bt * 64, v);
        if (bt == n64 - 1 && rem == 0) tile_release(b_tempty_acc, lane);
#pragma unroll
        for (int k = 0; k < 4; ++k) add16(v + 16 * k);
    }
    for (col += n64 * 64; col < cols; col += 16) {
        float v[16];
        tmem_ld16(taddr + col, v);
        if (col + 16 == cols) tile_release(b_tempty_acc, lane);
        add16(v);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(b_sfull_sb);   // publishes the staged windows
}

// Complex-beam epilogue of one warp for one tile: beams straight to HBM.
template <class O>
__device__ __forceinline__ void epi_complex_tile(const O &o, uint32_t taddr, int cols, int col0, int tt,
                                                 int lane, int b, bool bvalid, int cg)
{
    const int part = (lane >> 4) & 1;
    const float sg = bvalid ? o.wsig[(size_t)cg * o.b_pad + b] : 0.f;
    float2 *o2 = reinterpret_cast<float2 *>(o.out);
    const size_t ob = ((size_t)b * o.c_total + cg) * o.T;
    for (int ch = 0; ch < cols / 16; ++ch) {
        float v[16], x[16];
        tmem_ld16(taddr + ch * 16, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = __shfl_xor_sync(0xffffffffu, v[i], 16);
        const int t0 = tt * o.nt + col0 + ch * 16;
        // lanes 0-15 hold the re row and store samples 0-7 of the chunk;
        // lanes 16-31 hold the im row and store samples 8-15
        if (bvalid && part == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (t0 + i < o.T) o2[ob + t0 + i] = make_float2(v[i] * sg, x[i] * sg);
        } else if (bvalid) {
#pragma unroll
            for (int i = 8; i < 16; ++i)
                if (t0 + i < o.T) o2[ob + t0 + i] = make_float2(x[i] * sg, v[i] * sg);
        }
    }
}

// The store warp's write of one staged tile: one run of windows per beam.
// With a carried integration, window 0 first takes the partial sum that the
// previous chunk left, and window T_o (open at the end of this chunk) goes to
// acc_out instead of the output.
template <class O>
__device__ __forceinline__ void store_tile(const O &o, float *stg, int b_tile0, int cg, int tt, int lane)
{
    const int j0 = tt * o.wpt;
    if (o.acc_in && j0 == 0) {
        for (int bl = lane; bl < kBeamsPerMTile; bl += 32) {
            const int bb = b_tile0 + bl;
            if (bb < o.B) stg[bl * kMaxWinPerTile] += o.acc_in[(size_t)bb * o.c_total + cg];
        }
        __syncwarp();
    }
    if (o.acc_out && o.T_o >= j0 && o.T_o < j0 + o.wpt) {
        const int k = o.T_o - j0;
        for (int bl = lane; bl < kBeamsPerMTile; bl += 32) {
            const int bb = b_tile0 + bl;
            if (bb < o.B) o.acc_out[(size_t)bb * o.c_total + cg] = stg[bl * kMaxWinPerTile + k];
        }
    }
    const bool vec = (o.T_o & 3) == 0 && (o.wpt & 3) == 0 && ((uintptr_t)o.out & 15) == 0;
    const int nj = min(o.wpt, o.T_o - j0);
    if (vec && o.wpt == 4) {
        // one float4 per beam: lanes take beams lane and lane + 32
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int bl = lane + 32 * r;
            const int bb = b_tile0 + bl;
            if (bb < o.B && nj > 0) {
                const float4 v4 = *reinterpret_cast<const float4 *>(stg + bl * kMaxWinPerTile);
                *reinterpret_cast<float4 *>(o.out + ((size_t)bb * o.c_total + cg) * o.T_o + j0) = v4;
            }
        }
    } else if (vec) {
        const int per = o.wpt >> 2;
        for (int i = lane; i < kBeamsPerMTile * per; i += 32) {
            const int bl = i / per, k = (i % per) * 4;
            const int bb = b_tile0 + bl;
            if (bb < o.B && k < nj) {
                const float4 v4 = *reinterpret_cast<const float4 *>(stg + bl * kMaxWinPerTile + k);
                *reinterpret_cast<float4 *>(o.out + ((size_t)bb * o.c_total + cg) * o.T_o + j0 + k) = v4;
            }
        }
    } else {
        for (int i = lane; i < kBeamsPerMTile * o.wpt; i += 32) {
            const int bl = i / o.wpt, k = i % o.wpt;
            const int bb = b_tile0 + bl;
            if (bb < o.B && k < nj) o.out[((size_t)bb * o.c_total + cg) * o.T_o + j0 + k] = stg[bl * kMaxWinPerTile + k];
        }
    }
}

}  // namespace bfi
