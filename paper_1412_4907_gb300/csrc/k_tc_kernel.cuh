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
//   warp 0       TMA producer: voltage tiles [NT samples x K] double-buffered,
//                and the weight rows of a group of M tiles kept resident in
//                shared memory while the CTA walks along time (weights are
//                reused for every sample, Section 2.1)
//   warp 1       allocates 512 TMEM columns; one thread issues tcgen05.mma,
//                128 x NT x 16 (or x32 for FP8) per instruction, into two
//                NT-column FP32 accumulators (the epilogue drains one while
//                the next tile accumulates), stepping precomputed descriptor
//                words by one add per MMA
//   warps 2-17   epilogue in two groups of 8 that take alternate tiles (and
//                so alternate accumulators): while one group reads and sums a
//                tile the other is already waiting for the next, so the
//                accumulator's read-out and the squaring no longer sit in
//                series with the MMA of the tile after next.  In a group, two
//                warps per TMEM lane quarter, each on a half of the tile's
//                columns, read 64 columns at a time with tcgen05.ld and hand
//                the accumulator back to the MMA after the last load; squares
//                with packed FP32 FMAs, window sums in a fixed order, re+im
//                combination via one shuffle (the two rows of a beam are 16
//                lanes apart).  With 256-sample tiles and T_int of 16, 32 or
//                64 each warp stores its windows straight to the output
//                (direct path: nothing between the two loads but the squares
//                of the first); otherwise the window powers are staged in
//                shared memory for
//   warp 18      the store warp, which writes each staged tile as one run of
//                windows per beam (16-byte stores for 4 windows, 8-byte for
//                2), four tiles in flight.
// 19 warps: at most 96 registers a thread (five warps share an SM
// sub-partition's 16K registers).
// Work: the M tiles of a channel are split into weight groups; the CTAs are
// arranged as P sets of Gq CTAs, the CTAs of one set hold different groups
// and walk the same (channel, time-tile) range in step, so a voltage tile is
// read from DRAM once and served to the other group's CTA from L2.  Weights
// are reloaded only when the channel changes.
// Every wait is bounded (2 s); a timeout raises the plan's error word, all
// roles leave their loops, in-flight copies and MMAs are drained and TMEM is
// freed before the CTA exits.
#pragma once
#include <cudaTypedefs.h>

#include "k_tc.h"
#include "tc_common.cuh"

namespace bfi {

__device__ __forceinline__ void group_tiles(const TcKernelArgs &a, int g, int &m0, int &gs)
{
    if (g < a.g_rem) {
        gs = a.g_base + 1;
        m0 = g * (a.g_base + 1);
    } else {
        gs = a.g_base;
        m0 = a.g_rem * (a.g_base + 1) + (g - a.g_rem) * a.g_base;
    }
}

// WIN: 16, 32 or 64 = T_int known at compile time; 0 = any multiple of 16;
// -1 = any T_int (per-column window counter).
// Plans whose weights do not fit in shared memory (K >= 4 blocks) run the
// batched kernel's streamed pipeline instead (k_batch.cu).
// IN: BF_CI8 or BF_CI4 for integer inputs: the producer loads each raw tile
// by TMA (xmap is then the raw byte map) into one raw buffer, and a converter
// warp after the store warp (with DIRECT the idle store warp too) widens it
// into the next FP16 voltage stage and hands the buffer back; else 0
// (FP16/BF16/FP8 voltage tiles straight from TMA).
template <bool F8, int WIN, bool COMPLEX, bool DIRECT, int IN>
__global__ void __maxnreg__(96)
    k_tc(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap wmap, const TcKernelArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t sx = base;
    const uint32_t sw = sx + a.xst * a.x_stage_bytes;
    const uint32_t sr = sw + a.gmax * a.w_slot_bytes;   // the raw tile of integer inputs
    float *stage = reinterpret_cast<float *>(gbase + a.xst * a.x_stage_bytes + a.gmax * a.w_slot_bytes +
                                             a.raw_stage_bytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage + kStageDepth * kBeamsPerMTile * kMaxWinPerTile);
    const uint32_t b_xfull = smem_u32(bars + 0);                 // [kMaxXStages]
    const uint32_t b_xempty = smem_u32(bars + kMaxXStages);      // [kMaxXStages]
    const uint32_t b_tfull = smem_u32(bars + 2 * kMaxXStages);   // [kMaxAcc]
    const uint32_t b_tempty = b_tfull + 8 * kMaxAcc;              // [kMaxAcc]
    const uint32_t b_drain = b_tempty + 8 * kMaxAcc;
    const uint32_t b_wfull = b_drain + 8;                         // [gmax]
    const uint32_t b_wempty = b_wfull + 8 * a.gmax;               // [gmax]
    const uint32_t b_sfull = b_wempty + 8 * a.gmax;               // [stage]: every slice staged
    const uint32_t b_sempty = b_sfull + 8 * kStageDepth;          // [stage]: written out
    const uint32_t b_rfull = b_sempty + 8 * kStageDepth;          // raw tile landed
    const uint32_t b_rempty = b_rfull + 8;                        // raw tile widened
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 3 * kMaxXStages + 2 * kMaxAcc + 1 + 2 * a.gmax +
                                                         2 * kStageDepth);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // FP16/BF16/FP8 powers with the direct-store epilogue: the store warp has
    // nothing to store, so it issues the MMAs of every other tile (the second
    // accumulator) while warp 1 waits, commits and walks to its next tile.
    // Both issuers wait for every voltage stage and weight slot in order (so
    // neither runs a phase ahead of a barrier).  Integer inputs keep the store
    // warp as a second converter: with one converter 8-bit input lost 10%.
    constexpr bool TWO = DIRECT && IN == 0;
    constexpr unsigned kIssuers = TWO ? 2u : 1u;

    if (threadIdx.x == 0) {
        for (int i = 0; i < a.xst; ++i) {
            mbar_init(b_xfull + 8 * i, IN ? kConvWarps + (DIRECT ? 1 : 0) : 1);   // converters, or the TMA
            mbar_init(b_xempty + 8 * i, kIssuers);
        }
        mbar_init(b_rfull, 1);
        mbar_init(b_rempty, kConvWarps + (DIRECT ? 1 : 0));
        for (int i = 0; i < a.nacc; ++i) {
            mbar_init(b_tfull + 8 * i, 1);
            mbar_init(b_tempty + 8 * i, 8);   // the 8 warps of one group release each use
        }
        mbar_init(b_drain, kIssuers);
        for (int s = 0; s < a.gmax; ++s) {
            mbar_init(b_wfull + 8 * s, 1);
            mbar_init(b_wempty + 8 * s, kIssuers);
        }
        for (int i = 0; i < kStageDepth; ++i) {
            mbar_init(b_sfull + 8 * i, 4 * a.nsplit);   // the active epilogue warps
            mbar_init(b_sempty + 8 * i, 1);             // the store warp
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

    // this CTA: groups gq0, gq0 + gq, ...; (channel, time-tile) range of its set
    const int gq0 = blockIdx.x % a.gq;
    const int set = blockIdx.x / a.gq;
    const int n_sets = gridDim.x / a.gq;
    const long long ct0 = a.ct_total * set / n_sets;
    const long long ct1 = a.ct_total * (set + 1) / n_sets;
    const int c_first = (int)(ct0 / a.t_tiles), tt_first = (int)(ct0 % a.t_tiles);

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            uint32_t xcnt = 0, wcnt = 0, x_issued = 0, w_issued = 0, rcnt = 0;
            bool r_issued = false;
            int xs = 0;
            bool ok = true;
            for (int g = gq0; g < a.n_groups && ok; g += a.gq) {
                int m0, gs;
                group_tiles(a, g, m0, gs);
                int c = c_first, tt = tt_first;
                for (long long ct = ct0; ct < ct1; ++ct) {
                    if (IN) {   // the raw tile, once the converters have widened the last one
                        if (!mbar_wait(b_rempty, (rcnt & 1u) ^ 1u, abort_flag, a.err, kWaitLimitCycles)) {
                            ok = false;
                            break;
                        }
                        ++rcnt;
                        r_issued = true;
                        mbar_arrive_expect_tx(b_rfull, a.raw_stage_bytes);
                        for (int kb = 0; kb < a.kb; ++kb)
                            tma_load_3d(sr + kb * a.nt * a.raw_kb, &xmap, b_rfull, kb * a.raw_kb, tt * a.nt, c);
                    } else {
                        if (!mbar_wait(b_xempty + 8 * xs, ((xcnt >> xs) & 1u) ^ 1u, abort_flag, a.err,
                                       kWaitLimitCycles)) {
                            ok = false;
                            break;
                        }
                        xcnt ^= 1u << xs;
                        x_issued |= 1u << xs;
                        mbar_arrive_expect_tx(b_xfull + 8 * xs, a.x_stage_bytes);
                        for (int kb = 0; kb < a.kb; ++kb)
                            tma_load_3d(sx + xs * a.x_stage_bytes + kb * a.nt * 128, &xmap, b_xfull + 8 * xs,
                                        kb * a.ke, tt * a.nt, c);
                        if (++xs == a.xst) xs = 0;
                    }
                    if (ct == ct0 || tt == 0) {   // weights of (group, channel)
                        for (int s = 0; s < gs; ++s) {
                            if (!mbar_wait(b_wempty + 8 * s, ((wcnt >> s) & 1u) ^ 1u, abort_flag, a.err,
                                           kWaitLimitCycles)) {
                                ok = false;
                                break;
                            }
                            wcnt ^= 1u << s;
                            w_issued |= 1u << s;
                            mbar_arrive_expect_tx(b_wfull + 8 * s, a.w_slot_bytes);
                            for (int kb = 0; kb < a.kb; ++kb)
                                tma_load_3d(sw + s * a.w_slot_bytes + kb * 16384, &wmap, b_wfull + 8 * s,
                                            kb * a.ke, (m0 + s) * kRowsPerMTile, a.c_base + c);
                        }
                        if (!ok) break;
                    }
                    if (++tt == a.t_tiles) {
                        tt = 0;
                        ++c;
                    }
                }
            }
            if (*abort_flag) {   // let every issued copy land before the CTA exits
                for (int i = 0; i < a.xst; ++i)
                    if (x_issued & (1u << i)) drain_wait(b_xfull + 8 * i, ((xcnt >> i) & 1u) ^ 1u);
                if (r_issued) drain_wait(b_rfull, (rcnt - 1) & 1u);
                for (int s = 0; s < a.gmax; ++s)
                    if (w_issued & (1u << s)) drain_wait(b_wfull + 8 * s, ((wcnt >> s) & 1u) ^ 1u);
            }
        }
        __syncwarp();
    } else if (warp == 1 || (TWO && warp == kStoreWarp)) {
        // ---------------------------------------------------------- MMA issuers
        // one issuing thread, or two taking alternate tiles: each waits for
        // every voltage stage and weight slot, issues its own tiles, and
        // commits the stage and slot releases (barriers counting kIssuers)
        if (lane == 0) {
            const uint32_t par = warp == 1 ? 0u : 1u;
            uint32_t xpar = 0, wpar = 0, tpar = 0, kt = 0;
            int xs = 0, acc = 0;
            bool ok = true;
            // Descriptor words of the first weight slot and the first voltage stage;
            // every operand address below is an offset from these, added to the low
            // word (shared memory is below 256 KB, so the 14-bit start-address field
            // never carries).  Building each 64-bit descriptor anew made the issue of
            // one tcgen05.mma cost ~75-90 cycles; with one add it is ~50.
            const uint64_t w_desc0 = sdesc_sw128(sw), x_desc0 = sdesc_sw128(sx);
            const uint32_t w_hi = (uint32_t)(w_desc0 >> 32), x_hi = (uint32_t)(x_desc0 >> 32);
            const uint32_t w_lo0 = (uint32_t)w_desc0, x_lo0 = (uint32_t)x_desc0;
            const uint32_t w_slot16 = a.w_slot_bytes >> 4, x_stage16 = a.x_stage_bytes >> 4;
            const uint32_t x_kb16 = (uint32_t)(a.nt * 128) >> 4;
            for (int g = gq0; g < a.n_groups && ok; g += a.gq) {
                int m0, gs;
                group_tiles(a, g, m0, gs);
                (void)m0;
                int tt = tt_first;
                for (long long ct = ct0; ct < ct1 && ok; ++ct) {
                    const bool neww = (ct == ct0) || tt == 0;
                    const bool lastw = (ct + 1 == ct1) || tt + 1 == a.t_tiles;
                    if (!mbar_wait(b_xfull + 8 * xs, (xpar >> xs) & 1u, abort_flag, a.err, kWaitLimitCycles)) {
                        ok = false;
                        break;
                    }
                    xpar ^= 1u << xs;
                    for (int s = 0; s < gs; ++s, ++kt) {
                        if (neww) {
                            if (!mbar_wait(b_wfull + 8 * s, (wpar >> s) & 1u, abort_flag, a.err, kWaitLimitCycles)) {
                                ok = false;
                                break;
                            }
                            wpar ^= 1u << s;
                        }
                        if (TWO && (kt & 1u) != par) {   // the other issuer's tile
                            if (lastw) mma_commit(b_wempty + 8 * s);
                            if (++acc == a.nacc) acc = 0;
                            continue;
                        }
                        if (!mbar_wait(b_tempty + 8 * acc, ((tpar >> acc) & 1u) ^ 1u, abort_flag, a.err,
                                       kWaitLimitCycles)) {
                            ok = false;
                            break;
                        }
                        tpar ^= 1u << acc;
                        tc_fence_after();
                        const uint32_t d = tmem + acc * a.nt;
                        uint32_t wl = w_lo0 + s * w_slot16, xl = x_lo0 + xs * x_stage16;
                        for (int kb = 0; kb < a.kb; ++kb, wl += 16384 >> 4, xl += x_kb16)
#pragma unroll
                            for (int ks = 0; ks < 4; ++ks) {   // 32-byte K steps per 128-byte block
                                if (F8) mma_f8_w(d, wl + 2 * ks, w_hi, xl + 2 * ks, x_hi, a.idesc, (kb | ks) != 0);
                                else mma_f16_w(d, wl + 2 * ks, w_hi, xl + 2 * ks, x_hi, a.idesc, (kb | ks) != 0);
                            }
                        mma_commit(b_tfull + 8 * acc);
                        if (lastw) mma_commit(b_wempty + 8 * s);
                        if (++acc == a.nacc) acc = 0;
                    }
                    if (!ok) break;
                    mma_commit(b_xempty + 8 * xs);
                    if (++xs == a.xst) xs = 0;
                    if (++tt == a.t_tiles) tt = 0;
                }
            }
            mma_commit(b_drain);   // all issued MMAs complete before teardown
            drain_wait(b_drain, 0);
        }
        __syncwarp();
    } else if (warp < kStoreWarp && DIRECT) {
        // ---------------------------------------------- epilogue, direct stores
        // Power output with T_int = W in {16, 32, 64} and 256-sample tiles.
        // Warp h of a lane quarter reads its 128 columns (128h..) in two
        // 64-column loads, hands the accumulator back to the MMA after the
        // second, sums the squares of each window, combines the re and im rows
        // with one shuffle and stores its windows straight to the output (one
        // 8- or 16-byte store per beam).  With no staging buffer between the
        // loads the accumulator returns ~40% sooner than through the staged
        // path, which is what bounds the tile rate at 32 antennas (K = 64).
        constexpr int W = WIN > 0 ? WIN : 64;
        constexpr int NW = 64 / W;                    // windows per 64-column load
        const int e = warp - 2;
        const int grp = e >> 3;                       // this group takes the tiles with kt % 2 == grp
        const int q = warp & 3;                       // TMEM lane quarter
        const int h = (e & 7) >> 2;
        const int bq = q * 16 + (lane & 15);          // beam within the M tile
        const bool re_lane = lane < 16;
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + h * 128;
        const int jA = (h * 128) / W, jB = (h * 128 + 64) / W;   // first window of each load
        // NW-window runs are NW-aligned in the output (vector stores need the pointer aligned too)
        const bool vec_ok = (a.T_o % NW) == 0 && ((uintptr_t)a.out & (4 * NW - 1)) == 0;
        const bool pair_ok = (a.T_o % 2) == 0 && ((uintptr_t)a.out & 7) == 0;   // W = 64: windows jA, jA + 1
        uint32_t tpar = 0, kt = 0;
        int acc = 0;
        bool ok = true;
        for (int g = gq0; g < a.n_groups && ok; g += a.gq) {
            int m0, gs;
            group_tiles(a, g, m0, gs);
            int c = c_first, tt = tt_first;
            for (long long ct = ct0; ct < ct1 && ok; ++ct) {
                const int cg = a.c_base + c;
                const int j0 = tt * a.wpt;
                for (int s = 0; s < gs; ++s, ++kt) {
                    if ((int)(kt & 1u) != grp) {   // the other group's tile
                        if (++acc == a.nacc) acc = 0;
                        continue;
                    }
                    if (!mbar_wait(b_tfull + 8 * acc, (tpar >> acc) & 1u, abort_flag, a.err, kWaitLimitCycles)) {
                        ok = false;
                        break;
                    }
                    tpar ^= 1u << acc;
                    tc_fence_after();
                    const uint32_t ta = lane_base + acc * 256;
                    float pa[NW], pb[NW];
                    {
                        uint32_t r[64];
                        tmem_ld64r(ta, r);
#pragma unroll
                        for (int k = 0; k < NW; ++k) pa[k] = sumsq_pk<W>(r + k * W);
                    }
                    {
                        uint32_t r[64];
                        tmem_ld64r(ta + 64, r);
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive_relaxed(b_tempty + 8 * acc);
#pragma unroll
                        for (int k = 0; k < NW; ++k) pb[k] = sumsq_pk<W>(r + k * W);
                    }
#pragma unroll
                    for (int k = 0; k < NW; ++k) {
                        pa[k] += __shfl_xor_sync(0xffffffffu, pa[k], 16);
                        pb[k] += __shfl_xor_sync(0xffffffffu, pb[k], 16);
                    }
                    const int b = (m0 + s) * kBeamsPerMTile + bq;
                    if (re_lane && b < a.B) {
                        const float sc = a.wscale ? a.wscale[(size_t)cg * a.b_pad + b] : 1.f;
                        float *o = a.out + ((size_t)b * a.c_total + cg) * a.T_o + j0;
                        const int nA = a.T_o - (j0 + jA), nB = a.T_o - (j0 + jB);   // windows left
                        if (NW == 1 && pair_ok && nB >= 1) {
                            *reinterpret_cast<float2 *>(o + jA) = make_float2(pa[0] * sc, pb[0] * sc);
                        } else if (NW == 4 && vec_ok && nB >= 4) {
                            *reinterpret_cast<float4 *>(o + jA) = make_float4(pa[0] * sc, pa[1 % NW] * sc,
                                                                              pa[2 % NW] * sc, pa[3 % NW] * sc);
                            *reinterpret_cast<float4 *>(o + jB) = make_float4(pb[0] * sc, pb[1 % NW] * sc,
                                                                              pb[2 % NW] * sc, pb[3 % NW] * sc);
                        } else if (NW == 2 && vec_ok && nB >= 2) {
                            *reinterpret_cast<float2 *>(o + jA) = make_float2(pa[0] * sc, pa[1 % NW] * sc);
                            *reinterpret_cast<float2 *>(o + jB) = make_float2(pb[0] * sc, pb[1 % NW] * sc);
                        } else {
#pragma unroll
                            for (int k = 0; k < NW; ++k) {
                                if (k < nA) o[jA + k] = pa[k] * sc;
                                if (k < nB) o[jB + k] = pb[k] * sc;
                            }
                        }
                    }
                    if (++acc == a.nacc) acc = 0;
                }
                if (++tt == a.t_tiles) {
                    tt = 0;
                    ++c;
                }
            }
        }
    } else if (warp < kStoreWarp) {
        // -------------------------------------------------------------- epilogue
        const int e = warp - 2;
        const int grp = e >> 3;               // this group takes the tiles with kt % 2 == grp
        const int q = warp & 3;               // TMEM lane quarter this warp may access
        const int h = (e & 7) >> 2;           // column slice
        const int part = (lane >> 4) & 1;     // 0: re row, 1: im row
        const int bq = q * 16 + (lane & 15);  // beam within the M tile
        const int cols = a.nt / a.nsplit;
        const int col0 = h * cols;
        const bool active = h < a.nsplit;
        const int wps = COMPLEX ? 0 : cols / a.t_int;   // windows per slice
        uint32_t tpar = 0, kt = 0;
        int acc = 0;
        bool ok = true;
        for (int g = gq0; g < a.n_groups && ok; g += a.gq) {
            int m0, gs;
            group_tiles(a, g, m0, gs);
            int c = c_first, tt = tt_first;
            for (long long ct = ct0; ct < ct1 && ok; ++ct) {
                const int cg = a.c_base + c;
                for (int s = 0; s < gs; ++s, ++kt) {
                    if ((int)(kt & 1u) != grp) {   // the other group's tile
                        if (++acc == a.nacc) acc = 0;
                        continue;
                    }
                    if (!mbar_wait(b_tfull + 8 * acc, (tpar >> acc) & 1u, abort_flag, a.err, kWaitLimitCycles)) {
                        ok = false;
                        break;
                    }
                    tpar ^= 1u << acc;
                    const uint32_t sb = kt % kStageDepth;
                    const uint32_t use = kt / kStageDepth;
                    tc_fence_after();
                    const int b = (m0 + s) * kBeamsPerMTile + bq;
                    const bool bvalid = b < a.B;
                    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + acc * a.nt + col0;
                    // hand the accumulator back to the MMA as soon as it has been read
                    auto release = [&]() {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive_relaxed(b_tempty + 8 * acc);
                    };
                    if (COMPLEX) {
                        if (active) {
                            const float sg = bvalid ? a.wsig[(size_t)cg * a.b_pad + b] : 0.f;
                            float2 *o2 = reinterpret_cast<float2 *>(a.out);
                            const size_t ob = ((size_t)b * a.c_total + cg) * a.T;
                            for (int ch = 0; ch < cols / 16; ++ch) {
                                float v[16], o[16];
                                tmem_ld16(taddr + ch * 16, v);
#pragma unroll
                                for (int i = 0; i < 16; ++i) o[i] = __shfl_xor_sync(0xffffffffu, v[i], 16);
                                const int t0 = tt * a.nt + col0 + ch * 16;
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
                        }
                        release();
                    } else if (!active) {
                        release();
                    } else {
                        const float scale = bvalid ? (a.wscale ? a.wscale[(size_t)cg * a.b_pad + b] : 1.f) : 0.f;
                        float *stg = stage + sb * (kBeamsPerMTile * kMaxWinPerTile);
                        float ws = 0.f;
                        int wi = 0, cnt = 0;
                        bool staged = false;
                        auto emit = [&](float sum) {
                            const float pw = (sum + __shfl_xor_sync(0xffffffffu, sum, 16)) * scale;
                            if (!staged) {
                                // the staging buffer is free once the store warp has written out the
                                // tile that used it kStageDepth tiles ago; waited for here, after the
                                // accumulator (or its first slice) is read, so that this wait is not
                                // in the path between the MMA and the read-out
                                staged = true;
                                if (!mbar_wait(b_sempty + 8 * sb, (use & 1u) ^ 1u, abort_flag, a.err, kWaitLimitCycles))
                                    ok = false;
                            }
                            if (part == 0) stg[bq * kMaxWinPerTile + h * wps + wi] = pw;
                            ++wi;
                        };
                        auto add16 = [&](const float *v) {
                            if (WIN >= 0) {
                                ws += sumsq16(v);
                                cnt += 16;
                                if (cnt == a.t_int) {
                                    emit(ws);
                                    ws = 0.f;
                                    cnt = 0;
                                }
                            } else {
#pragma unroll
                                for (int i = 0; i < 16; ++i) {
                                    ws = fmaf(v[i], v[i], ws);
                                    if (++cnt == a.t_int) {
                                        emit(ws);
                                        ws = 0.f;
                                        cnt = 0;
                                    }
                                }
                            }
                        };
                        int col = 0;
                        if (WIN > 0 && cols % 64 == 0) {
                            for (; col < cols; col += 64) {
                                uint32_t r[64];
                                tmem_ld64r(taddr + col, r);
                                if (col + 64 == cols) release();
#pragma unroll
                                for (int k = 0; k < 64 / (WIN > 0 ? WIN : 64); ++k)
                                    emit(sumsq_pk<(WIN > 0 ? WIN : 64)>(r + k * (WIN > 0 ? WIN : 64)));
                            }
                        }
                        const int n64 = (cols - col) / 64, rem = (cols - col) % 64;   // rem is a multiple of 16
                        for (int bt = 0; bt < n64; ++bt) {
                            float v[64];
                            tmem_ld64(taddr + col + bt * 64, v);
                            if (bt == n64 - 1 && rem == 0) release();
#pragma unroll
                            for (int k = 0; k < 4; ++k) add16(v + 16 * k);
                        }
                        for (col += n64 * 64; col < cols; col += 16) {
                            float v[16];
                            tmem_ld16(taddr + col, v);
                            if (col + 16 == cols) release();
                            add16(v);
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(b_sfull + 8 * sb);   // publishes the staged windows
                    }
                    if (++acc == a.nacc) acc = 0;
                    if (!ok) break;
                }
                if (++tt == a.t_tiles) {
                    tt = 0;
                    ++c;
                }
            }
        }
    } else if (IN && (warp > kStoreWarp || (DIRECT && warp == kStoreWarp))) {
        // ------------------------------------------------------ converter warps
        // for each (channel, time tile), in the producer's order: wait for the
        // raw tile, widen its K blocks into the voltage stage, publish it
        constexpr int nconv = (kConvWarps + (DIRECT ? 1 : 0)) * 32;
        const int tid = (warp - kStoreWarp - (DIRECT ? 0 : 1)) * 32 + lane;
        const uint8_t *raw = gbase + (size_t)a.xst * a.x_stage_bytes + (size_t)a.gmax * a.w_slot_bytes;
        uint32_t rcnt = 0, xcnt = 0;
        int xs = 0;
        bool ok = true;
        for (int g = gq0; g < a.n_groups && ok; g += a.gq) {
            for (long long ct = ct0; ct < ct1; ++ct) {
                if (!mbar_wait(b_rfull, rcnt & 1u, abort_flag, a.err, kWaitLimitCycles) ||
                    !mbar_wait(b_xempty + 8 * xs, ((xcnt >> xs) & 1u) ^ 1u, abort_flag, a.err, kWaitLimitCycles)) {
                    ok = false;
                    break;
                }
                ++rcnt;
                xcnt ^= 1u << xs;
                uint8_t *dst = gbase + (size_t)xs * a.x_stage_bytes;
                for (int kb = 0; kb < a.kb; ++kb)
                    widen_block_smem<IN>(raw + (size_t)kb * a.nt * a.raw_kb, dst + (size_t)kb * a.nt * 128, a.nt,
                                         tid, nconv);
                __syncwarp();
                if (lane == 0) mbar_arrive(b_rempty);   // the raw buffer is read: the next tile may land
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(b_xfull + 8 * xs);
                if (++xs == a.xst) xs = 0;
            }
        }
    } else if (warp == kStoreWarp && !COMPLEX && !DIRECT) {
        // ------------------------------------------------------------ store warp
        // writes each staged tile as one run of windows per beam
        uint32_t kt = 0;
        bool ok = true;
        const bool vec = (a.T_o & 3) == 0 && (a.wpt & 3) == 0 && ((uintptr_t)a.out & 15) == 0;
        const bool vec2 = (a.T_o & 1) == 0 && (a.wpt & 1) == 0 && ((uintptr_t)a.out & 7) == 0;
        for (int g = gq0; g < a.n_groups && ok; g += a.gq) {
            int m0, gs;
            group_tiles(a, g, m0, gs);
            int c = c_first, tt = tt_first;
            for (long long ct = ct0; ct < ct1 && ok; ++ct) {
                const int cg = a.c_base + c;
                const int j0 = tt * a.wpt;
                const int nj = min(a.wpt, a.T_o - j0);
                for (int s = 0; s < gs; ++s, ++kt) {
                    const uint32_t sb = kt % kStageDepth;
                    if (!mbar_wait(b_sfull + 8 * sb, (kt / kStageDepth) & 1u, abort_flag, a.err, kWaitLimitCycles)) {
                        ok = false;
                        break;
                    }
                    const float *stg = stage + sb * (kBeamsPerMTile * kMaxWinPerTile);
                    const int b_tile0 = (m0 + s) * kBeamsPerMTile;
                    if (vec && a.wpt == 4) {
                        // one float4 per beam: lanes take beams lane and lane + 32
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            const int bl = lane + 32 * r;
                            const int bb = b_tile0 + bl;
                            if (bb < a.B && nj > 0) {
                                const float4 v4 = *reinterpret_cast<const float4 *>(stg + bl * kMaxWinPerTile);
                                *reinterpret_cast<float4 *>(a.out + ((size_t)bb * a.c_total + cg) * a.T_o + j0) = v4;
                            }
                        }
                    } else if (vec2 && a.wpt == 2) {
                        // one float2 per beam
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            const int bl = lane + 32 * r;
                            const int bb = b_tile0 + bl;
                            if (bb < a.B && nj > 0) {
                                const float2 v2 = *reinterpret_cast<const float2 *>(stg + bl * kMaxWinPerTile);
                                *reinterpret_cast<float2 *>(a.out + ((size_t)bb * a.c_total + cg) * a.T_o + j0) = v2;
                            }
                        }
                    } else if (vec) {
                        const int per = a.wpt >> 2;
                        for (int i = lane; i < kBeamsPerMTile * per; i += 32) {
                            const int bl = i / per, k = (i % per) * 4;
                            const int bb = b_tile0 + bl;
                            if (bb < a.B && k < nj) {
                                const float4 v4 = *reinterpret_cast<const float4 *>(stg + bl * kMaxWinPerTile + k);
                                *reinterpret_cast<float4 *>(a.out + ((size_t)bb * a.c_total + cg) * a.T_o + j0 + k) = v4;
                            }
                        }
                    } else {
                        for (int i = lane; i < kBeamsPerMTile * a.wpt; i += 32) {
                            const int bl = i / a.wpt, k = i % a.wpt;
                            const int bb = b_tile0 + bl;
                            if (bb < a.B && k < nj)
                                a.out[((size_t)bb * a.c_total + cg) * a.T_o + j0 + k] = stg[bl * kMaxWinPerTile + k];
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive_relaxed(b_sempty + 8 * sb);
                }
                if (++tt == a.t_tiles) {
                    tt = 0;
                    ++c;
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ----------------------------------------------------------- launchers
template <bool F8, int WIN, bool CPX, bool DIRECT, int IN>
static cudaError_t launch_v(const CUtensorMap &xm, const CUtensorMap &wm, const TcKernelArgs &ka, int grid, int smem,
                            cudaStream_t s)
{
    auto kern = k_tc<F8, WIN, CPX, DIRECT, IN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kTcThreads + (IN ? kConvWarps * 32 : 0), smem, s>>>(xm, wm, ka);
    return cudaGetLastError();
}

template <bool F8, int WIN, bool CPX, bool DIRECT>
static cudaError_t launch_in(const CUtensorMap &xm, const CUtensorMap &wm, const TcKernelArgs &ka, int in_dtype,
                             int grid, int smem, cudaStream_t s)
{
    if (F8) return launch_v<F8, WIN, CPX, DIRECT, 0>(xm, wm, ka, grid, smem, s);   // FP8 inputs only
    switch (in_dtype) {
    case BF_CI8: return launch_v<F8, WIN, CPX, DIRECT, BF_CI8>(xm, wm, ka, grid, smem, s);
    case BF_CI4: return launch_v<F8, WIN, CPX, DIRECT, BF_CI4>(xm, wm, ka, grid, smem, s);
    default: return launch_v<F8, WIN, CPX, DIRECT, 0>(xm, wm, ka, grid, smem, s);
    }
}

// Power tiles of 256 samples split in two 128-column slices, with a window
// known at compile time, take the direct-store epilogue; every other case the
// staged one (the store warp writes runs of windows).
template <bool F8, int WIN, bool CPX>
static cudaError_t launch_one(const CUtensorMap &xm, const CUtensorMap &wm, const TcKernelArgs &ka, int in_dtype,
                              int grid, int smem, cudaStream_t s)
{
    if constexpr (!CPX && WIN > 0) {
        if (ka.nt == 256 && ka.nsplit == 2) return launch_in<F8, WIN, CPX, true>(xm, wm, ka, in_dtype, grid, smem, s);
    }
    return launch_in<F8, WIN, CPX, false>(xm, wm, ka, in_dtype, grid, smem, s);
}

template <bool F8, int IN>
cudaError_t launch_tc_family(const CUtensorMap &xm, const CUtensorMap &wm, const TcKernelArgs &ka, int win, bool cpx,
                             int grid, int smem, cudaStream_t s)
{
    if (cpx) return launch_one<F8, 0, true>(xm, wm, ka, IN, grid, smem, s);
    switch (win) {
    case 64: return launch_one<F8, 64, false>(xm, wm, ka, IN, grid, smem, s);
    case 32: return launch_one<F8, 32, false>(xm, wm, ka, IN, grid, smem, s);
    case 16: return launch_one<F8, 16, false>(xm, wm, ka, IN, grid, smem, s);
    case 0: return launch_one<F8, 0, false>(xm, wm, ka, IN, grid, smem, s);
    default: return launch_one<F8, -1, false>(xm, wm, ka, IN, grid, smem, s);
    }
}

}  // namespace bfi
