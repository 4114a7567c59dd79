// Batched persistent tensor-core beamformer: the jobs of several plans
// (sub-arrays, beam sets and channel counts of uneven sizes, or chunks of
// several streams) in one launch.
//
// Every job keeps its own plan (weights, per-beam scales) and its own input
// and output buffers; the launch reads a table with one entry per job (the
// two TMA tensor maps and the job's shape), in its parameters or in device
// memory.  Work units are (job, channel, time tile, M tile), M tile fastest,
// numbered over all jobs.  In a launch over several jobs each CTA's producer
// takes the next unit from a counter in device memory (zeroed before the
// launch), so the units in flight at any moment are a window of neighbouring
// units, of one channel of one job most of the time: its weight and voltage
// tiles are shared through L2, and a CTA that runs slower simply takes fewer
// units.  (A fixed stride, CTA i taking units i, i + G, ..., let the CTAs
// drift apart over a long launch: on the 20 sub-array jobs of 128 and 256
// antennas of the uneven-batch workload one launch read 135 GB from DRAM
// against 79 GB for the same jobs launched one at a time.)  A launch over
// one job keeps the fixed stride, which measured faster there.
// Every job runs the streamed pipeline (one 128-byte K block of weights and
// voltages per stage), so any antenna count fits the same kernel; the
// epilogue and store warp are the single-plan kernel's.
//
// A batch step (bf_batch_execute) sends jobs of fewer than 4 K blocks (the
// short-K sub-arrays) to their plans' resident-weight kernel instead, on a
// few forked branches: streaming a 16 KB weight block per stage for a
// 64-element K block puts three times the single-plan kernel's shared-memory
// and L2 bytes on every MMA (on the 28 jobs of 16 to 64 antennas of the
// uneven-batch workload this kernel took 25.8 ms against 20-21 ms for their
// resident-weight launches).  Of the other jobs, each large one gets a launch
// of this kernel to itself and the small ones share one launch.  The step
// can be captured in a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "batch.h"
#include "tc_common.cuh"

namespace bfi {

struct BatchArgs {
    const BatchJob *jobs;
    int n_jobs;
    long long total_units;
    int nt, nsplit, wpt, t_int, xst, nacc;
    uint32_t stage_bytes;   // 16384 + nt * 128
    unsigned *err;
    unsigned long long *next;   // the next unit to take; zero at launch
};

__device__ __forceinline__ int job_of(const BatchJob *jobs, int n_jobs, long long u)
{
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].unit0 <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// What the MMA issuer, the epilogue and the store warp need to know about
// one tile, written by the producer (which takes the units) into a ring in
// shared memory, so the 16 epilogue warps carry no unit state (their
// registers go to the accumulator read-out).  A slot is reused once the
// consumer of its descriptor (the epilogue group or the store warp) and the
// MMA issuer have both released it.
struct __align__(16) TileDesc {
    const float *wscale;   // per-beam power scale rows of the job's first channel, or NULL
    const float *wsig;     // per-beam amplitude scale rows, offset likewise (complex output)
    float *out;            // the job's powers (or complex beams), offset to its first channel
    const float *acc_in;   // carried-window sums, offset likewise, or NULL
    float *acc_out;
    int b0, n_beams, b_pad, c, tt, T, T_o, c_total, last;   // last != 0: no more tiles
    int kbn, ks_last;      // the job's K blocks, and MMA k-steps holding antennas in its last block
    uint32_t idesc;        // the job's MMA instruction descriptor
};
constexpr int kDescRing = 16;

// CPX: complex beams [B][C][T][2] straight from the epilogue (the store warp
// only recycles the descriptor slots); otherwise integrated powers.
// DIRECT (powers, 256-sample tiles, T_int of 16, 32 or 64): the epilogue warps
// store their windows straight to the output, route the carried windows
// themselves and hand the descriptor slot back; the store warp has no work.
template <bool F8, int WIN, bool CPX, bool DIRECT>
__global__ void __maxnreg__(96) k_tc_batch(const BatchArgs a, const __grid_constant__ ParamJobs pj)
{
    const BatchJob *jobs = a.jobs ? a.jobs : pj.j;   // a table in device memory, or jobs passed by value
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t sx = base;
    float *stage = reinterpret_cast<float *>(gbase + a.xst * a.stage_bytes);
    TileDesc *desc = reinterpret_cast<TileDesc *>(stage + kStageDepth * kBeamsPerMTile * kMaxWinPerTile);
    uint64_t *bars = reinterpret_cast<uint64_t *>(desc + kDescRing);
    const uint32_t b_full = smem_u32(bars + 0);                  // [kMaxXStages]
    const uint32_t b_empty = smem_u32(bars + kMaxXStages);       // [kMaxXStages]
    const uint32_t b_tfull = smem_u32(bars + 2 * kMaxXStages);   // [kMaxAcc]
    const uint32_t b_tempty = b_tfull + 8 * kMaxAcc;              // [kMaxAcc]
    const uint32_t b_drain = b_tempty + 8 * kMaxAcc;
    const uint32_t b_sfull = b_drain + 8;                         // [kStageDepth]
    const uint32_t b_sempty = b_sfull + 8 * kStageDepth;          // [kStageDepth]
    const uint32_t b_dfull = b_sempty + 8 * kStageDepth;          // [kDescRing]
    const uint32_t b_dempty = b_dfull + 8 * kDescRing;            // [kDescRing]
    const uint32_t b_mempty = b_dempty + 8 * kDescRing;           // [kDescRing] (the MMA issuer's release)
    uint32_t *tmem_holder =
        reinterpret_cast<uint32_t *>(bars + 2 * kMaxXStages + 2 * kMaxAcc + 1 + 2 * kStageDepth + 3 * kDescRing);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < a.xst; ++i) {
            mbar_init(b_full + 8 * i, 1);
            mbar_init(b_empty + 8 * i, 1);
        }
        for (int i = 0; i < a.nacc; ++i) {
            mbar_init(b_tfull + 8 * i, 1);
            mbar_init(b_tempty + 8 * i, kEpiWarps / 2);   // one group releases each use
        }
        mbar_init(b_drain, 1);
        for (int i = 0; i < kStageDepth; ++i) {
            mbar_init(b_sfull + 8 * i, 4 * a.nsplit);
            mbar_init(b_sempty + 8 * i, 1);
        }
        for (int i = 0; i < kDescRing; ++i) {
            mbar_init(b_dfull + 8 * i, 1);
            mbar_init(b_dempty + 8 * i, DIRECT ? 8 : 1);   // the epilogue group, or the store warp
            mbar_init(b_mempty + 8 * i, 1);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_holder), kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            uint32_t cnt = 0, issued = 0, kt = 0;
            int st = 0;
            bool ok = true;
            const CUtensorMap *xmap = nullptr, *wmap = nullptr;
            int kbn = 0, ke = 0, t_shift = 0, c_base = 0, j = 0, jcur = -1, mt = 1, t_tiles = 1;
            long long unit0 = 0;
            TileDesc d{};
            const uint32_t bytes = 16384 + a.nt * 128;
            // publishes one tile descriptor (after its last readers have released the slot)
            auto publish = [&](const TileDesc &v) -> bool {
                const uint32_t slot = kt % kDescRing;
                const uint32_t ph = ((kt / kDescRing) & 1u) ^ 1u;
                if (!mbar_wait(b_dempty + 8 * slot, ph, abort_flag, a.err, kWaitLimitCycles) ||
                    !mbar_wait(b_mempty + 8 * slot, ph, abort_flag, a.err, kWaitLimitCycles))
                    return false;
                desc[slot] = v;
                mbar_arrive(b_dfull + 8 * slot);
                ++kt;
                return true;
            };
            // units from the launch's counter, or (no counter) units blockIdx.x,
            // + gridDim.x, ...
            long long u = a.next ? (long long)atomicAdd(a.next, 1ull) : (long long)blockIdx.x;
            if (u < a.total_units) j = job_of(jobs, a.n_jobs, u);
            while (ok && u < a.total_units) {
                // the next unit is taken now; its number is needed after this one's loads
                const long long u_next = a.next ? (long long)atomicAdd(a.next, 1ull) : u + gridDim.x;
                while (u >= jobs[j].unit0 + jobs[j].units) ++j;   // units only increase (empty jobs skipped)
                if (j != jcur) {
                    jcur = j;
                    const BatchJob &J = jobs[j];
                    xmap = &J.xmap;
                    wmap = &J.wmap;
                    prefetch_tensormap(xmap);
                    prefetch_tensormap(wmap);
                    kbn = J.kb;
                    ke = J.ke;
                    t_shift = J.t_shift;
                    c_base = J.c_base;
                    mt = J.mt;
                    t_tiles = J.t_tiles;
                    unit0 = J.unit0;
                    d.wscale = J.wscale ? J.wscale + (size_t)J.c_base * J.b_pad : nullptr;
                    d.wsig = J.wsig + (size_t)J.c_base * J.b_pad;
                    d.out = J.out + (size_t)J.c_base * (CPX ? 2 * (size_t)J.T : (size_t)J.T_o);
                    d.T = J.T;
                    d.acc_in = J.acc_in ? J.acc_in + J.c_base : nullptr;
                    d.acc_out = J.acc_out ? J.acc_out + J.c_base : nullptr;
                    d.n_beams = J.B;
                    d.b_pad = J.b_pad;
                    d.T_o = J.T_o;
                    d.c_total = J.c_total;
                    d.kbn = J.kb;
                    d.ks_last = J.ks_last;
                    d.idesc = J.idesc;
                }
                // (job, channel, time tile, M tile), M tile fastest (a job has
                // fewer than 2^31 units: 32-bit divisions)
                const uint32_t v = (uint32_t)(u - unit0);
                const int m = (int)(v % (uint32_t)mt);
                const uint32_t r = v / (uint32_t)mt;
                const int tt = (int)(r % (uint32_t)t_tiles);
                const int c = (int)(r / (uint32_t)t_tiles);
                d.b0 = m * kBeamsPerMTile;
                d.c = c;
                d.tt = tt;
                d.last = 0;
                if (!publish(d)) break;
                for (int kb = 0; kb < kbn; ++kb) {
                    if (!mbar_wait(b_empty + 8 * st, ((cnt >> st) & 1u) ^ 1u, abort_flag, a.err, kWaitLimitCycles)) {
                        ok = false;
                        break;
                    }
                    cnt ^= 1u << st;
                    issued |= 1u << st;
                    const uint32_t dst = sx + st * a.stage_bytes;
                    mbar_arrive_expect_tx(b_full + 8 * st, bytes);
                    tma_load_3d(dst, wmap, b_full + 8 * st, kb * ke, m * kRowsPerMTile, c_base + c);
                    // window 0 starts t_shift samples before the chunk: those rows
                    // (negative time coordinates) read as zeros
                    tma_load_3d(dst + 16384, xmap, b_full + 8 * st, kb * ke, tt * a.nt - t_shift, c);
                    if (++st == a.xst) st = 0;
                }
                u = u_next;
            }
            // two end markers: one for each epilogue group's next tile (the MMA
            // issuer stops at the first)
            d.last = 1;
            if (!*abort_flag && publish(d)) publish(d);
            if (*abort_flag)
                for (int i = 0; i < a.xst; ++i)
                    if (issued & (1u << i)) drain_wait(b_full + 8 * i, ((cnt >> i) & 1u) ^ 1u);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ----------------------------------------------------------- MMA issuer
        // (one issuer: a second one taking alternate tiles would have to skip
        // the other's stage fills without waiting, and with tiles of several
        // K blocks it can fall two phases behind on a stage, where a parity
        // wait can no longer tell the phases apart)
        if (lane == 0) {
            uint32_t par = 0, tpar = 0;
            int st = 0, acc = 0;
            bool ok = true;
            // descriptor words of stage 0; a stage's operands are an offset added to the
            // low word (start address in 16-byte units; no carry below 256 KB)
            const uint64_t s_desc0 = sdesc_sw128(sx);
            const uint32_t s_hi = (uint32_t)(s_desc0 >> 32), s_lo0 = (uint32_t)s_desc0;
            const uint32_t stage16 = a.stage_bytes >> 4;
            for (uint32_t kt = 0; ok; ++kt) {
                // the tile's K extent from its descriptor, then the slot is released
                const uint32_t slot = kt % kDescRing;
                if (!mbar_wait(b_dfull + 8 * slot, (kt / kDescRing) & 1u, abort_flag, a.err, kWaitLimitCycles)) break;
                const TileDesc &D = desc[slot];
                const int last = D.last, kbn = D.kbn, ks_last = D.ks_last;
                const uint32_t idesc = D.idesc;
                mbar_arrive(b_mempty + 8 * slot);
                if (last) break;
                if (!mbar_wait(b_tempty + 8 * acc, ((tpar >> acc) & 1u) ^ 1u, abort_flag, a.err, kWaitLimitCycles)) {
                    ok = false;
                    break;
                }
                tpar ^= 1u << acc;
                tc_fence_after();
                const uint32_t dacc = tmem + acc * a.nt;
                for (int kb = 0; kb < kbn; ++kb) {
                    if (!mbar_wait(b_full + 8 * st, (par >> st) & 1u, abort_flag, a.err, kWaitLimitCycles)) {
                        ok = false;
                        break;
                    }
                    par ^= 1u << st;
                    tc_fence_after();
                    const uint32_t wl = s_lo0 + st * stage16, xl = wl + (16384 >> 4);
                    // the last K block may hold fewer than 4 k-steps of antennas (the
                    // rest is zero padding): those MMAs are skipped
                    const int ksn = kb + 1 == kbn ? ks_last : 4;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        if (ks >= ksn) break;
                        if (F8) mma_f8_w(dacc, wl + 2 * ks, s_hi, xl + 2 * ks, s_hi, idesc, (kb | ks) != 0);
                        else mma_f16_w(dacc, wl + 2 * ks, s_hi, xl + 2 * ks, s_hi, idesc, (kb | ks) != 0);
                    }
                    mma_commit(b_empty + 8 * st);
                    if (++st == a.xst) st = 0;
                }
                if (!ok) break;
                mma_commit(b_tfull + 8 * acc);
                if (++acc == a.nacc) acc = 0;
            }
            mma_commit(b_drain);
            drain_wait(b_drain, 0);
        }
        __syncwarp();
    } else if (warp < kStoreWarp && DIRECT) {
        // ---------------------------------------------- epilogue, direct stores
        // As in the single-plan kernel: warp h of a lane quarter reads its 128
        // columns (128h..) in two 64-column loads, releases the accumulator
        // after the second, sums each window's squares, combines re and im
        // rows with one shuffle and writes its windows itself: window 0 first
        // takes the partial sum carried in, the window left open at the end of
        // the chunk goes to acc_out, the others to the output.
        constexpr int W = WIN > 0 ? WIN : 64;
        constexpr int NW = 64 / W;                    // windows per 64-column load
        const int e = warp - 2;
        const int grp = e >> 3;
        const int q = warp & 3;
        const int h = (e & 7) >> 2;
        const int bq = q * 16 + (lane & 15);
        const bool re_lane = lane < 16;
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + h * 128;
        const int jA = (h * 128) / W, jB = (h * 128 + 64) / W;
        for (uint32_t kt = grp;; kt += 2) {
            const uint32_t slot = kt % kDescRing;
            if (!mbar_wait(b_dfull + 8 * slot, (kt / kDescRing) & 1u, abort_flag, a.err, kWaitLimitCycles)) break;
            const TileDesc &D = desc[slot];
            if (D.last) break;
            // the tile's fields into registers, then the slot goes back to the producer
            const int b = D.b0 + bq;
            const bool bvalid = b < D.n_beams;
            const int c = D.c, T_o = D.T_o, j0 = D.tt * a.wpt;
            const size_t row = (size_t)b * D.c_total + c;
            const float sc = (re_lane && bvalid && D.wscale) ? D.wscale[(size_t)c * D.b_pad + b] : 1.f;
            float *const o = D.out + row * T_o + j0;
            const float *const acc_in = D.acc_in;
            float *const acc_out = D.acc_out;
            __syncwarp();
            if (lane == 0) mbar_arrive(b_dempty + 8 * slot);
            const int acc = (int)(kt % (uint32_t)a.nacc);
            if (!mbar_wait(b_tfull + 8 * acc, (kt / a.nacc) & 1u, abort_flag, a.err, kWaitLimitCycles)) break;
            tc_fence_after();
            const uint32_t ta = lane_base + acc * a.nt;
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
                tile_release(b_tempty + 8 * acc, lane);
#pragma unroll
                for (int k = 0; k < NW; ++k) pb[k] = sumsq_pk<W>(r + k * W);
            }
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                pa[k] = (pa[k] + __shfl_xor_sync(0xffffffffu, pa[k], 16)) * sc;
                pb[k] = (pb[k] + __shfl_xor_sync(0xffffffffu, pb[k], 16)) * sc;
            }
            if (re_lane && bvalid) {
                const bool inner = (j0 > 0 || !acc_in) && j0 + jB + NW <= T_o;
                const uintptr_t oa = (uintptr_t)(o + jA);
                if (inner && NW == 1 && (oa & 7) == 0) {
                    *reinterpret_cast<float2 *>(o + jA) = make_float2(pa[0], pb[0]);
                } else if (inner && NW == 2 && (oa & 7) == 0) {
                    *reinterpret_cast<float2 *>(o + jA) = make_float2(pa[0], pa[1 % NW]);
                    *reinterpret_cast<float2 *>(o + jB) = make_float2(pb[0], pb[1 % NW]);
                } else if (inner && NW == 4 && (oa & 15) == 0) {
                    *reinterpret_cast<float4 *>(o + jA) = make_float4(pa[0], pa[1 % NW], pa[2 % NW], pa[3 % NW]);
                    *reinterpret_cast<float4 *>(o + jB) = make_float4(pb[0], pb[1 % NW], pb[2 % NW], pb[3 % NW]);
                } else {
                    // edge tiles: the carried-in window 0, the open window T_o, the tail
#pragma unroll
                    for (int k = 0; k < 2 * NW; ++k) {
                        const int jl = k < NW ? jA + k : jB + (k - NW);
                        float p = k < NW ? pa[k] : pb[k - NW];
                        const int j = j0 + jl;
                        if (j == 0 && acc_in) p += acc_in[row];
                        if (j < T_o) o[jl] = p;
                        else if (j == T_o && acc_out) acc_out[row] = p;
                    }
                }
            }
        }
    } else if (warp < kStoreWarp) {
        // -------------------------------------------------------------- epilogue
        // two groups of 8 warps take alternate tiles (and so alternate
        // accumulators: nacc is even); in a group, two warps per TMEM lane
        // quarter, each on a half of the tile's columns
        const int e = warp - 2;
        const int grp = e >> 3;
        const int q = warp & 3;
        const int h = (e & 7) >> 2;
        const int bq = q * 16 + (lane & 15);
        const int cols = a.nt / a.nsplit;
        const int col0 = h * cols;
        const bool active = h < a.nsplit;
        for (uint32_t kt = grp;; kt += 2) {
            const uint32_t slot = kt % kDescRing;
            if (!mbar_wait(b_dfull + 8 * slot, (kt / kDescRing) & 1u, abort_flag, a.err, kWaitLimitCycles)) break;
            const TileDesc &D = desc[slot];
            if (D.last) break;
            const int acc = (int)(kt % (uint32_t)a.nacc);
            if (!mbar_wait(b_tfull + 8 * acc, (kt / a.nacc) & 1u, abort_flag, a.err, kWaitLimitCycles)) break;
            const uint32_t sb = kt % kStageDepth;
            if (active && !mbar_wait(b_sempty + 8 * sb, ((kt / kStageDepth) & 1u) ^ 1u, abort_flag, a.err,
                                     kWaitLimitCycles))
                break;
            tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + acc * a.nt + col0;
            const uint32_t tempty = b_tempty + 8 * acc;
            if (!active) {
                tile_release(tempty, lane);
            } else if (CPX) {
                struct {
                    int nt, T, c_total, b_pad;
                    const float *wsig;
                    float *out;
                } o{a.nt, D.T, D.c_total, D.b_pad, D.wsig, D.out};
                const int b = D.b0 + bq;
                epi_complex_tile(o, taddr, cols, col0, D.tt, lane, b, b < D.n_beams, D.c);
                tile_release(tempty, lane);
                __syncwarp();
                if (lane == 0) mbar_arrive(b_sfull + 8 * sb);   // done with the descriptor
            } else {
                struct {
                    int t_int, b_pad;
                    const float *wscale;
                } o{a.t_int, D.b_pad, D.wscale};
                const int b = D.b0 + bq;
                epi_power_tile<WIN>(o, taddr, cols, h, lane, bq, b, b < D.n_beams, D.c,
                                    stage + sb * (kBeamsPerMTile * kMaxWinPerTile), tempty, b_sfull + 8 * sb);
            }
        }
    } else if (warp == kStoreWarp && !DIRECT) {
        // ------------------------------------------------------------ store warp
        for (uint32_t kt = 0;; ++kt) {
            const uint32_t slot = kt % kDescRing;
            if (!mbar_wait(b_dfull + 8 * slot, (kt / kDescRing) & 1u, abort_flag, a.err, kWaitLimitCycles)) break;
            const TileDesc &D = desc[slot];
            if (D.last) break;
            const uint32_t sb = kt % kStageDepth;
            if (!mbar_wait(b_sfull + 8 * sb, (kt / kStageDepth) & 1u, abort_flag, a.err, kWaitLimitCycles)) break;
            if (!CPX) {
                const TileOut o{a.nt,     a.nsplit, a.wpt, a.t_int, 0,        D.T_o,    D.n_beams,
                                D.b_pad,  D.c_total, D.wscale, nullptr, D.out, D.acc_in, D.acc_out};
                store_tile(o, stage + sb * (kBeamsPerMTile * kMaxWinPerTile), D.b0, D.c, D.tt, lane);
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive_relaxed(b_sempty + 8 * sb);
                mbar_arrive(b_dempty + 8 * slot);   // the producer may reuse the descriptor slot
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

}  // namespace bfi

// ----------------------------------------------------------------- host side
namespace bfi {

static int batch_stage_bytes(int nt) { return 16384 + nt * 128; }
static int batch_layout_end(int xst, int nt)
{
    return 1024 + xst * batch_stage_bytes(nt) + kStageDepth * kBeamsPerMTile * kMaxWinPerTile * 4 +
           kDescRing * (int)sizeof(TileDesc) + 8 * (2 * kMaxXStages + 2 * kMaxAcc + 1 + 2 * kStageDepth + 3 * kDescRing) +
           8;
}

// The attribute is a per-kernel maximum shared by every batch: it is set to
// the largest size any batch asks for, so one batch never lowers another's.
template <bool F8, int WIN, bool CPX, bool DIRECT>
static cudaError_t batch_attr()
{
    return cudaFuncSetAttribute(k_tc_batch<F8, WIN, CPX, DIRECT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kSmemLimit);
}

template <bool F8, int WIN, bool CPX, bool DIRECT>
static cudaError_t batch_launch(const BatchArgs &ka, const ParamJobs &pj, int grid, int smem, cudaStream_t s)
{
    k_tc_batch<F8, WIN, CPX, DIRECT><<<grid, kTcThreads, smem, s>>>(ka, pj);
    return cudaGetLastError();
}

static int batch_win(int t_int)
{
    return (t_int == 64 || t_int == 32 || t_int == 16) ? t_int : (t_int % 16 == 0 ? 0 : -1);
}

// Calls F.template run<F8, WIN, CPX, DIRECT>() for the core's operand format,
// window specialisation and output kind.
template <bool F8, class F>
static cudaError_t batch_dispatch_f(const BatchCore &core, F &f)
{
    if (core.cpx) return f.template run<F8, 0, true, false>();
    switch (batch_win(core.t_int)) {
    case 64: return core.direct ? f.template run<F8, 64, false, true>() : f.template run<F8, 64, false, false>();
    case 32: return core.direct ? f.template run<F8, 32, false, true>() : f.template run<F8, 32, false, false>();
    case 16: return core.direct ? f.template run<F8, 16, false, true>() : f.template run<F8, 16, false, false>();
    case 0: return f.template run<F8, 0, false, false>();
    default: return f.template run<F8, -1, false, false>();
    }
}

template <class F>
static cudaError_t batch_dispatch(const BatchCore &core, F &&f)
{
    return core.f8 ? batch_dispatch_f<true>(core, f) : batch_dispatch_f<false>(core, f);
}

struct BatchAttr {
    template <bool F8, int WIN, bool CPX, bool DIRECT>
    cudaError_t run() const { return batch_attr<F8, WIN, CPX, DIRECT>(); }
};

struct BatchLaunch {
    const BatchArgs &ka;
    const ParamJobs &pj;
    int grid, smem;
    cudaStream_t s;
    template <bool F8, int WIN, bool CPX, bool DIRECT>
    cudaError_t run() const { return batch_launch<F8, WIN, CPX, DIRECT>(ka, pj, grid, smem, s); }
};

bf_status batch_core_init(BatchCore *core, bf_plan *const *plans, int n, int tile_t)
{
    if (!plans || n < 1) return set_error(BF_ERR_ARG, "need at least one plan");
    const bf_plan *p0 = plans[0];
    if (!p0) return set_error(BF_ERR_ARG, "NULL plan");
    for (int i = 0; i < n; ++i) {
        const bf_plan *p = plans[i];
        if (!p) return set_error(BF_ERR_ARG, "NULL plan");
        if (p->wf.simt) return set_error(BF_ERR_UNSUPPORTED, "batches run tensor-core plans (not BF_C32)");
        if (p->wf.op != p0->wf.op)
            return set_error(BF_ERR_UNSUPPORTED, "all plans of a batch must share the operand format");
        if (p->t_int != p0->t_int) return set_error(BF_ERR_UNSUPPORTED, "all plans of a batch must share T_int");
        if (p->device != p0->device) return set_error(BF_ERR_UNSUPPORTED, "all plans must be on one device");
    }
    const int t_int = p0->t_int;
    int g = 16, t = t_int;
    while (t) {
        const int r = g % t;
        g = t;
        t = r;
    }
    const int unit = 16 / g * t_int;   // lcm(16, T_int)
    int nt = 0;
    for (int cand = 256; cand >= unit && cand >= 16; cand -= 16) {
        if (cand % unit || cand / t_int > kMaxWinPerTile) continue;
        if (tile_t && cand != tile_t) continue;
        nt = cand;
        break;
    }
    if (!nt) return set_error(BF_ERR_UNSUPPORTED, "no tile width fits this T_int (and request)");
    BatchCore c;
    c.nt = nt;
    c.t_int = t_int;
    c.nsplit = ((nt / 2) % 16 == 0 && (nt / 2) % t_int == 0) ? 2 : 1;
    c.wpt = nt / t_int;
    c.nacc = std::min(kMaxAcc, kTmemCols / nt) & ~1;   // even: each epilogue group keeps its own accumulators
    c.f8 = p0->wf.op == kOpE4M3;
    c.direct = batch_win(t_int) > 0 && nt == 256 && c.nsplit == 2;
    c.num_sms = std::max(1, p0->num_sms);
    const int fixed = batch_layout_end(0, nt);
    c.xst = std::min(kMaxXStages, (kSmemLimit - fixed) / batch_stage_bytes(nt));
    c.smem = std::max(batch_layout_end(c.xst, nt), 116 * 1024);
    if (c.xst < 2 || batch_layout_end(c.xst, nt) > c.smem || c.smem > kSmemLimit)
        return set_error(BF_ERR_UNSUPPORTED, "batch stages do not fit in shared memory");
    cudaError_t e = batch_dispatch(c, BatchAttr{});
    if (e == cudaSuccess) {   // the complex-output variant of the same format (single plans)
        BatchCore cc = c;
        cc.cpx = true;
        e = batch_dispatch(cc, BatchAttr{});
    }
    if (e != cudaSuccess) return cuda_error(e, "batch kernel attribute");
    *core = c;
    return BF_OK;
}

bf_status batch_fill_job(const BatchCore &core, BatchJob *J, const bf_plan *p, const void *x_mma, int T,
                         float *out, int t_shift, const float *acc_in, float *acc_out, int c_base, int c_count)
{
    if (core.cpx && (t_shift || acc_in || acc_out))
        return set_error(BF_ERR_ARG, "complex beam output carries no integration window");
    if (c_count < 0) c_count = p->C - c_base;
    if (c_base < 0 || c_count < 0 || c_base + c_count > p->C) return set_error(BF_ERR_ARG, "channel range");
    if (T < 0) return set_error(BF_ERR_ARG, "n_samp must be >= 0");
    if (t_shift < 0 || t_shift >= p->t_int) return set_error(BF_ERR_ARG, "carried samples must be in [0, T_int)");
    const WeightFormat &f = p->wf;
    memset((void *)J, 0, sizeof(BatchJob));
    const int frame = t_shift + T;   // samples from the start of window 0
    const int T_o = frame / p->t_int;
    const int partial = (acc_out && frame % p->t_int) ? 1 : 0;
    J->C = c_count;
    J->c_base = c_base;
    J->c_total = p->C;
    // complex beams: every sample; powers: the samples of whole (and carried-out) windows
    J->t_tiles = core.cpx ? (T + core.nt - 1) / core.nt : ((T_o + partial) * p->t_int + core.nt - 1) / core.nt;
    J->mt = f.m_pad / kRowsPerMTile;
    J->kb = f.kb;
    J->ke = f.ke;
    J->T = T;
    J->T_o = T_o;
    J->B = p->B;
    J->b_pad = f.b_pad;
    J->t_shift = t_shift;
    const int rem = (2 * p->N) % f.ke;   // operand elements in a partly padded last K block
    const int per_step = f.ke / 4;       // elements per MMA k-step (16 x 16-bit or 32 x 8-bit = 32 bytes)
    J->ks_last = rem ? (rem + per_step - 1) / per_step : 4;
    const uint32_t fmt = (f.op == kOpBF16) ? 1u : 0u;
    J->idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(core.nt >> 3) << 17) |
               ((uint32_t)(kRowsPerMTile >> 4) << 24);
    J->wscale = f.qmax > 0.f ? p->d_wscale : nullptr;
    J->wsig = p->d_wsig;
    J->out = out;
    J->acc_in = t_shift > 0 ? acc_in : nullptr;
    J->acc_out = partial ? acc_out : nullptr;
    const bool work = core.cpx ? T > 0 : (T_o + partial) > 0;
    J->units = work ? (long long)c_count * J->t_tiles * J->mt : 0;
    if (J->units >= (1LL << 31)) {
        J->units = 0;
        return set_error(BF_ERR_UNSUPPORTED, "a job of 2^31 or more tiles (split its channels)");
    }
    if (J->units > 0) {
        if (T == 0) {   // nothing to read: the carried sum passes straight through
            J->units = 0;
            return set_error(BF_ERR_ARG, "a chunk with no samples cannot continue a window");
        }
        if (!encode_voltage_map(&J->xmap, x_mma, 2 * p->N, T, c_count, f.es, f.ke, core.nt))
            return set_error(BF_ERR_ARG, "voltage tensor map rejected (pointer or row stride not 16-byte aligned?)");
        if (!encode_weight_map(&J->wmap, p->d_w, f.k_pad, f.m_pad, p->C, f.es, f.ke))
            return set_error(BF_ERR_CUDA, "weight tensor map rejected");
    }
    return BF_OK;
}

long long batch_index(BatchJob *jobs, int n)
{
    long long u = 0;
    for (int j = 0; j < n; ++j) {
        jobs[j].unit0 = u;
        u += jobs[j].units;
    }
    return u;
}

static cudaError_t core_launch(const BatchCore &core, const BatchJob *d_jobs, const ParamJobs &pj, int n,
                               long long total_units, unsigned *d_err, unsigned long long *d_next, cudaStream_t s)
{
    if (total_units == 0) return cudaSuccess;
    if (d_next) {
        cudaError_t e = cudaMemsetAsync(d_next, 0, sizeof(unsigned long long), s);   // the launch takes units from 0
        if (e != cudaSuccess) return e;
    }
    BatchArgs ka;
    ka.jobs = d_jobs;
    ka.n_jobs = n;
    ka.total_units = total_units;
    ka.nt = core.nt;
    ka.nsplit = core.nsplit;
    ka.wpt = core.wpt;
    ka.t_int = core.t_int;
    ka.xst = core.xst;
    ka.nacc = core.nacc;
    ka.stage_bytes = (uint32_t)batch_stage_bytes(core.nt);
    ka.err = d_err;
    ka.next = d_next;
    const int grid = (int)std::min<long long>(core.num_sms, total_units);
    return batch_dispatch(core, BatchLaunch{ka, pj, grid, core.smem, s});
}

cudaError_t batch_core_launch(const BatchCore &core, const BatchJob *d_jobs, int n, long long total_units,
                              unsigned *d_err, unsigned long long *d_next, cudaStream_t s)
{
    static const ParamJobs unused{};
    return core_launch(core, d_jobs, unused, n, total_units, d_err, d_next, s);
}

cudaError_t batch_core_launch_params(const BatchCore &core, const BatchJob *jobs, int n, long long total_units,
                                     unsigned *d_err, unsigned long long *d_next, cudaStream_t s)
{
    if (n < 1 || n > kParamJobs) return cudaErrorInvalidValue;
    ParamJobs pj;
    memcpy((void *)pj.j, (const void *)jobs, sizeof(BatchJob) * n);
    return core_launch(core, nullptr, pj, n, total_units, d_err, d_next, s);
}

cudaError_t batch_core_launch_one(const BatchCore &core, const BatchJob &job, unsigned *d_err, cudaStream_t s)
{
    BatchJob j = job;
    j.unit0 = 0;
    return batch_core_launch_params(core, &j, 1, j.units, d_err, nullptr, s);
}

}  // namespace bfi

using namespace bfi;

// Branches of a step for the resident-weight launches: jobs of fewer than 4
// K blocks run their plan's own kernel (weights resident in shared memory,
// each voltage tile serving a group of M tiles), several at a time, so the
// tail of one fills with the CTAs of the next.
constexpr int kBranches = 4;

// Units per CTA from which a streamed-weight job of a batch step gets a
// launch of its own (about 100 microseconds of work or more, against a few
// for a launch in a graph).
constexpr long long kOwnLaunchRounds = 64;

struct bf_batch {
    std::vector<bf_plan *> plans;
    int n = 0;
    BatchCore core;
    std::vector<char> resident;   // job -> runs the plan's resident-weight kernel, not the persistent launch
    std::vector<float *> out;
    cudaStream_t branch[kBranches] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kBranches] = {};
    BatchJob *h_jobs = nullptr;   // pinned [2n]: the table, then the shared launch's rows (a captured copy reads them at replay)
    std::vector<int> slot;        // job -> its row of the table (rows in order of decreasing K)
    BatchJob *d_jobs = nullptr;
    std::vector<void *> expand_buf;   // per job, FP16 copies of 8/4-bit inputs
    std::vector<size_t> expand_bytes;
    std::vector<const void *> in;
    std::vector<int> n_samp;
    std::vector<char> set;
    long long total_units = 0;
    double flops = 0.0;
    cudaStream_t last_stream = nullptr;
    bool launched = false;   // a step was enqueued on last_stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    unsigned *d_err = nullptr;
    unsigned long long *d_next = nullptr;   // work counter of the persistent launch
};

static void batch_free(bf_batch *b)
{
    if (!b) return;
    if (b->launched) cudaStreamSynchronize(b->last_stream);
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->h_jobs) cudaFreeHost(b->h_jobs);
    if (b->d_jobs) cudaFree(b->d_jobs);
    if (b->d_err) cudaFree(b->d_err);
    if (b->d_next) cudaFree(b->d_next);
    for (void *p : b->expand_buf)
        if (p) cudaFree(p);
    for (int k = 0; k < kBranches; ++k) {
        if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    delete b;
}

static void drop_graph(bf_batch *b)
{
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
}

extern "C" {

bf_status bf_batch_create(bf_batch **out, bf_plan *const *plans, int n_plans, int tile_t)
{
    clear_error();
    if (!out) return set_error(BF_ERR_ARG, "out is NULL");
    *out = nullptr;
    for (int i = 0; plans && i < n_plans; ++i) {
        if (plans[i] && plans[i]->layout != BF_LAYOUT_CTN)   // the kernel reads [C][T][N] voltages as given
            return set_error(BF_ERR_UNSUPPORTED, "batches take the CTN layout");
        if (plans[i] && plans[i]->wbufs != 1)   // the batch keeps the plans' weight pointers
            return set_error(BF_ERR_UNSUPPORTED, "plans with double-buffered weights cannot join a batch");
    }
    BatchCore core;
    bf_status st = batch_core_init(&core, plans, n_plans, tile_t);
    if (st != BF_OK) return st;
    bf_batch *b = new bf_batch();
    b->plans.assign(plans, plans + n_plans);
    b->n = n_plans;
    b->core = core;
    // The launch walks the table's rows in order.  Rows are sorted by
    // decreasing K blocks (then by job): on the 48 uneven sub-array jobs a
    // launch with the long-K jobs first took 80 ms against 84-86 ms in the
    // callers' order and 87 ms with the short-K jobs first.  The order only
    // changes which units run when; each job still writes its own outputs.
    std::vector<int> order(n_plans);
    for (int i = 0; i < n_plans; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return plans[x]->wf.kb > plans[y]->wf.kb; });
    b->slot.assign(n_plans, 0);
    for (int r = 0; r < n_plans; ++r) b->slot[order[r]] = r;
    cudaError_t e;
    // pinned table: the rows, then as many staging rows for the shared launch's upload
    if ((e = cudaHostAlloc((void **)&b->h_jobs, 2 * sizeof(BatchJob) * n_plans, cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_jobs, sizeof(BatchJob) * n_plans)) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_err, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_next, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMemset(b->d_err, 0, sizeof(unsigned))) != cudaSuccess) {
        batch_free(b);
        return cuda_error(e, "batch allocation");
    }
    b->resident.assign(n_plans, 0);
    bool any_resident = false;
    for (int j = 0; j < n_plans; ++j) any_resident |= (b->resident[j] = !plans[j]->tc.stream) != 0;
    if (any_resident) {
        if ((e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) != cudaSuccess) {
            batch_free(b);
            return cuda_error(e, "batch event");
        }
        for (int k = 0; k < kBranches; ++k)
            if ((e = cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming)) != cudaSuccess) {
                batch_free(b);
                return cuda_error(e, "batch branch stream");
            }
    }
    b->out.assign(n_plans, nullptr);
    memset((void *)b->h_jobs, 0, 2 * sizeof(BatchJob) * n_plans);
    b->expand_buf.assign(n_plans, nullptr);
    b->expand_bytes.assign(n_plans, 0);
    b->in.assign(n_plans, nullptr);
    b->n_samp.assign(n_plans, 0);
    b->set.assign(n_plans, 0);
    *out = b;
    return BF_OK;
}

bf_status bf_batch_set(bf_batch *b, int job, const void *x, int T, float *out)
{
    clear_error();
    if (!b) return set_error(BF_ERR_ARG, "batch is NULL");
    if (job < 0 || job >= b->n) return set_error(BF_ERR_ARG, "job index out of range");
    if (T < 0) return set_error(BF_ERR_ARG, "n_samp must be >= 0");
    bf_plan *p = b->plans[job];
    const int T_o = T / p->t_int;
    if (T_o > 0 && (!x || !out)) return set_error(BF_ERR_ARG, "NULL voltage or output pointer");
    if (((uintptr_t)x & 15) || ((uintptr_t)out & 15))
        return set_error(BF_ERR_ARG, "voltages and powers must be 16-byte aligned");
    if (b->launched) {
        cudaError_t e = cudaStreamSynchronize(b->last_stream);   // the table may be read by a copy in flight
        if (e != cudaSuccess) return cuda_error(e, "batch synchronize");
    }
    drop_graph(b);   // a captured step refers to the old inputs
    const void *xin = x;
    // FP16 widening of 8/4-bit inputs for the persistent launch, and for
    // resident-weight jobs whose rows TMA cannot read raw
    const bool expand = (p->dtype == BF_CI8 || p->dtype == BF_CI4) && (!b->resident[job] || p->tc.raw_kb == 0);
    if (expand && T_o > 0) {
        const size_t need = (size_t)p->C * T * p->N * 4;
        if (b->expand_bytes[job] < need) {
            if (b->expand_buf[job]) cudaFree(b->expand_buf[job]);
            b->expand_buf[job] = nullptr;
            b->expand_bytes[job] = 0;
            cudaError_t e = cudaMalloc(&b->expand_buf[job], need);
            if (e != cudaSuccess) return cuda_error(e, "batch expansion buffer");
            b->expand_bytes[job] = need;
        }
        xin = b->expand_buf[job];
    }
    BatchJob J;
    if (b->resident[job]) {
        memset((void *)&J, 0, sizeof(J));   // no units in the persistent launch
    } else {
        bf_status st = batch_fill_job(b->core, &J, p, xin, T, out, 0, nullptr, nullptr);
        if (st != BF_OK) return st;
    }
    b->h_jobs[b->slot[job]] = J;
    b->in[job] = x;
    b->out[job] = out;
    b->n_samp[job] = T;
    b->set[job] = 1;
    b->total_units = batch_index(b->h_jobs, b->n);
    double fl = 0.0;
    for (int j = 0; j < b->n; ++j)
        if (b->set[j]) {
            const bf_plan *q = b->plans[j];
            fl += 8.0 * q->N * q->B * q->C * (double)b->n_samp[j];
        }
    b->flops = fl;
    return BF_OK;
}

bf_status bf_batch_execute(bf_batch *b, void *stream)
{
    clear_error();
    if (!b) return set_error(BF_ERR_ARG, "batch is NULL");
    for (int j = 0; j < b->n; ++j)
        if (!b->set[j]) return set_error(BF_ERR_STATE, "every job needs bf_batch_set before execute");
    cudaStream_t s = (cudaStream_t)stream;
    // resident-weight jobs with whole windows, most work first
    std::vector<int> res;
    for (int j = 0; j < b->n; ++j)
        if (b->resident[j] && b->n_samp[j] / b->plans[j]->t_int > 0) res.push_back(j);
    if (b->total_units == 0 && res.empty()) return BF_OK;
    auto work = [&](int j) { return (double)b->plans[j]->N * b->plans[j]->B * b->plans[j]->C * b->n_samp[j]; };
    std::stable_sort(res.begin(), res.end(), [&](int x, int y) { return work(x) > work(y); });
    b->last_stream = s;
    b->launched = true;
    cudaError_t e;
    auto expand_into = [&](int j, cudaStream_t st) -> cudaError_t {
        const bf_plan *p = b->plans[j];
        return launch_expand_to_f16(b->in[j], p->dtype, b->expand_buf[j], (long long)p->C * b->n_samp[j] * p->N, p->N,
                                    st);
    };
    auto is_int = [&](int j) { return b->plans[j]->dtype == BF_CI8 || b->plans[j]->dtype == BF_CI4; };
    if (!res.empty()) {
        // fork: each job goes to the branch with the least work so far
        if ((e = cudaEventRecord(b->ev_fork, s)) != cudaSuccess) return cuda_error(e, "batch fork");
        double load[kBranches] = {};
        bool used[kBranches] = {};
        bf_status st = BF_OK;
        for (int j : res) {
            int k = 0;
            for (int i = 1; i < kBranches; ++i)
                if (load[i] < load[k]) k = i;
            load[k] += work(j);
            cudaStream_t bs = b->branch[k];
            if (!used[k]) {
                if ((e = cudaStreamWaitEvent(bs, b->ev_fork, 0)) != cudaSuccess) {
                    st = cuda_error(e, "batch fork");
                    break;
                }
                used[k] = true;
            }
            bf_plan *p = b->plans[j];
            const void *xin = b->in[j];
            if (is_int(j) && p->tc.raw_kb == 0) {
                if ((e = expand_into(j, bs)) != cudaSuccess) {
                    st = cuda_error(e, "integer expansion");
                    break;
                }
                xin = b->expand_buf[j];
            }
            TcArgs ta;
            ta.x = xin;
            ta.c_base = 0;
            ta.c_launch = p->C;
            ta.c_total = p->C;
            ta.T = b->n_samp[j];
            ta.T_o = b->n_samp[j] / p->t_int;
            ta.t_int = p->t_int;
            ta.complex_out = 0;
            ta.out = b->out[j];
            ta.err = b->d_err;
            std::string why;
            if ((e = launch_tc(p, ta, bs, &why)) != cudaSuccess) {
                st = why.empty() ? cuda_error(e, "tensor-core kernel (batch job)")
                                 : set_error(BF_ERR_CUDA, "tensor-core kernel (batch job): " + why);
                break;
            }
        }
        // join (also after a failure, so `stream` still covers what was enqueued)
        for (int k = 0; k < kBranches; ++k) {
            if (!used[k]) continue;
            if ((e = cudaEventRecord(b->ev_join[k], b->branch[k])) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s, b->ev_join[k], 0)) != cudaSuccess) {
                if (st == BF_OK) st = cuda_error(e, "batch join");
            }
        }
        if (st != BF_OK) return st;
    }
    if (b->total_units == 0) return BF_OK;
    for (int j = 0; j < b->n; ++j)
        if (!b->resident[j] && b->h_jobs[b->slot[j]].units > 0 && is_int(j))
            if ((e = expand_into(j, s)) != cudaSuccess) return cuda_error(e, "integer expansion");
    // Jobs of at least kOwnLaunchRounds units per CTA get a launch of their
    // own, one after another on the fixed stride: a kernel boundary starts
    // every CTA on the job together, so the units in flight stay within a
    // channel or two.  The rest share one launch on the work counter.
    std::vector<BatchJob> rows;
    long long shared_units = 0;
    for (int r = 0; r < b->n; ++r) {
        BatchJob J = b->h_jobs[r];
        if (J.units == 0) continue;
        if (J.units >= kOwnLaunchRounds * (long long)b->core.num_sms) {
            if ((e = batch_core_launch_one(b->core, J, b->d_err, s)) != cudaSuccess)
                return cuda_error(e, "batched tensor-core kernel");
            continue;
        }
        J.unit0 = shared_units;
        shared_units += J.units;
        rows.push_back(J);
    }
    if (rows.empty()) return BF_OK;
    if ((int)rows.size() <= kParamJobs) {
        e = batch_core_launch_params(b->core, rows.data(), (int)rows.size(), shared_units, b->d_err, b->d_next, s);
    } else {
        BatchJob *dst = b->h_jobs + b->n;   // the staging rows behind the table
        std::copy(rows.begin(), rows.end(), dst);
        e = cudaMemcpyAsync(b->d_jobs, dst, sizeof(BatchJob) * rows.size(), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_error(e, "batch table upload");
        e = batch_core_launch(b->core, b->d_jobs, (int)rows.size(), shared_units, b->d_err, b->d_next, s);
    }
    if (e != cudaSuccess) return cuda_error(e, "batched tensor-core kernel");
    return BF_OK;
}

bf_status bf_batch_capture(bf_batch *b, void *stream)
{
    clear_error();
    if (!b) return set_error(BF_ERR_ARG, "batch is NULL");
    if (!stream) return set_error(BF_ERR_ARG, "capture needs a non-default stream");
    cudaStream_t s = (cudaStream_t)stream;
    drop_graph(b);
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_error(e, "begin capture");
    const bool was = b->launched;
    bf_status st = bf_batch_execute(b, stream);
    b->launched = was;   // nothing ran yet
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (st != BF_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_error(e, "end capture");
    e = cudaGraphInstantiate(&b->graph_exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_error(e, "graph instantiate");
    }
    b->graph = g;
    return BF_OK;
}

bf_status bf_batch_replay(bf_batch *b, void *stream)
{
    clear_error();
    if (!b) return set_error(BF_ERR_ARG, "batch is NULL");
    if (!b->graph_exec) return set_error(BF_ERR_STATE, "no captured step (bf_batch_capture first)");
    cudaError_t e = cudaGraphLaunch(b->graph_exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_error(e, "graph launch");
    b->last_stream = (cudaStream_t)stream;
    b->launched = true;
    return BF_OK;
}

bf_status bf_batch_sync(bf_batch *b)
{
    clear_error();
    if (!b) return set_error(BF_ERR_ARG, "batch is NULL");
    cudaError_t e = b->launched ? cudaStreamSynchronize(b->last_stream) : cudaSuccess;
    if (e != cudaSuccess) return cuda_error(e, "batch synchronize");
    unsigned err = 0;
    e = cudaMemcpy(&err, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "read status word");
    if (err) {
        cudaMemset(b->d_err, 0, sizeof(unsigned));
        return set_error(BF_ERR_TIMEOUT, "a device-side wait of the batched kernel timed out");
    }
    return BF_OK;
}

bf_status bf_batch_query(const bf_batch *b, int *tile_t, long long *units, double *flops)
{
    clear_error();
    if (!b) return set_error(BF_ERR_ARG, "batch is NULL");
    if (tile_t) *tile_t = b->core.nt;
    if (units) *units = b->total_units;
    if (flops) *flops = b->flops;
    return BF_OK;
}

bf_status bf_batch_destroy(bf_batch *b)
{
    clear_error();
    batch_free(b);
    return BF_OK;
}

}  // extern "C"
