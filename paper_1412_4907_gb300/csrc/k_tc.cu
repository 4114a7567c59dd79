// Host side of the resident-weight tensor-core beamformer (the kernel and its
// structure: k_tc_kernel.cuh): tile choice, shared-memory layout checks and
// the launch.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "bf_internal.h"
#include "k_tc.h"
#include "tc_common.cuh"

namespace bfi {

// ----------------------------------------------------------------- host side
static int gcd_i(int x, int y)
{
    while (y) {
        int t = x % y;
        x = y;
        y = t;
    }
    return x;
}

static int stage_bytes() { return kStageDepth * kBeamsPerMTile * kMaxWinPerTile * (int)sizeof(float); }
static int ctrl_bytes() { return 8 * (3 * kMaxXStages + 2 * kMaxAcc + 1 + 2 * 16 + 2 * kStageDepth) + 16; }

// End of the kernel's shared-memory layout for a configuration, computed the
// way the kernel computes its offsets (1024 bytes of alignment slack, voltage
// stages, resident weight slots, the raw tile of integer inputs, staging ring,
// barriers, TMEM holder and abort flag).
static size_t layout_end(const TcConfig &c, int kb)
{
    const size_t x_stage = (size_t)kb * c.nt * 128;
    const size_t gmax = (size_t)c.group;
    const size_t w_slot = (size_t)kb * 16384;
    const size_t raw_tile = (size_t)kb * c.nt * c.raw_kb;
    return 1024 + (size_t)c.xst * x_stage + raw_tile + gmax * w_slot + (size_t)stage_bytes() +
           8 * (size_t)(3 * kMaxXStages + 2 * kMaxAcc + 1 + 2 * gmax + 2 * kStageDepth) + 8;
}

static bool layout_ok(const TcConfig &c, int kb)
{
    return !c.stream && layout_end(c, kb) <= (size_t)c.smem && c.smem <= kSmemLimit && c.xst >= 2 &&
           c.xst <= kMaxXStages && c.group <= 16 && c.nt >= 16 && c.nt <= 256 && c.nt % 16 == 0;
}

bool tc_choose(bf_plan *p, const TcRequest &req, TcConfig *cfg, std::string *why)
{
    const WeightFormat &f = p->wf;
    const int t_int = p->t_int;
    const long long unit = 16LL / gcd_i(16, t_int) * t_int;   // lcm(16, T_int)
    if (unit > 256) {
        *why = "tensor-core kernel needs lcm(16, T_int) <= 256";
        return false;
    }
    const int mt = f.m_pad / kRowsPerMTile;
    // 8/4-bit inputs are widened inside the kernel when TMA can read their
    // rows (a row stride that is a multiple of 16 bytes); otherwise they are
    // widened to FP16 in a pass before the kernel
    int raw_kb = 0;
    if (p->dtype == BF_CI8 && (2 * p->N) % 16 == 0) raw_kb = 64;
    if (p->dtype == BF_CI4 && p->N % 16 == 0) raw_kb = 32;
    if (f.kb >= 4) {
        // many antennas: the weights do not stay resident; the batched kernel's
        // streamed pipeline (k_batch.cu, one job) runs the plan with this tile
        // width and sizes its own stages (a weight and a voltage K block each)
        for (int nt = 256; nt >= (int)unit; nt -= 16) {
            if (nt % unit) continue;
            if (req.tile_t && nt != req.tile_t) continue;
            if (nt / t_int > kMaxWinPerTile) continue;
            TcConfig c;
            c.stream = true;
            c.nt = nt;
            c.xst = 0;
            c.nsplit = ((nt / 2) % 16 == 0 && (nt / 2) % t_int == 0) ? 2 : 1;
            c.fast_windows = (t_int % 16) == 0;
            c.n_groups = 1;
            c.group = mt;
            c.smem = 0;
            *cfg = c;
            return true;
        }
        *why = "requested tile configuration does not fit the streamed tensor-core pipeline";
        return false;
    }
    for (int nt = 256; nt >= (int)unit; nt -= 16) {
        if (nt % unit) continue;
        if (req.tile_t && nt != req.tile_t) continue;
        if (nt / t_int > kMaxWinPerTile) continue;   // staged window powers per tile
        const int x_stage = f.kb * nt * 128;
        const int raw_tile = f.kb * nt * raw_kb;   // integer inputs: one raw tile beside the stages
        const int w_slot = f.kb * 16384;
        // default: the fewest weight groups per channel (each group re-reads the
        // voltage tile), then the most voltage stages in flight; a request fixes
        // the stage count and/or the group size
        bool found = false;
        TcConfig best;
        for (int xst = kMaxXStages; xst >= 2; --xst) {
            if (req.x_stages && xst != req.x_stages) continue;
            const int fixed = xst * x_stage + raw_tile + stage_bytes() + ctrl_bytes() + 1024;
            const int avail = kSmemLimit - fixed;
            if (avail < w_slot) continue;
            int g = std::min(mt, std::min(16, avail / w_slot));
            if (req.group_tiles) {
                if (req.group_tiles > g) continue;
                g = req.group_tiles;
            }
            TcConfig c;
            c.nt = nt;
            c.xst = xst;
            c.raw_kb = raw_kb;
            c.nsplit = ((nt / 2) % 16 == 0 && (nt / 2) % t_int == 0) ? 2 : 1;
            c.fast_windows = (t_int % 16) == 0;
            c.n_groups = (mt + g - 1) / g;
            const int g_base = mt / c.n_groups, g_rem = mt % c.n_groups;
            c.group = g_base + (g_rem ? 1 : 0);
            c.smem = std::max(fixed + c.group * w_slot, 116 * 1024);   // one CTA per SM: it owns all TMEM
            if (!found || c.n_groups < best.n_groups) {
                best = c;
                found = true;
            }
        }
        if (!found) continue;
        if (!layout_ok(best, f.kb)) {
            *why = "internal tiling inconsistency (shared-memory layout exceeds the allocation)";
            return false;
        }
        *cfg = best;
        return true;
    }
    *why = (req.tile_t || req.x_stages || req.group_tiles)
               ? "requested tile configuration does not fit the tensor-core kernel"
               : "antenna count too large for the resident-weight tensor-core kernel";
    return false;
}

cudaError_t launch_tc(bf_plan *p, const TcArgs &ta, cudaStream_t s, std::string *why)
{
    const WeightFormat &f = p->wf;
    const TcConfig &cfg = p->tc;
    if (ta.T == 0 || ta.c_launch == 0) return cudaSuccess;
    if (cfg.stream) {   // callers send streamed-weight plans to the batched pipeline
        *why = "plan has streamed weights (K >= 4 blocks): not a resident-weight launch";
        return cudaErrorInvalidConfiguration;
    }
    CUtensorMap xm, wm;
    const bool widen = cfg.raw_kb > 0;   // raw integer samples, widened in the kernel
    const int row_bytes = p->N * (p->dtype == BF_CI8 ? 2 : 1);
    if (widen ? !encode_raw_map(&xm, ta.x, row_bytes, ta.T, ta.c_launch, cfg.raw_kb, cfg.nt)
              : !encode_voltage_map(&xm, ta.x, 2 * p->N, ta.T, ta.c_launch, f.es, f.ke, cfg.nt)) {
        *why = "voltage tensor map rejected (pointer or row stride not 16-byte aligned?)";
        return cudaErrorInvalidValue;
    }
    if (!encode_weight_map(&wm, p->d_w, f.k_pad, f.m_pad, p->C, f.es, f.ke)) {
        *why = "weight tensor map rejected";
        return cudaErrorInvalidValue;
    }
    TcKernelArgs ka;
    const int mt = f.m_pad / kRowsPerMTile;
    ka.n_groups = cfg.n_groups;
    ka.g_base = mt / cfg.n_groups;
    ka.g_rem = mt % cfg.n_groups;
    ka.gmax = cfg.group;
    // power output needs the samples of whole windows only (the tail is dropped)
    const int t_used = ta.complex_out ? ta.T : ta.T_o * ta.t_int;
    ka.t_tiles = (t_used + cfg.nt - 1) / cfg.nt;
    ka.ct_total = (long long)ta.c_launch * ka.t_tiles;
    ka.nt = cfg.nt;
    ka.kb = f.kb;
    ka.ke = f.ke;
    ka.nsplit = cfg.nsplit;
    ka.wpt = cfg.nt / ta.t_int;
    ka.xst = cfg.xst;
    ka.nacc = std::min(kMaxAcc, kTmemCols / cfg.nt) & ~1;   // even: each group keeps its own accumulators
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
    ka.wscale = f.qmax > 0.f ? p->d_wscale : nullptr;   // unscaled formats multiply by 1
    ka.wsig = p->d_wsig;
    ka.out = ta.out;
    ka.err = ta.err ? ta.err : p->d_err;
    ka.raw_kb = cfg.raw_kb;
    ka.raw_stage_bytes = (uint32_t)(f.kb * cfg.nt * cfg.raw_kb);
    if (ka.ct_total == 0) return cudaSuccess;
    if (!layout_ok(cfg, f.kb) || ka.gmax != cfg.group) {   // final guard before launch
        *why = "internal tiling inconsistency (shared-memory layout exceeds the allocation)";
        return cudaErrorInvalidConfiguration;
    }
    // sets of gq CTAs hold different weight groups and walk the same range in step
    ka.gq = std::min(cfg.n_groups, p->num_sms);
    const long long n_sets = std::max<long long>(1, std::min<long long>(p->num_sms / ka.gq, ka.ct_total));
    const int grid = (int)(n_sets * ka.gq);
    const bool f8 = f.op == kOpE4M3;
    const int win = (ta.t_int == 64 || ta.t_int == 32 || ta.t_int == 16) ? ta.t_int : (ta.t_int % 16 == 0 ? 0 : -1);
    const bool cpx = ta.complex_out != 0;
    if (f8) return launch_tc_family<true, 0>(xm, wm, ka, win, cpx, grid, cfg.smem, s);
    switch (widen ? p->dtype : 0) {
    case BF_CI8: return launch_tc_family<false, BF_CI8>(xm, wm, ka, win, cpx, grid, cfg.smem, s);
    case BF_CI4: return launch_tc_family<false, BF_CI4>(xm, wm, ka, win, cpx, grid, cfg.smem, s);
    default: return launch_tc_family<false, 0>(xm, wm, ka, win, cpx, grid, cfg.smem, s);
    }
}

}  // namespace bfi
