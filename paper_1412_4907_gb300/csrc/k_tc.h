// Kernel arguments of the resident-weight tensor-core beamformer and the
// launcher of its variants (k_tc_kernel.cuh holds the kernel; each of
// k_tc_f16.cu, k_tc_f8.cu, k_tc_i8.cu and k_tc_i4.cu compiles one family, so
// the variants build in parallel).
#pragma once
#include <cudaTypedefs.h>

#include "bf_internal.h"

namespace bfi {

struct TcKernelArgs {
    long long ct_total;                 // channels x time tiles
    int n_groups, g_base, g_rem, gmax;  // weight groups of M tiles
    int gq;                             // CTAs per set (distinct groups walked in step)
    int t_tiles, nt, kb, ke, nsplit, wpt, xst;   // xst: voltage stages in flight
    int nacc;                                    // TMEM accumulators in flight
    int c_base, c_total, T, T_o, t_int, B, b_pad;
    uint32_t idesc;
    uint32_t x_stage_bytes, w_slot_bytes;
    const float *wscale;   // [C][b_pad] sigma^2
    const float *wsig;     // [C][b_pad] sigma
    float *out;
    unsigned *err;
    uint32_t raw_stage_bytes;   // 8/4-bit inputs: raw bytes of one voltage tile (kb x nt x raw_kb), else 0
    int raw_kb;                 // raw bytes of one K block per sample row (64 int8, 32 4-bit)
};

// Launches the variant for window specialisation win (16, 32, 64 = T_int;
// 0 = any multiple of 16; -1 = any), output kind (complex beams or powers)
// and epilogue, within the family of operand format F8 (FP8 E4M3 operands)
// and input kind IN (BF_CI8 / BF_CI4: 8/4-bit samples widened in the kernel;
// 0: FP16/BF16/FP8 voltages by TMA).
template <bool F8, int IN>
cudaError_t launch_tc_family(const CUtensorMap &xm, const CUtensorMap &wm, const TcKernelArgs &ka, int win, bool cpx,
                             int grid, int smem, cudaStream_t s);

extern template cudaError_t launch_tc_family<false, 0>(const CUtensorMap &, const CUtensorMap &, const TcKernelArgs &,
                                                       int, bool, int, int, cudaStream_t);
extern template cudaError_t launch_tc_family<true, 0>(const CUtensorMap &, const CUtensorMap &, const TcKernelArgs &,
                                                      int, bool, int, int, cudaStream_t);
extern template cudaError_t launch_tc_family<false, BF_CI8>(const CUtensorMap &, const CUtensorMap &,
                                                            const TcKernelArgs &, int, bool, int, int, cudaStream_t);
extern template cudaError_t launch_tc_family<false, BF_CI4>(const CUtensorMap &, const CUtensorMap &,
                                                            const TcKernelArgs &, int, bool, int, int, cudaStream_t);

}  // namespace bfi
