// Host helpers shared by the tensor-core launchers: K-major 3-D TMA tensor
// maps with the 128-byte swizzle.
#pragma once
#include <cudaTypedefs.h>

#include "bf_internal.h"

namespace bfi {

// The driver's tensor-map encoder (fetched once through the runtime), or NULL.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// Voltages [C][T][2N] read in boxes of ke x nt x 1 elements.
bool encode_voltage_map(CUtensorMap *m, const void *x, int two_n, int T, int C, int es, int ke, int nt);

// Weight rows [C][M_pad][K_pad] read in boxes of ke x 128 x 1 elements.
bool encode_weight_map(CUtensorMap *m, const void *w, int k_pad, int m_pad, int C, int es, int ke);

// Raw 8/4-bit voltages [C][T][row_bytes] read unswizzled in boxes of
// box_bytes x nt x 1 bytes (row_bytes and box_bytes multiples of 16).
bool encode_raw_map(CUtensorMap *m, const void *x, int row_bytes, int T, int C, int box_bytes, int nt);

}  // namespace bfi
