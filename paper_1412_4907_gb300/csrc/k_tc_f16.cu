// Resident-weight tensor-core beamformer: the variants for FP16 and BF16 voltages.
#include "k_tc_kernel.cuh"

namespace bfi {

template cudaError_t launch_tc_family<false, 0>(const CUtensorMap &, const CUtensorMap &, const TcKernelArgs &, int,
                                                 bool, int, int, cudaStream_t);

}  // namespace bfi
