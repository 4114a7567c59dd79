// Resident-weight tensor-core beamformer: the variants for 4-bit complex integer voltages (widened in the kernel).
#include "k_tc_kernel.cuh"

namespace bfi {

template cudaError_t launch_tc_family<false, BF_CI4>(const CUtensorMap &, const CUtensorMap &, const TcKernelArgs &, int,
                                                 bool, int, int, cudaStream_t);

}  // namespace bfi
