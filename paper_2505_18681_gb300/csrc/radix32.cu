// Onesweep pass kernels for 32-bit keys (int32, uint32, float32).
#include "radix_launch.cuh"

namespace evosort {

cudaError_t launch_onesweep_u32(bool pairs, int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                const RadixArgs& a, int pass) {
    return pairs ? launch_onesweep_shape<uint32_t, true>(block, kpt, rank, grid, sms, s, a, pass)
                 : launch_onesweep_shape<uint32_t, false>(block, kpt, rank, grid, sms, s, a, pass);
}

}  // namespace evosort
