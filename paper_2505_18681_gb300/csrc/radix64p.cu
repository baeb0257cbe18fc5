// Onesweep pass kernels: 64-bit keys, key/value pairs.
#include "radix_launch.cuh"

namespace evosort {

cudaError_t launch_onesweep_u64_pairs(int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                  const RadixArgs& a, int pass) {
    return launch_onesweep_shape<uint64_t, true>(block, kpt, rank, grid, sms, s, a, pass);
}

}  // namespace evosort
