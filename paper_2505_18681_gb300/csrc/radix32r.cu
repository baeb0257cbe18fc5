// Register-tile onesweep pass kernels (onesweep_reg.cuh): 32-bit keys, keys
// only and key/value pairs.
#include "onesweep_reg.cuh"
#include "radix_launch.cuh"

namespace evosort {

cudaError_t launch_onesweep_reg_u32(bool pairs, int block, int kpt, int rank, size_t grid, int sms,
                                    cudaStream_t s, const RadixArgs& a, int pass) {
#define EVOSORT_CASE(B, K) \
    if (!pairs && block == B && kpt == K) return launch_reg_rank<uint32_t, false, B, K>(rank, grid, sms, s, a, pass);
    EVOSORT_REG_SHAPES_U32_KEYS(EVOSORT_CASE)
#undef EVOSORT_CASE
#define EVOSORT_CASE(B, K) \
    if (pairs && block == B && kpt == K) return launch_reg_rank<uint32_t, true, B, K>(rank, grid, sms, s, a, pass);
    EVOSORT_REG_SHAPES_U32_PAIRS(EVOSORT_CASE)
#undef EVOSORT_CASE
    return cudaErrorInvalidConfiguration;
}

}  // namespace evosort
