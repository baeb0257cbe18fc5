// Instantiation table of the onesweep pass kernel.  Each key width gets its own
// translation unit (radix32.cu, radix64.cu) so the two compile in parallel.
#pragma once

#include "radix.cuh"

namespace evosort {

// (threads per CTA, keys per thread) pairs compiled into the library.
#define EVOSORT_TILE_SHAPES(X) \
    X(256, 8)                  \
    X(256, 16)                 \
    X(512, 8)                  \
    X(512, 16)                 \
    X(256, 24)

template <typename U, bool PAIRS, int BLOCK, int KPT, int MAXB, int RANK>
cudaError_t launch_onesweep_inst(size_t grid, int sms, cudaStream_t s, const RadixArgs& a, int pass) {
    auto kern = radix_onesweep<U, PAIRS, BLOCK, KPT, MAXB, RANK>;
    const size_t smem = onesweep_smem_bytes(BLOCK, KPT, (int)sizeof(U), PAIRS, a.d);
    static size_t configured = 0;   // largest dynamic smem size set so far
    static int resident[16] = {0};  // resident CTAs per SM, by digit width
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    if (resident[a.d] == 0) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BLOCK, smem);
        if (e != cudaSuccess) return e;
        resident[a.d] = nb > 0 ? nb : 1;
    }
    // persistent grid: every SM full, never more CTAs than tiles
    size_t g = (size_t)sms * resident[a.d];
    if (g > grid) g = grid;
    if (g < 1) g = 1;
    kern<<<(unsigned)g, BLOCK, smem, s>>>(a, pass);
    return cudaGetLastError();
}

template <typename U, bool PAIRS>
cudaError_t launch_onesweep_shape(int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                  const RadixArgs& a, int pass) {
    const bool wide = a.d > 8;
#define EVOSORT_CASE(B, K)                                                                        \
    if (block == B && kpt == K) {                                                                 \
        if (wide)                                                                                 \
            return rank == 2 ? launch_onesweep_inst<U, PAIRS, B, K, 11, 2>(grid, sms, s, a, pass)      \
                             : launch_onesweep_inst<U, PAIRS, B, K, 11, 1>(grid, sms, s, a, pass);     \
        return rank == 2 ? launch_onesweep_inst<U, PAIRS, B, K, 8, 2>(grid, sms, s, a, pass)           \
                         : launch_onesweep_inst<U, PAIRS, B, K, 8, 1>(grid, sms, s, a, pass);          \
    }
    EVOSORT_TILE_SHAPES(EVOSORT_CASE)
#undef EVOSORT_CASE
    return cudaErrorInvalidConfiguration;
}

inline bool onesweep_shape_supported(int block, int kpt) {
#define EVOSORT_CASE(B, K) \
    if (block == B && kpt == K) return true;
    EVOSORT_TILE_SHAPES(EVOSORT_CASE)
#undef EVOSORT_CASE
    return false;
}

// True if the tile shape is compiled in and its shared memory fits a CTA.
inline bool onesweep_config_fits(int w, bool pairs, int block, int kpt, int d) {
    return onesweep_shape_supported(block, kpt) && onesweep_smem_bytes(block, kpt, w, pairs, d) <= kMaxDynSmem;
}

// Defined in radix32.cu / radix64.cu.
cudaError_t launch_onesweep_u32(bool pairs, int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                const RadixArgs& a, int pass);
cudaError_t launch_onesweep_u64(bool pairs, int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                const RadixArgs& a, int pass);
cudaError_t launch_radix_aux(int w, int which, size_t grid, size_t smem, cudaStream_t s, const RadixArgs& a,
                             int inplace);

}  // namespace evosort
