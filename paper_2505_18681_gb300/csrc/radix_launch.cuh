// Instantiation table of the onesweep pass kernel.  Each (key width, pairs)
// combination has its own translation unit so they compile in parallel.
#pragma once

#include "radix.cuh"

namespace evosort {

// (threads per CTA, keys per thread) pairs compiled into the library.
#define EVOSORT_TILE_SHAPES(X) \
    X(256, 8)                  \
    X(256, 16)                 \
    X(1024, 4)                 \
    X(512, 8)                  \
    X(512, 16)                 \
    X(512, 32)                 \
    X(1024, 8)                 \
    X(1024, 16)

template <typename U, bool PAIRS, int BLOCK, int KPT, int D, int RANK>
cudaError_t launch_onesweep_inst(size_t grid, int sms, cudaStream_t s, const RadixArgs& a, int pass) {
    auto kern = radix_onesweep<U, PAIRS, BLOCK, KPT, D, RANK>;
    const size_t smem = onesweep_smem_bytes(BLOCK, KPT, (int)sizeof(U), PAIRS, D, RANK);
    static int resident = 0;   // resident CTAs per SM
    if (resident == 0) {
        cudaError_t e = cudaSuccess;
        if (smem > 48 * 1024)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BLOCK, smem);
        if (e != cudaSuccess) return e;
        resident = nb > 0 ? nb : 1;
    }
    // persistent grid: every SM full, never more CTAs than tiles
    size_t g = (size_t)sms * resident;
    if (g > grid) g = grid;
    if (g < 1) g = 1;
    kern<<<(unsigned)g, BLOCK, smem, s>>>(a, pass);
    return cudaGetLastError();
}

// Digit widths 4..11 with per-bit ballot ranking; shared match-mask ranking
// for 4..8; match.any ranking for d = 8.
template <typename U, bool PAIRS, int B, int K>
cudaError_t launch_onesweep_d(int rank, size_t grid, int sms, cudaStream_t s, const RadixArgs& a, int pass) {
    if (rank == 1) {
        if (a.d == 8) return launch_onesweep_inst<U, PAIRS, B, K, 8, 1>(grid, sms, s, a, pass);
        return cudaErrorInvalidConfiguration;
    }
    if (rank == 3) {
        switch (a.d) {
            case 4: return launch_onesweep_inst<U, PAIRS, B, K, 4, 3>(grid, sms, s, a, pass);
            case 5: return launch_onesweep_inst<U, PAIRS, B, K, 5, 3>(grid, sms, s, a, pass);
            case 6: return launch_onesweep_inst<U, PAIRS, B, K, 6, 3>(grid, sms, s, a, pass);
            case 7: return launch_onesweep_inst<U, PAIRS, B, K, 7, 3>(grid, sms, s, a, pass);
            case 8: return launch_onesweep_inst<U, PAIRS, B, K, 8, 3>(grid, sms, s, a, pass);
        }
        return cudaErrorInvalidConfiguration;
    }
    switch (a.d) {
        case 4: return launch_onesweep_inst<U, PAIRS, B, K, 4, 2>(grid, sms, s, a, pass);
        case 5: return launch_onesweep_inst<U, PAIRS, B, K, 5, 2>(grid, sms, s, a, pass);
        case 6: return launch_onesweep_inst<U, PAIRS, B, K, 6, 2>(grid, sms, s, a, pass);
        case 7: return launch_onesweep_inst<U, PAIRS, B, K, 7, 2>(grid, sms, s, a, pass);
        case 8: return launch_onesweep_inst<U, PAIRS, B, K, 8, 2>(grid, sms, s, a, pass);
        case 9: return launch_onesweep_inst<U, PAIRS, B, K, 9, 2>(grid, sms, s, a, pass);
        case 10: return launch_onesweep_inst<U, PAIRS, B, K, 10, 2>(grid, sms, s, a, pass);
        case 11: return launch_onesweep_inst<U, PAIRS, B, K, 11, 2>(grid, sms, s, a, pass);
    }
    return cudaErrorInvalidConfiguration;
}

template <typename U, bool PAIRS>
cudaError_t launch_onesweep_shape(int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                  const RadixArgs& a, int pass) {
#define EVOSORT_CASE(B, K) \
    if (block == B && kpt == K) return launch_onesweep_d<U, PAIRS, B, K>(rank, grid, sms, s, a, pass);
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
inline bool onesweep_config_fits(int w, bool pairs, int block, int kpt, int d, int rank) {
    return onesweep_shape_supported(block, kpt) &&
           onesweep_smem_bytes(block, kpt, w, pairs, d, rank) <= kMaxDynSmem;
}

// Compiled ranking variants: ballot for every width, shared match masks for
// widths up to 8, match.any for 8-bit digits; adaptive (4: match masks or
// match.any, chosen per pass) for 8-bit digits.
inline bool onesweep_rank_supported(int rank, int d) {
    return rank == 2 || (rank == 1 && d == 8) || (rank == 3 && d <= 8) || (rank == 4 && d == 8);
}
inline bool onesweep_rank_fits(int rank, int block, int kpt, int w, bool pairs, int d) {
    return (rank != 3 && rank != 4) || match_masks_fit(block, kpt, w, pairs, d);
}

// Defined in radix32k.cu, radix32p.cu, radix64k.cu, radix64p.cu.
cudaError_t launch_onesweep_u32_keys(int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                     const RadixArgs& a, int pass);
cudaError_t launch_onesweep_u32_pairs(int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                      const RadixArgs& a, int pass);
cudaError_t launch_onesweep_u64_keys(int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                     const RadixArgs& a, int pass);
cudaError_t launch_onesweep_u64_pairs(int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                      const RadixArgs& a, int pass);
// Register-tile pass kernels (onesweep_reg.cuh): (threads per CTA, keys per
// thread) compiled per key width and form, 8-bit digits, rank modes 1, 3, 4.
#define EVOSORT_REG_SHAPES_U32_KEYS(X) X(1024, 16) X(512, 16)
#define EVOSORT_REG_SHAPES_U32_PAIRS(X) X(1024, 12) X(1024, 8)
#define EVOSORT_REG_SHAPES_U64_KEYS(X) X(1024, 12) X(1024, 8) X(512, 8)
#define EVOSORT_REG_SHAPES_U64_PAIRS(X) X(1024, 12) X(1024, 8) X(512, 8)

// Defined in radix32r.cu and radix64r.cu.
cudaError_t launch_onesweep_reg_u32(bool pairs, int block, int kpt, int rank, size_t grid, int sms,
                                    cudaStream_t s, const RadixArgs& a, int pass);
cudaError_t launch_onesweep_reg_u64(bool pairs, int block, int kpt, int rank, size_t grid, int sms,
                                    cudaStream_t s, const RadixArgs& a, int pass);

// True if the register tile of this shape is compiled for the key width and
// form and supports the digit width and rank mode.
inline bool reg_config_fits(int w, bool pairs, int block, int kpt, int d, int rank) {
    if (d != 8 || (rank != 1 && rank != 3 && rank != 4)) return false;
    bool shape = false;
#define EVOSORT_CASE(B, K) \
    if (block == B && kpt == K) shape = true;
    if (w == 4 && !pairs) { EVOSORT_REG_SHAPES_U32_KEYS(EVOSORT_CASE) }
    if (w == 4 && pairs) { EVOSORT_REG_SHAPES_U32_PAIRS(EVOSORT_CASE) }
    if (w == 8 && !pairs) { EVOSORT_REG_SHAPES_U64_KEYS(EVOSORT_CASE) }
    if (w == 8 && pairs) { EVOSORT_REG_SHAPES_U64_PAIRS(EVOSORT_CASE) }
#undef EVOSORT_CASE
    return shape;
}

// Defined in radix_aux.cu.
cudaError_t launch_onesweep_u32(bool pairs, int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                const RadixArgs& a, int pass);
cudaError_t launch_onesweep_u64(bool pairs, int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                const RadixArgs& a, int pass);
cudaError_t launch_radix_aux(int w, int which, size_t grid, size_t smem, cudaStream_t s, const RadixArgs& a,
                             int inplace);

}  // namespace evosort
