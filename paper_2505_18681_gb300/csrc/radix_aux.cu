// Histogram, scan/plan and fixup kernels of both key widths, and the
// dispatch to the per-width onesweep translation units.
#include "radix_launch.cuh"

namespace evosort {

cudaError_t launch_onesweep_u32(bool pairs, int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                const RadixArgs& a, int pass) {
    return pairs ? launch_onesweep_u32_pairs(block, kpt, rank, grid, sms, s, a, pass)
                 : launch_onesweep_u32_keys(block, kpt, rank, grid, sms, s, a, pass);
}

cudaError_t launch_onesweep_u64(bool pairs, int block, int kpt, int rank, size_t grid, int sms, cudaStream_t s,
                                const RadixArgs& a, int pass) {
    return pairs ? launch_onesweep_u64_pairs(block, kpt, rank, grid, sms, s, a, pass)
                 : launch_onesweep_u64_keys(block, kpt, rank, grid, sms, s, a, pass);
}

// which: 0 = histogram, 1 = scan/plan, 2 = fixup, 3 = rebased histogram
// (8-bit digits only)
cudaError_t launch_radix_aux(int w, int which, size_t grid, size_t smem, cudaStream_t s, const RadixArgs& a,
                             int inplace) {
    if (which == 0 || which == 3) {
        static bool configured = false;
        if (!configured) {
            cudaFuncSetAttribute(radix_histogram<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kHistSmem);
            cudaFuncSetAttribute(radix_histogram<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kHistSmem);
            cudaFuncSetAttribute(radix_histogram8<uint32_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kHistSmem);
            cudaFuncSetAttribute(radix_histogram8<uint64_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kHistSmem);
            cudaFuncSetAttribute(radix_histogram8<uint32_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kHistSmem);
            cudaFuncSetAttribute(radix_histogram8<uint64_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kHistSmem);
            configured = true;
        }
        (void)smem;
        const size_t hs = (size_t)a.npass * ((size_t)1 << a.d) * hist_cols(a.npass, a.d) * 4;
        if (which == 3) {
            if (a.d != 8) return cudaErrorInvalidValue;
            if (w == 4)
                radix_histogram8<uint32_t, true><<<(unsigned)grid, kHistThreads, hs, s>>>(a);
            else
                radix_histogram8<uint64_t, true><<<(unsigned)grid, kHistThreads, hs, s>>>(a);
        } else if (a.d == 8 && w == 4)
            radix_histogram8<uint32_t, false><<<(unsigned)grid, kHistThreads, hs, s>>>(a);
        else if (a.d == 8)
            radix_histogram8<uint64_t, false><<<(unsigned)grid, kHistThreads, hs, s>>>(a);
        else if (w == 4)
            radix_histogram<uint32_t><<<(unsigned)grid, kHistThreads, hs, s>>>(a);
        else
            radix_histogram<uint64_t><<<(unsigned)grid, kHistThreads, hs, s>>>(a);
    } else if (which == 1) {
        radix_scan_plan<<<1, 1024, 0, s>>>(a, inplace);
    } else {
        if (w == 4)
            radix_fixup<uint32_t><<<(unsigned)grid, 256, 0, s>>>(a);
        else
            radix_fixup<uint64_t><<<(unsigned)grid, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace evosort
