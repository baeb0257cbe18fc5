// Per-rank kernels of the multi-GPU sort of one array (the paper names an
// MPI extension as future work; it has no algorithm for it).  Each rank holds
// a slice of the keys.  The ranks agree on which part of the key range each
// one owns from two reductions over all ranks:
//   K_range  the smallest and largest key of the slice, in the key map's
//            order (the global range is their minimum and maximum);
//   K_bins   a histogram of the slice's keys over nbins equal parts of the
//            global range: bin = (mapped key - base) >> shift, with base the
//            global minimum and shift chosen so that every key falls in
//            [0, nbins).  Summed over ranks, its prefix sums place the
//            boundaries between ranks.
// A slice sorted by the library then sends, to each rank, the contiguous run
// of its keys whose bins that rank owns (the host derives the run lengths
// from the slice's own histogram).
#include "evosort.h"
#include "api_internal.h"
#include "common.cuh"

namespace evosort {
namespace {

constexpr int kShardThreads = 512;

template <typename U>
__global__ void __launch_bounds__(kShardThreads) key_range_kernel(const U* keys, size_t n, KeyMap map,
                                                                   unsigned long long* range) {
    U mn = (U)~(U)0, mx = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const U k = map_fwd(keys[i], map);
        mn = k < mn ? k : mn;
        mx = k > mx ? k : mx;
    }
    unsigned long long a = mn, b = mx;
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y0 = __shfl_xor_sync(0xffffffffu, a, o);
        const unsigned long long y1 = __shfl_xor_sync(0xffffffffu, b, o);
        a = y0 < a ? y0 : a;
        b = y1 > b ? y1 : b;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&range[0], a);
        atomicMax(&range[1], b);
    }
}

template <typename U>
__global__ void __launch_bounds__(kShardThreads) range_bins_kernel(const U* keys, size_t n, KeyMap map, U base,
                                                                    int shift, int nbins, unsigned long long* counts) {
    extern __shared__ uint32_t s_bin[];
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) s_bin[i] = 0u;
    __syncthreads();
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const U k = (U)(map_fwd(keys[i], map) - base);
        unsigned long long b = (unsigned long long)k >> shift;
        if (b >= (unsigned long long)nbins) b = nbins - 1;   // only for keys outside the stated range
        atomicAdd(&s_bin[b], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbins; i += blockDim.x)
        if (s_bin[i]) atomicAdd(&counts[i], (unsigned long long)s_bin[i]);
}

unsigned grid_for(size_t n) {
    const size_t want = (n + kShardThreads - 1) / kShardThreads;
    const size_t cap = (size_t)sm_count() * 4;
    return (unsigned)(want < cap ? (want ? want : 1) : cap);
}

}  // namespace
}  // namespace evosort

using namespace evosort;

extern "C" {

evosort_status evosort_key_range(const void* keys, size_t n, evosort_dtype dt, int descending,
                                 unsigned long long* range, void* stream) {
    set_error("");
    if (dt < EVOSORT_I32 || dt > EVOSORT_F64 || !range || (n && !keys)) {
        set_error("evosort_key_range: bad argument");
        return EVOSORT_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // range[0] starts at the largest value (atomicMin), range[1] at zero (atomicMax)
    cudaError_t e = cudaMemsetAsync(range, 0xFF, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(range + 1, 0, sizeof(unsigned long long), s);
    const KeyMap map = key_map_for(dt, descending != 0);
    if (e == cudaSuccess && n) {
        if (dtype_bytes(dt) == 4)
            key_range_kernel<uint32_t><<<grid_for(n), kShardThreads, 0, s>>>((const uint32_t*)keys, n, map, range);
        else
            key_range_kernel<uint64_t><<<grid_for(n), kShardThreads, 0, s>>>((const uint64_t*)keys, n, map, range);
        e = cudaGetLastError();
        count_launches(1);
    }
    if (e != cudaSuccess) {
        set_error(std::string("evosort_key_range: ") + cudaGetErrorString(e));
        return EVOSORT_ERR_CUDA;
    }
    return EVOSORT_OK;
}

evosort_status evosort_range_histogram(const void* keys, size_t n, evosort_dtype dt, int descending,
                                       unsigned long long base, int shift, int nbins, unsigned long long* counts,
                                       void* stream) {
    set_error("");
    if (dt < EVOSORT_I32 || dt > EVOSORT_F64 || !counts || (n && !keys) || nbins < 1 || nbins > 8192 ||
        shift < 0 || shift >= 8 * dtype_bytes(dt)) {
        set_error("evosort_range_histogram: bad argument");
        return EVOSORT_ERR_INVALID;
    }
    if (!n) return EVOSORT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const KeyMap map = key_map_for(dt, descending != 0);
    const size_t smem = (size_t)nbins * sizeof(uint32_t);
    if (dtype_bytes(dt) == 4)
        range_bins_kernel<uint32_t><<<grid_for(n), kShardThreads, smem, s>>>((const uint32_t*)keys, n, map,
                                                                            (uint32_t)base, shift, nbins, counts);
    else
        range_bins_kernel<uint64_t><<<grid_for(n), kShardThreads, smem, s>>>((const uint64_t*)keys, n, map,
                                                                            (uint64_t)base, shift, nbins, counts);
    const cudaError_t e = cudaGetLastError();
    count_launches(1);
    if (e != cudaSuccess) {
        set_error(std::string("evosort_range_histogram: ") + cudaGetErrorString(e));
        return EVOSORT_ERR_CUDA;
    }
    return EVOSORT_OK;
}

}  // extern "C"
