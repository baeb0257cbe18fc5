// Small-array path of the dispatcher (Algorithm 5, AdaptivePartitionSort):
// the paper hands arrays below its threshold T_np to a library sort instead
// of running its parallel sorts on them.  On the GPU the device-wide radix
// sort of a few thousand keys is all fixed cost (a histogram launch, a scan
// launch, one launch per pass, a copy, and a scratch allocation), so arrays of
// at most small_cap keys are sorted by ONE CTA in shared memory in a single
// launch that needs no scratch memory: the keys (and values) are loaded and
// mapped to the order-preserving key space, sorted by the shared-memory merge
// sort of Algorithm 3 (insertion-sorted base runs, then pairwise merges with
// merge-path splits), mapped back and stored.  Stable, so key/value sorts get
// the stable argsort.
#include "evosort.h"
#include "api_internal.h"
#include "common.cuh"
#include "smem_sort.cuh"

namespace evosort {
namespace {

constexpr int kSmallThreads = 512;
constexpr int kSmallRun = 16;   // longest insertion-sorted base run

template <typename U, bool PAIRS>
__global__ void __launch_bounds__(kSmallThreads) small_sort_kernel(const U* in, U* out, const uint32_t* vin,
                                                                    uint32_t* vout, int n, KeyMap map, int tins) {
    extern __shared__ __align__(16) unsigned char smem[];
    U* k0 = (U*)smem;
    U* k1 = k0 + n;
    uint32_t* v0 = (uint32_t*)(k1 + n);
    uint32_t* v1 = v0 + (PAIRS ? n : 0);
    for (int i = threadIdx.x; i < n; i += kSmallThreads) {
        k0[i] = map_fwd(in[i], map);
        if (PAIRS) v0[i] = vin[i];
    }
    __syncthreads();
    const int which = smem_merge_sort<U, PAIRS, kSmallRun>(k0, k1, v0, v1, n, tins);
    const U* ks = which ? k1 : k0;
    const uint32_t* vs = which ? v1 : v0;
    // in place (in == out) is safe: every input was read before the sort
    for (int i = threadIdx.x; i < n; i += kSmallThreads) {
        out[i] = map_inv(ks[i], map);
        if (PAIRS) vout[i] = vs[i];
    }
}

size_t small_smem(int n, int w, bool pairs) { return (size_t)2 * n * (w + (pairs ? 4 : 0)); }

template <typename U, bool PAIRS>
cudaError_t launch_small(const void* in, void* out, const uint32_t* vin, uint32_t* vout, int n, KeyMap map,
                         int tins, cudaStream_t s) {
    auto kern = small_sort_kernel<U, PAIRS>;
    static bool configured = false;
    if (!configured) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)small_smem(kSmallMax, (int)sizeof(U), PAIRS));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    kern<<<1, kSmallThreads, small_smem(n, (int)sizeof(U), PAIRS), s>>>((const U*)in, (U*)out, vin, vout, n, map,
                                                                      tins);
    return cudaGetLastError();
}

}  // namespace

int small_sort(const void* in, void* out, const uint32_t* vin, uint32_t* vout, size_t n, int dt, const Plan& pl,
               cudaStream_t s, std::string* err) {
    const int w = dtype_bytes(dt);
    const bool pairs = vout != nullptr;
    if (n > (size_t)kSmallMax) {
        *err = "small-array path: more keys than it holds";
        return EVOSORT_ERR_INVALID;
    }
    const KeyMap map = key_map_for(dt, pl.descending);
    // base runs: the insertion threshold, capped at kSmallRun (runs are
    // insertion-sorted in registers, then merged by every thread): a replayed
    // graph of int32 sorts takes 8.1 us per 1000 keys and 18.2 us per 4096
    // keys with 16-key runs, against 9.0 / 20.8 us with 4-key runs
    const int tins = pl.insertion_threshold > kSmallRun ? kSmallRun : pl.insertion_threshold;
    const int call = prof_call_begin(nullptr, 0, s);
    cudaError_t e;
    {
        ProfScope ps(call, EVOSORT_K_SMALL, -1, 2.0 * (double)n * (w + (pairs ? 4 : 0)), n, s);
        if (w == 4)
            e = pairs ? launch_small<uint32_t, true>(in, out, vin, vout, (int)n, map, tins, s)
                      : launch_small<uint32_t, false>(in, out, vin, vout, (int)n, map, tins, s);
        else
            e = pairs ? launch_small<uint64_t, true>(in, out, vin, vout, (int)n, map, tins, s)
                      : launch_small<uint64_t, false>(in, out, vin, vout, (int)n, map, tins, s);
    }
    prof_call_end(call, s, nullptr);
    count_launches(1);
    if (e != cudaSuccess) {
        *err = std::string("small-array sort launch: ") + cudaGetErrorString(e);
        return EVOSORT_ERR_CUDA;
    }
    return EVOSORT_OK;
}

}  // namespace evosort
