// Counting sort of keys whose range is narrow, inside the radix path (keys
// only, 8-bit digits).  Not a step of the paper's algorithms: when K1's key
// range shows at most kCountBins distinct values between the smallest and
// the largest key, but at least 256 (so the radix sort would run two or more
// passes), every key is counted by value and the output written from the
// counts: one read and one write of the keys instead of a read and a write
// per pass.
//
//   K_cv radix_count_values  after K2: decides from K1's key range and order
//                            flags (every CTA the same way); if it applies,
//                            CTA 0 marks every pass inactive and the fixup
//                            as none, and each CTA counts its keys' values
//                            (mapped key - smallest key) into shared bins and
//                            adds them to the global bins.
//   K_cf radix_count_fill    same decision; each CTA forms the exclusive
//                            prefix of the global bins in shared memory and
//                            writes value j at output positions
//                            [prefix[j], prefix[j + 1]) with 16-byte stores.
// Inputs already in order, or in exact reverse order, keep K2's copy (they
// need no counting).  The bins (kCountBins 64-bit words) are scratch the host
// zeroes with the rest of the radix scratch.
#include "radix.cuh"
#include "api_internal.h"

namespace evosort {
namespace {

constexpr int kCountBins = 8192;
constexpr int kCountThreads = 1024;

template <typename U>
__device__ __forceinline__ bool counting_applies(const RadixArgs& a, U* base) {
    if (!a.range || !(a.range[RNG_FLAGS] & RNG_RECORDED)) return false;
    if (a.order[ORD_DESCENT] == 0 || a.order[ORD_ASCENT] == 0) return false;   // K2 copies these
    const U mn = (U)~(U)a.range[RNG_NOTMIN];
    const U span = (U)((U)a.range[RNG_MAX] - mn);
    if ((unsigned long long)span < 256ull || (unsigned long long)span >= (unsigned long long)kCountBins)
        return false;
    *base = mn;
    return true;
}

template <typename U>
__global__ void __launch_bounds__(kCountThreads) radix_count_values(RadixArgs a, unsigned long long* bins) {
    __shared__ uint32_t s_h[kCountBins];
    U base;
    if (!counting_applies<U>(a, &base)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int p = 0; p < a.npass; ++p) a.desc[p].active = 0;
        a.desc[a.npass].fixup = FIX_NONE;
    }
    for (int i = threadIdx.x; i < kCountBins; i += blockDim.x) s_h[i] = 0u;
    __syncthreads();
    const U* keys = (const U*)a.in;
    const size_t n = a.n;
    const KeyMap map = a.map;
    constexpr int V = 16 / sizeof(U);
    size_t head = ((16 - ((uintptr_t)keys & 15)) & 15) / sizeof(U);
    if (head > n) head = n;
    const size_t nvec = (n - head) / V;
    const size_t tail0 = head + nvec * V;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t gthreads = (size_t)gridDim.x * blockDim.x;
    auto one = [&](U raw) { atomicAdd(&s_h[(uint32_t)(U)(map_fwd(raw, map) - base)], 1u); };
    if (gtid < head) one(keys[gtid]);
    if (gtid < n - tail0) one(keys[tail0 + gtid]);
    const uint4* vp = (const uint4*)(keys + head);
    constexpr int kUnroll = 4;
    for (size_t c0 = gtid; c0 < nvec; c0 += gthreads * kUnroll) {
        uint4 q[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const size_t c = c0 + (size_t)u * gthreads;
            if (c < nvec) q[u] = __ldcs(vp + c);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (c0 + (size_t)u * gthreads < nvec) {
                U k[V];
                memcpy(k, &q[u], 16);
#pragma unroll
                for (int j = 0; j < V; ++j) one(k[j]);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kCountBins; i += blockDim.x)
        if (s_h[i]) atomicAdd(&bins[i], (unsigned long long)s_h[i]);
}

template <typename U>
__global__ void __launch_bounds__(kCountThreads) radix_count_fill(RadixArgs a, const unsigned long long* bins) {
    extern __shared__ unsigned long long s_start[];   // kCountBins + 1
    __shared__ unsigned long long s_part[kCountThreads / 32];
    U base;
    if (!counting_applies<U>(a, &base)) return;
    // exclusive prefix of the bins: each thread sums a run of kCountBins /
    // kCountThreads bins, the runs' totals are scanned, then each run is
    // written out
    constexpr int PER = kCountBins / kCountThreads;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long run[PER];
    unsigned long long tot = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        run[j] = bins[tid * PER + j];
        tot += run[j];
    }
    unsigned long long inc = tot;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_part[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < kCountThreads / 32 ? s_part[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kCountThreads / 32) s_part[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    unsigned long long ex = inc - tot + (warp > 0 ? s_part[warp - 1] : 0ull);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        s_start[tid * PER + j] = ex;
        ex += run[j];
    }
    if (tid == kCountThreads - 1) s_start[kCountBins] = ex;
    __syncthreads();
    // value index of output position i: the last j with start[j] <= i
    auto value_at = [&](size_t i) {
        int lo = 0, hi = kCountBins - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_start[mid] <= i)
                lo = mid;
            else
                hi = mid - 1;
        }
        return lo;
    };
    const KeyMap map = a.map;
    U* out = (U*)a.out;
    const size_t n = a.n;
    constexpr int V = 16 / sizeof(U);
    size_t head = ((16 - ((uintptr_t)out & 15)) & 15) / sizeof(U);
    if (head > n) head = n;
    const size_t nvec = (n - head) / V;
    const size_t tail0 = head + nvec * V;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + tid;
    const size_t gthreads = (size_t)gridDim.x * blockDim.x;
    if (gtid < head) out[gtid] = map_inv((U)(base + (U)value_at(gtid)), map);
    if (gtid < n - tail0) out[tail0 + gtid] = map_inv((U)(base + (U)value_at(tail0 + gtid)), map);
    uint4* vp = (uint4*)(out + head);
    for (size_t c = gtid; c < nvec; c += gthreads) {
        const size_t i0 = head + c * V;
        int j = value_at(i0);
        U k[V];
#pragma unroll
        for (int t = 0; t < V; ++t) {
            while (j + 1 < kCountBins && s_start[j + 1] <= i0 + t) ++j;
            k[t] = map_inv((U)(base + (U)j), map);
        }
        uint4 q;
        memcpy(&q, k, 16);
        __stcs(vp + c, q);
    }
}

template <typename U>
cudaError_t launch_counting(const RadixArgs& a, unsigned long long* bins, cudaStream_t s) {
    static bool configured = false;
    const size_t smem = (kCountBins + 1) * sizeof(unsigned long long);
    if (!configured) {
        const cudaError_t e =
            cudaFuncSetAttribute(radix_count_fill<U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int sms = sm_count();
    const size_t want = (a.n / (16 / sizeof(U)) + kCountThreads - 1) / kCountThreads;
    const unsigned grid = (unsigned)(want < (size_t)sms * 2 ? (want ? want : 1) : (size_t)sms * 2);
    radix_count_values<U><<<grid, kCountThreads, 0, s>>>(a, bins);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    radix_count_fill<U><<<grid, kCountThreads, smem, s>>>(a, bins);
    return cudaGetLastError();
}

}  // namespace

size_t counting_bins_bytes() { return (size_t)kCountBins * sizeof(unsigned long long); }

cudaError_t launch_radix_counting(int w, const RadixArgs& a, unsigned long long* bins, cudaStream_t s) {
    return w == 4 ? launch_counting<uint32_t>(a, bins, s) : launch_counting<uint64_t>(a, bins, s);
}

}  // namespace evosort
