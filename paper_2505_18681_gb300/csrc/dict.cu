// Sort of an array whose keys take a few distinct values (the dispatcher's
// "few" class: at most kDictMax distinct keys in its sample).  Not a step of
// the paper's algorithms: its dispatcher (Algorithm 5) picks a method by the
// input's properties, and for a handful of distinct keys a counting sort over
// the sample's values moves each key twice (one read, one write) where the
// radix sort runs all its passes.
//
//   K_dc dict_count  every key is mapped to the order-preserving key space and
//                    looked up (binary search) among the sample's distinct
//                    values; a CTA counts hits per value in lane-private shared
//                    counters and adds them to global counts; a key that is
//                    not among them sets a miss flag.
//   host             reads the counts and the flag (one small synchronous
//                    copy).  A miss means the sample did not see every value:
//                    the caller then runs the radix sort on the untouched
//                    input.
//   K_df dict_fill   otherwise writes value j at output positions
//                    [prefix[j], prefix[j + 1]), mapped back, with 16-byte
//                    stores.
//
// Keys only: equal keys are identical bit patterns, so the output is the
// sorted array itself.  In place works (the fill runs after every key was
// read).  The scratch (counts and flag, about 1 KB) comes from the
// stream-ordered pool.
#include <cstring>
#include <string>
#include <vector>

#include "evosort.h"
#include "api_internal.h"
#include "common.cuh"

namespace evosort {
namespace {

constexpr int kDictThreads = 512;
constexpr int kFillThreads = 256;

struct DictVals {
    unsigned long long v[kDictMax];   // distinct mapped keys, ascending
    int m;
};
struct DictPrefix {
    unsigned long long start[kDictMax + 1];   // exclusive prefix of the counts, start[m] = n
    int m;
};

template <typename U>
__global__ void __launch_bounds__(kDictThreads) dict_count(const U* keys, size_t n, KeyMap map, DictVals d,
                                                            unsigned long long* counts, uint32_t* miss) {
    __shared__ U s_v[kDictMax];
    __shared__ uint32_t s_c[kDictMax * 32];   // (value, lane): a lane only touches its own bank
    const int m = d.m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s_v[i] = (U)d.v[i];
    for (int i = threadIdx.x; i < m * 32; i += blockDim.x) s_c[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    bool bad = false;
    auto one = [&](U raw) {
        const U k = map_fwd(raw, map);
        int lo = 0, hi = m;   // first value >= k
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_v[mid] < k)
                lo = mid + 1;
            else
                hi = mid;
        }
        if (lo < m && s_v[lo] == k)
            atomicAdd(&s_c[lo * 32 + lane], 1u);
        else
            bad = true;
    };
    constexpr int V = 16 / sizeof(U);
    size_t head = ((16 - ((uintptr_t)keys & 15)) & 15) / sizeof(U);
    if (head > n) head = n;
    const size_t nvec = (n - head) / V;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t gthreads = (size_t)gridDim.x * blockDim.x;
    if (gtid < head) one(keys[gtid]);
    const size_t tail0 = head + nvec * V;
    if (gtid < n - tail0) one(keys[tail0 + gtid]);
    const uint4* vp = (const uint4*)(keys + head);
    // grid-stride over 16-byte chunks, kUnroll chunks per step whose loads
    // are all issued before the lookups (enough bytes in flight per SM)
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
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(miss, 1u);
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        unsigned long long sum = 0;
        for (int l = 0; l < 32; ++l) sum += s_c[j * 32 + l];
        if (sum) atomicAdd(&counts[j], sum);
    }
}

template <typename U>
__global__ void __launch_bounds__(kFillThreads) dict_fill(U* out, size_t n, KeyMap map, DictVals d, DictPrefix p) {
    __shared__ unsigned long long s_start[kDictMax + 1];
    __shared__ U s_key[kDictMax];
    const int m = p.m;
    for (int i = threadIdx.x; i <= m; i += blockDim.x) s_start[i] = p.start[i];
    for (int i = threadIdx.x; i < m; i += blockDim.x) s_key[i] = map_inv((U)d.v[i], map);
    __syncthreads();
    // value index of output position i: the last j with start[j] <= i
    auto value_at = [&](size_t i) {
        int lo = 0, hi = m - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_start[mid] <= i)
                lo = mid;
            else
                hi = mid - 1;
        }
        return lo;
    };
    constexpr int V = 16 / sizeof(U);
    size_t head = ((16 - ((uintptr_t)out & 15)) & 15) / sizeof(U);
    if (head > n) head = n;
    const size_t nvec = (n - head) / V;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t gthreads = (size_t)gridDim.x * blockDim.x;
    if (gtid < head) out[gtid] = s_key[value_at(gtid)];
    const size_t tail0 = head + nvec * V;
    if (gtid < n - tail0) out[tail0 + gtid] = s_key[value_at(tail0 + gtid)];
    uint4* vp = (uint4*)(out + head);
    for (size_t c = gtid; c < nvec; c += gthreads) {
        const size_t i0 = head + c * V;
        int j = value_at(i0);
        U k[V];
#pragma unroll
        for (int t = 0; t < V; ++t) {
            while (j + 1 < m && s_start[j + 1] <= i0 + t) ++j;
            k[t] = s_key[j];
        }
        uint4 q;
        memcpy(&q, k, 16);
        __stcs(vp + c, q);
    }
}

template <typename U>
int dict_sort_t(const void* in, void* out, size_t n, const KeyMap& map, const std::vector<uint64_t>& dict,
                cudaStream_t s, bool* done, std::string* err) {
    DictVals d;
    std::memset(&d, 0, sizeof(d));
    d.m = (int)dict.size();
    for (int i = 0; i < d.m; ++i) d.v[i] = dict[i];
    void* scratch = nullptr;
    const size_t sbytes = (kDictMax + 1) * sizeof(unsigned long long);
    cudaError_t e = cudaMallocAsync(&scratch, sbytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *err = std::string("dictionary sort scratch: ") + cudaGetErrorString(e);
        return EVOSORT_ERR_NOMEM;
    }
    unsigned long long* counts = (unsigned long long*)scratch;
    uint32_t* miss = (uint32_t*)(counts + kDictMax);
    e = cudaMemsetAsync(scratch, 0, sbytes, s);
    const int sms = sm_count();
    const size_t want = (n / (sizeof(U) == 4 ? 4 : 2) + kDictThreads - 1) / kDictThreads;
    const unsigned grid = (unsigned)(want < (size_t)sms * 4 ? (want ? want : 1) : (size_t)sms * 4);
    const int call = prof_call_begin(nullptr, 0, s);
    {
        ProfScope ps(call, EVOSORT_K_DICT, 0, (double)n * sizeof(U), n, s);
        if (e == cudaSuccess) {
            dict_count<U><<<grid, kDictThreads, 0, s>>>((const U*)in, n, map, d, counts, miss);
            e = cudaGetLastError();
        }
    }
    std::vector<unsigned long long> host(kDictMax + 1, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host.data(), scratch, sbytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    count_launches(1);
    if (e != cudaSuccess) {
        cudaFreeAsync(scratch, s);
        prof_call_end(call, s, nullptr);
        *err = std::string("dictionary count: ") + cudaGetErrorString(e);
        return EVOSORT_ERR_CUDA;
    }
    uint32_t missed = 0;
    std::memcpy(&missed, &host[kDictMax], sizeof(missed));
    DictPrefix p;
    std::memset(&p, 0, sizeof(p));
    p.m = d.m;
    unsigned long long run = 0;
    for (int j = 0; j < d.m; ++j) {
        p.start[j] = run;
        run += host[j];
    }
    p.start[d.m] = run;
    // a key outside the sample's values, or counts that do not add up to n
    // (which only an inconsistent run could produce): the caller sorts by radix
    if (missed || run != (unsigned long long)n) {
        cudaFreeAsync(scratch, s);
        prof_call_end(call, s, nullptr);
        *done = false;
        return EVOSORT_OK;
    }
    {
        ProfScope ps(call, EVOSORT_K_DICT, 1, (double)n * sizeof(U), n, s);
        const size_t wantf = (n / (sizeof(U) == 4 ? 4 : 2) + kFillThreads - 1) / kFillThreads;
        const unsigned gridf = (unsigned)(wantf < (size_t)sms * 8 ? (wantf ? wantf : 1) : (size_t)sms * 8);
        dict_fill<U><<<gridf, kFillThreads, 0, s>>>((U*)out, n, map, d, p);
        e = cudaGetLastError();
    }
    count_launches(1);
    cudaFreeAsync(scratch, s);
    prof_call_end(call, s, nullptr);
    if (e != cudaSuccess) {
        *err = std::string("dictionary fill: ") + cudaGetErrorString(e);
        return EVOSORT_ERR_CUDA;
    }
    *done = true;
    return EVOSORT_OK;
}

}  // namespace

int dict_sort(const void* in, void* out, size_t n, int dt, bool descending, const std::vector<uint64_t>& dict,
              cudaStream_t s, bool* done, std::string* err) {
    *done = false;
    if (dict.empty() || dict.size() > (size_t)kDictMax) return EVOSORT_OK;
    const KeyMap map = key_map_for(dt, descending);
    return dtype_bytes(dt) == 4 ? dict_sort_t<uint32_t>(in, out, n, map, dict, s, done, err)
                                : dict_sort_t<uint64_t>(in, out, n, map, dict, s, done, err);
}

}  // namespace evosort
