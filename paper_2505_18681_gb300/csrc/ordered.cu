// Sort of an array the dispatcher's sample shows in order (every sampled
// neighbour pair non-decreasing, or every one non-increasing, in the order
// the sort produces).  Not a step of the paper's algorithms: its dispatcher
// (Algorithm 5) picks a method by the input's properties, and an input that
// is already sorted needs one read and one write, where the radix path reads
// it for its histogram (which finds the same order) and then copies it.
//
//   ordered_pass  reads the keys once, checks that every key is in order with
//                 its successor (in the key map's order) and writes the output
//                 as it goes: a copy (keys, and values for key/value sorts), a
//                 reversed copy (keys only, input in reverse order), or
//                 nothing (in place, input in order).  A key out of order sets
//                 a flag.
//   host          reads the flag (one small synchronous copy).  If it is set
//                 the caller runs the radix sort, which rewrites the whole
//                 output from the untouched input (the input is never written
//                 here: in place only the check runs).
//
// The scratch (one flag word) comes from the stream-ordered pool.
#include <cstring>
#include <string>

#include "evosort.h"
#include "api_internal.h"
#include "common.cuh"

namespace evosort {
namespace {

constexpr int kOrdThreads = 256;

enum : int { ORD_COPY = 0, ORD_CHECK = 1, ORD_REVERSE = 2 };

// MODE: ORD_COPY (out = in, in order), ORD_CHECK (in place, in order),
// ORD_REVERSE (out = reversed in, in reverse order; keys only).
template <typename U, bool PAIRS, int MODE>
__global__ void __launch_bounds__(kOrdThreads) ordered_pass(const U* in, U* out, const uint32_t* vin, uint32_t* vout,
                                                             size_t n, KeyMap map, uint32_t* bad) {
    constexpr int V = 16 / sizeof(U);
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t gthreads = (size_t)gridDim.x * blockDim.x;
    bool wrong = false;
    // keys in order: non-decreasing for copies and checks, non-increasing
    // for reversals (then the reversed output is non-decreasing)
    auto in_order = [&](U a, U b) { return MODE == ORD_REVERSE ? a >= b : a <= b; };
    auto put = [&](size_t i, U raw) {
        if (MODE == ORD_COPY) {
            out[i] = raw;
            if (PAIRS) vout[i] = vin[i];
        } else if (MODE == ORD_REVERSE) {
            out[n - 1 - i] = raw;
        }
    };
    size_t head = ((16 - ((uintptr_t)in & 15)) & 15) / sizeof(U);
    if (head > n) head = n;
    const size_t nvec = (n - head) / V;
    const size_t tail0 = head + nvec * V;
    // scalar keys: the unaligned head and the tail
    auto scalar = [&](size_t i) {
        const U raw = in[i];
        if (i + 1 < n && !in_order(map_fwd(raw, map), map_fwd(in[i + 1], map))) wrong = true;
        put(i, raw);
    };
    if (gtid < head) scalar(gtid);
    if (gtid < n - tail0) scalar(tail0 + gtid);
    const uint4* vp = (const uint4*)(in + head);
    for (size_t c = gtid; c < nvec; c += gthreads) {
        const size_t i0 = head + c * V;
        const uint4 q = __ldcs(vp + c);
        U k[V];
        memcpy(k, &q, 16);
        const U next = i0 + V < n ? in[i0 + V] : (U)0;   // first key of the next chunk (cached by its reader)
#pragma unroll
        for (int t = 0; t < V; ++t) {
            const U a = map_fwd(k[t], map);
            if (t + 1 < V) {
                if (!in_order(a, map_fwd(k[t + 1], map))) wrong = true;
            } else if (i0 + V < n) {
                if (!in_order(a, map_fwd(next, map))) wrong = true;
            }
        }
        if (MODE == ORD_COPY && (((uintptr_t)(out + i0)) & 15) == 0) {
            __stcs((uint4*)(out + i0), q);
            if (PAIRS) {
#pragma unroll
                for (int t = 0; t < V; ++t) vout[i0 + t] = vin[i0 + t];
            }
        } else {
#pragma unroll
            for (int t = 0; t < V; ++t) put(i0 + t, k[t]);
        }
    }
    if (__any_sync(0xffffffffu, wrong) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

template <typename U, bool PAIRS, int MODE>
cudaError_t launch_ordered(const void* in, void* out, const uint32_t* vin, uint32_t* vout, size_t n, const KeyMap& map,
                           uint32_t* bad, cudaStream_t s) {
    const int sms = sm_count();
    const size_t want = (n / (16 / sizeof(U)) + kOrdThreads - 1) / kOrdThreads;
    const size_t cap = (size_t)sms * 8;
    const unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
    ordered_pass<U, PAIRS, MODE><<<grid, kOrdThreads, 0, s>>>((const U*)in, (U*)out, vin, vout, n, map, bad);
    return cudaGetLastError();
}

template <typename U>
cudaError_t launch_mode(int mode, bool pairs, const void* in, void* out, const uint32_t* vin, uint32_t* vout, size_t n,
                        const KeyMap& map, uint32_t* bad, cudaStream_t s) {
    if (mode == ORD_REVERSE) return launch_ordered<U, false, ORD_REVERSE>(in, out, vin, vout, n, map, bad, s);
    if (mode == ORD_CHECK)
        return pairs ? launch_ordered<U, true, ORD_CHECK>(in, out, vin, vout, n, map, bad, s)
                     : launch_ordered<U, false, ORD_CHECK>(in, out, vin, vout, n, map, bad, s);
    return pairs ? launch_ordered<U, true, ORD_COPY>(in, out, vin, vout, n, map, bad, s)
                 : launch_ordered<U, false, ORD_COPY>(in, out, vin, vout, n, map, bad, s);
}

}  // namespace

int ordered_sort(const void* in, void* out, const uint32_t* vin, uint32_t* vout, size_t n, int dt, bool descending,
                 int hint, cudaStream_t s, bool* done, std::string* err) {
    *done = false;
    const bool pairs = vout != nullptr;
    const bool inplace = in == out;
    int mode;
    if (hint > 0)
        mode = inplace ? ORD_CHECK : ORD_COPY;
    else if (hint < 0 && !pairs && !inplace)
        mode = ORD_REVERSE;   // a reversed key/value input is only sorted by a reversal when no two keys are equal
    else
        return EVOSORT_OK;
    const KeyMap map = key_map_for(dt, descending);
    void* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, 256, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *err = std::string("ordered path scratch: ") + cudaGetErrorString(e);
        return EVOSORT_ERR_NOMEM;
    }
    uint32_t* bad = (uint32_t*)scratch;
    e = cudaMemsetAsync(bad, 0, sizeof(uint32_t), s);
    const int call = prof_call_begin(nullptr, 0, s);
    {
        const int w = dtype_bytes(dt);
        const double bytes = (double)n * (w + (pairs ? 4 : 0)) * (mode == ORD_CHECK ? 1 : 2);
        ProfScope ps(call, EVOSORT_K_ORDERED, mode, bytes, n, s);
        if (e == cudaSuccess)
            e = w == 4 ? launch_mode<uint32_t>(mode, pairs, in, out, vin, vout, n, map, bad, s)
                       : launch_mode<uint64_t>(mode, pairs, in, out, vin, vout, n, map, bad, s);
    }
    uint32_t flag = 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, bad, sizeof(flag), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(scratch, s);
    prof_call_end(call, s, nullptr);
    count_launches(1);
    if (e != cudaSuccess) {
        *err = std::string("ordered path: ") + cudaGetErrorString(e);
        return EVOSORT_ERR_CUDA;
    }
    *done = flag == 0;
    return EVOSORT_OK;
}

}  // namespace evosort
