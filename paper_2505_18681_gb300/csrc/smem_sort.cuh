// Sorting building blocks that work on data already on chip: a warp bitonic
// sort of keys held in registers and a CTA merge sort of a tile held in
// shared memory (insertion-sorted base runs, then pairwise merges with
// merge-path splits per thread, as in Algorithm 3).
#pragma once

#include "common.cuh"

namespace evosort {

// Merge-path split: number of keys of run A among the first k outputs of the
// stable merge of A (length la) and B (length lb).
template <typename U, typename AccA, typename AccB>
__device__ __forceinline__ size_t merge_path(AccA A, size_t la, AccB B, size_t lb, size_t k) {
    size_t lo = k > lb ? k - lb : 0;
    size_t hi = k < la ? k : la;
    while (lo < hi) {
        const size_t mid = (lo + hi) >> 1;
        if ((U)B(k - 1 - mid) < (U)A(mid))
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// CTA merge sort of len <= capacity keys (and values) in shared memory.
// k0/v0 hold the input; k1/v1 are scratch of the same size.  Base runs of
// tins keys are insertion-sorted (one thread per run), then merged pairwise,
// the run width doubling.  Stable.  Returns 0 if the result is in k0/v0, 1 if
// in k1/v1.  All threads of the CTA must call it.
// ---------------------------------------------------------------------------
template <typename U, bool PAIRS>
__device__ int smem_merge_sort(U* k0, U* k1, uint32_t* v0, uint32_t* v1, int len, int tins) {
    const int nt = blockDim.x;
    const int runs = (len + tins - 1) / tins;
    for (int r = threadIdx.x; r < runs; r += nt) {
        const int lo = r * tins;
        const int hi = lo + tins < len ? lo + tins : len;
        for (int i = lo + 1; i < hi; ++i) {
            const U key = k0[i];
            const uint32_t val = PAIRS ? v0[i] : 0u;
            int j = i;
            while (j > lo && k0[j - 1] > key) {   // strictly greater: stable
                k0[j] = k0[j - 1];
                if (PAIRS) v0[j] = v0[j - 1];
                --j;
            }
            k0[j] = key;
            if (PAIRS) v0[j] = val;
        }
    }
    __syncthreads();
    const int chunk = (len + nt - 1) / nt;
    U* ks = k0;
    U* kd = k1;
    uint32_t* vs = v0;
    uint32_t* vd = v1;
    int which = 0;
    for (int w = tins; w < len; w <<= 1) {
        int o = threadIdx.x * chunk;
        const int oend = o + chunk < len ? o + chunk : len;
        while (o < oend) {
            const int pbase = (o / (2 * w)) * (2 * w);
            const int la = (pbase + w < len ? pbase + w : len) - pbase;
            const int lb = (pbase + 2 * w < len ? pbase + 2 * w : len) - pbase - la;
            const U* A = ks + pbase;
            const U* B = A + la;
            const int k = o - pbase;
            int ia = (int)merge_path<U>([&](size_t i) { return A[i]; }, la, [&](size_t i) { return B[i]; }, lb,
                                        (size_t)k);
            int ib = k - ia;
            const int stop = (pbase + la + lb < oend ? pbase + la + lb : oend);
            for (; o < stop; ++o) {
                const bool takeB = ia >= la || (ib < lb && B[ib] < A[ia]);
                if (takeB) {
                    kd[o] = B[ib];
                    if (PAIRS) vd[o] = vs[pbase + la + ib];
                    ++ib;
                } else {
                    kd[o] = A[ia];
                    if (PAIRS) vd[o] = vs[pbase + ia];
                    ++ia;
                }
            }
        }
        __syncthreads();
        U* t = ks; ks = kd; kd = t;
        uint32_t* tv = vs; vs = vd; vd = tv;
        which ^= 1;
    }
    return which;
}

// ---------------------------------------------------------------------------
// Warp bitonic sort of 32*KW keys, ascending.  Lane L holds keys
// [L*KW, (L+1)*KW) of the sequence in k[0..KW) (blocked layout); KW is a power
// of two.  Not stable (used for keys-only sorts, where equal keys are
// identical bit patterns, so the output is the same either way).
// ---------------------------------------------------------------------------
template <typename U>
__device__ __forceinline__ void cmp_swap(U& a, U& b, bool up) {
    const U lo = a < b ? a : b;
    const U hi = a < b ? b : a;
    a = up ? lo : hi;
    b = up ? hi : lo;
}

template <typename U, int KW>
__device__ __forceinline__ void warp_bitonic_sort(U (&k)[KW]) {
    const int lane = threadIdx.x & 31;
    constexpr int N = 32 * KW;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= KW) {
                // partner element lives in another lane at the same register
                const int lstride = stride / KW;
#pragma unroll
                for (int r = 0; r < KW; ++r) {
                    const int idx = lane * KW + r;
                    const bool up = ((idx & size) == 0);
                    const U other = __shfl_xor_sync(0xffffffffu, k[r], lstride);
                    const bool lower = (lane & lstride) == 0;   // this lane holds the lower index
                    const bool keep_min = (lower == up);
                    const U mn = k[r] < other ? k[r] : other;
                    const U mx = k[r] < other ? other : k[r];
                    k[r] = keep_min ? mn : mx;
                }
            } else {
#pragma unroll
                for (int r = 0; r < KW; ++r) {
                    if ((r & stride) == 0) {
                        const int idx = lane * KW + r;
                        const bool up = ((idx & size) == 0);
                        cmp_swap(k[r], k[r + stride], up);
                    }
                }
            }
        }
    }
}

}  // namespace evosort
