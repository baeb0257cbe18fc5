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

// Longest base run sorted in registers: 32 keys of 4 bytes, 16 of 8 bytes
// (with their values); longer runs are insertion-sorted in shared memory.
template <typename U>
__host__ __device__ constexpr int reg_run_max() { return sizeof(U) == 4 ? 32 : 16; }

// Insertion sort of the first len <= R keys (and values) of a register array:
// key i moves left past every strictly greater key, one neighbour exchange at
// a time, so equal keys keep their order (stable).  The loops are unrolled
// over R, so the arrays stay in registers; positions len..R-1 are not touched.
template <typename U, bool PAIRS, int R>
__device__ __forceinline__ void reg_insertion_sort(U (&k)[R], uint32_t (&v)[R], int len) {
#pragma unroll
    for (int i = 1; i < R; ++i) {
        if (i < len) {
#pragma unroll
            for (int j = i; j > 0; --j) {
                const bool sw = k[j - 1] > k[j];
                const U lo = sw ? k[j] : k[j - 1];
                const U hi = sw ? k[j - 1] : k[j];
                k[j - 1] = lo;
                k[j] = hi;
                if (PAIRS) {
                    const uint32_t vl = sw ? v[j] : v[j - 1];
                    const uint32_t vh = sw ? v[j - 1] : v[j];
                    v[j - 1] = vl;
                    v[j] = vh;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// CTA merge sort of len <= capacity keys (and values) in shared memory.
// k0/v0 hold the input; k1/v1 are scratch of the same size.  Base runs of
// tins keys are insertion-sorted (one thread per run: in registers up to R
// keys, in shared memory beyond), then merged pairwise, the run
// width doubling.  Stable.  Returns 0 if the result is in k0/v0, 1 if in
// k1/v1.  All threads of the CTA must call it.
// ---------------------------------------------------------------------------
template <typename U, bool PAIRS, int R = reg_run_max<U>(), bool PAD = false>
__device__ int smem_merge_sort(U* k0, U* k1, uint32_t* v0, uint32_t* v1, int len, int tins) {
    // element i of each array lives at ix(i): with PAD, one spare word per 32
    // (the caller sizes the arrays for that), so lanes whose positions are a
    // power of two apart fall in different banks
    auto ix = [](int i) { return PAD ? i + (i >> 5) : i; };
    const int nt = blockDim.x;
    const int runs = (len + tins - 1) / tins;
    if (tins <= R) {
        // one run per thread, loaded into registers, sorted, stored back
        // (a thread's run is contiguous in shared memory, so a warp's lanes
        // sit tins words apart; registers keep the exchanges off the banks)
        for (int r = threadIdx.x; r < runs; r += nt) {
            const int lo = r * tins;
            const int m = lo + tins < len ? tins : len - lo;
            U k[R];
            uint32_t v[R];
#pragma unroll
            for (int j = 0; j < R; ++j) {
                k[j] = j < m ? k0[ix(lo + j)] : (U)0;
                v[j] = (PAIRS && j < m) ? v0[ix(lo + j)] : 0u;
            }
            reg_insertion_sort<U, PAIRS, R>(k, v, m);
#pragma unroll
            for (int j = 0; j < R; ++j)
                if (j < m) {
                    k0[ix(lo + j)] = k[j];
                    if (PAIRS) v0[ix(lo + j)] = v[j];
                }
        }
    } else {
        for (int r = threadIdx.x; r < runs; r += nt) {
            const int lo = r * tins;
            const int hi = lo + tins < len ? lo + tins : len;
            for (int i = lo + 1; i < hi; ++i) {
                const U key = k0[ix(i)];
                const uint32_t val = PAIRS ? v0[ix(i)] : 0u;
                int j = i;
                while (j > lo && k0[ix(j - 1)] > key) {   // strictly greater: stable
                    k0[ix(j)] = k0[ix(j - 1)];
                    if (PAIRS) v0[ix(j)] = v0[ix(j - 1)];
                    --j;
                }
                k0[ix(j)] = key;
                if (PAIRS) v0[ix(j)] = val;
            }
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
            const int bbase = pbase + la;
            const int k = o - pbase;
            int ia = (int)merge_path<U>([&](size_t i) { return ks[ix(pbase + (int)i)]; }, la,
                                        [&](size_t i) { return ks[ix(bbase + (int)i)]; }, lb, (size_t)k);
            int ib = k - ia;
            const int stop = (pbase + la + lb < oend ? pbase + la + lb : oend);
            // head key of each run in a register: one shared load per output
            U ha = ia < la ? ks[ix(pbase + ia)] : (U)0;
            U hb = ib < lb ? ks[ix(bbase + ib)] : (U)0;
            for (; o < stop; ++o) {
                const bool takeB = ia >= la || (ib < lb && hb < ha);
                if (takeB) {
                    kd[ix(o)] = hb;
                    if (PAIRS) vd[ix(o)] = vs[ix(bbase + ib)];
                    ++ib;
                    if (ib < lb) hb = ks[ix(bbase + ib)];
                } else {
                    kd[ix(o)] = ha;
                    if (PAIRS) vd[ix(o)] = vs[ix(pbase + ia)];
                    ++ia;
                    if (ia < la) ha = ks[ix(pbase + ia)];
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
