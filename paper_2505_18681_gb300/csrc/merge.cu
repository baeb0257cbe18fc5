// Bottom-up parallel mergesort (Algorithm 3 of the paper, RefinedParallelMergeSort):
// the array is cut into base runs of chunkSize = T_insertion keys, each run is
// insertion-sorted, then runs are merged pairwise with the run length
// doubling (currSize, 2 currSize, ...) until one run remains.  A run without
// a partner is carried to the next round unchanged.
//
// GPU mapping:
//   K4 merge_block_sort   one CTA per tile of T = T_ins * 2^m keys (the largest
//                         such tile that fits): loads the tile into shared
//                         memory, insertion-sorts its base runs (one thread per
//                         run, in registers for runs of up to 32 4-byte or 16
//                         8-byte keys), then performs the in-tile merge rounds
//                         in shared memory with merge-path splits per thread;
//   K5 merge_partition    for each global round, the merge-path split of every
//                         output tile boundary (binary search along the
//                         cross-diagonal of the two runs of its pair);
//   K6 merge_pass         one CTA per output tile: stages its slices of the two
//                         runs in shared memory, merges them (merge-path per
//                         thread) and writes the tile coalesced.
// All merges are stable: on equal keys the left run's key comes first.  Keys
// are compared through the order-preserving map of their dtype, applied on the
// first load and undone on the last store.
#include "evosort.h"
#include "api_internal.h"
#include "common.cuh"
#include "smem_sort.cuh"

namespace evosort {

namespace {

constexpr int kMB = 256;       // threads per CTA
constexpr int kMEPT = 16;      // keys per thread
constexpr int kMTile = kMB * kMEPT;   // keys per CTA tile (global merge rounds)

struct MergeArgs {
    const void* in;
    void* out;
    void* tmp;
    const uint32_t* vin;
    uint32_t* vout;
    uint32_t* vtmp;
    size_t n;
    KeyMap map;
    int tins;        // base run length (insertion threshold)
    int btile;       // block-sort tile: tins * 2^m <= kMTile
};

// Shared arrays of a tile are padded with one word per 32: index i lives at
// i + i / 32, so lanes whose positions lie a power of two apart (a thread's
// run or its block of outputs) fall in different banks.
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }
constexpr int kMTilePad = kMTile + kMTile / 32;

// ---------------------------------------------------------------------------
// K4: block sort of one tile (base runs insertion-sorted, then merged).
// ---------------------------------------------------------------------------
template <typename U, bool PAIRS>
__global__ void __launch_bounds__(kMB) merge_block_sort(MergeArgs a, int dst_sel, int last) {
    extern __shared__ __align__(16) unsigned char smem[];
    U* k0 = (U*)smem;
    U* k1 = k0 + kMTilePad;
    uint32_t* v0 = (uint32_t*)(k1 + kMTilePad);
    uint32_t* v1 = v0 + (PAIRS ? kMTilePad : 0);
    const int T = a.btile;
    const size_t base = (size_t)blockIdx.x * T;
    const int len = (int)((a.n - base) < (size_t)T ? (a.n - base) : (size_t)T);
    const U* src = (const U*)a.in;
    {
        // every load of a thread is issued before its shared stores
        U t[kMEPT];
        uint32_t tv[PAIRS ? kMEPT : 1];
#pragma unroll
        for (int r = 0; r < kMEPT; ++r) {
            const int i = r * kMB + threadIdx.x;
            if (i < len) {
                t[r] = src[base + i];
                if (PAIRS) tv[PAIRS ? r : 0] = a.vin[base + i];
            }
        }
#pragma unroll
        for (int r = 0; r < kMEPT; ++r) {
            const int i = r * kMB + threadIdx.x;
            if (i < len) {
                k0[pad32(i)] = map_fwd(t[r], a.map);
                if (PAIRS) v0[pad32(i)] = tv[PAIRS ? r : 0];
            }
        }
    }
    __syncthreads();
    // insertion-sorted base runs, then the in-tile merge rounds (Algorithm 3)
    const int which = smem_merge_sort<U, PAIRS, reg_run_max<U>(), true>(k0, k1, v0, v1, len, a.tins);
    const U* ks = which ? k1 : k0;
    const uint32_t* vs = which ? v1 : v0;
    U* dst = dst_sel ? (U*)a.tmp : (U*)a.out;
    uint32_t* vdst = dst_sel ? a.vtmp : a.vout;
    for (int i = threadIdx.x; i < len; i += kMB) {
        dst[base + i] = last ? map_inv(ks[pad32(i)], a.map) : ks[pad32(i)];
        if (PAIRS) vdst[base + i] = vs[pad32(i)];
    }
}

// ---------------------------------------------------------------------------
// K5: merge-path splits of every output tile boundary for runs of width w.
// split[j] = keys of the left run of its pair among outputs [pair start, j*T).
// ---------------------------------------------------------------------------
template <typename U>
__global__ void __launch_bounds__(256) merge_partition(const U* __restrict__ src, size_t n, size_t w,
                                                       size_t ntiles, size_t* __restrict__ split) {
    const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j > ntiles) return;
    size_t o = j * kMTile;
    if (o > n) o = n;
    const size_t pbase = (o / (2 * w)) * (2 * w);
    const size_t la = (pbase + w < n ? pbase + w : n) - pbase;
    const size_t lb = (pbase + 2 * w < n ? pbase + 2 * w : n) - pbase - la;
    const U* A = src + pbase;
    const U* B = A + la;
    split[j] = merge_path<U>([&](size_t i) { return A[i]; }, la, [&](size_t i) { return B[i]; }, lb, o - pbase);
}

// ---------------------------------------------------------------------------
// K6: one output tile of a global merge round.
// The tile's slices of the two runs are staged in shared memory, each thread
// merges kMEPT consecutive outputs from its merge-path split, and the tile is
// written back coalesced.  The staging arrays are padded with one word per 32
// (index i lives at i + i / 32), so the lanes of a warp, whose outputs and
// split points lie about kMEPT keys apart, fall in different banks; the merge
// keeps the head key of each run in a register, one shared load per output.
// ---------------------------------------------------------------------------
// resident CTAs per SM the register budget allows for: 6 for 4-byte keys
// alone, 4 with values or for 8-byte keys, 2 for 8-byte keys with values
template <typename U, bool PAIRS>
__host__ __device__ constexpr int merge_pass_ctas() {
    return sizeof(U) == 4 ? (PAIRS ? 4 : 6) : (PAIRS ? 2 : 4);
}

template <typename U, bool PAIRS>
__global__ void __launch_bounds__(kMB, merge_pass_ctas<U, PAIRS>()) merge_pass(const U* __restrict__ src, U* __restrict__ dst,
                                                  const uint32_t* __restrict__ vsrc, uint32_t* __restrict__ vdst,
                                                  size_t n, size_t w, const size_t* __restrict__ split, KeyMap map,
                                                  int last) {
    extern __shared__ __align__(16) unsigned char smem[];
    U* sk = (U*)smem;                          // staged slices (padded)
    U* so = sk + kMTilePad;                    // merged output (padded)
    uint32_t* sv = (uint32_t*)(so + kMTilePad);
    uint32_t* sov = sv + (PAIRS ? kMTilePad : 0);
    const size_t j = blockIdx.x;
    const size_t o0 = j * kMTile;
    const size_t o1 = o0 + kMTile < n ? o0 + kMTile : n;
    // the tile may straddle one pair boundary; handle each piece in turn
    size_t o = o0;
    int piece = 0;
    while (o < o1) {
        const size_t pbase = (o / (2 * w)) * (2 * w);
        const size_t la = (pbase + w < n ? pbase + w : n) - pbase;
        const size_t lb = (pbase + 2 * w < n ? pbase + 2 * w : n) - pbase - la;
        const size_t pend = pbase + la + lb;
        const size_t e = pend < o1 ? pend : o1;
        // splits at o and e within this pair
        const size_t ka = o - pbase, kb = e - pbase;
        // a piece that starts the tile starts at split[j]; a second piece starts
        // at its pair's beginning.  A piece ends at the pair's end, or at the
        // tile end, whose split (relative to the same pair) is split[j + 1].
        const size_t a0 = (piece == 0) ? split[j] : 0;
        const size_t a1 = (e == pend) ? la : split[j + 1];
        const size_t b0 = ka - a0, b1 = kb - a1;
        const int na = (int)(a1 - a0), nb = (int)(b1 - b0);
        const U* A = src + pbase + a0;
        const U* B = src + pbase + la + b0;
        const int cnt = na + nb;
        {
            // all of a thread's loads are issued before its shared stores, so
            // kMEPT of them are in flight at once
            U t[kMEPT];
            uint32_t tv[PAIRS ? kMEPT : 1];
#pragma unroll
            for (int r = 0; r < kMEPT; ++r) {
                const int i = r * kMB + threadIdx.x;
                if (i < cnt) {
                    const bool inA = i < na;
                    t[r] = inA ? A[i] : B[i - na];
                    if (PAIRS) tv[PAIRS ? r : 0] = inA ? vsrc[pbase + a0 + i] : vsrc[pbase + la + b0 + (i - na)];
                }
            }
#pragma unroll
            for (int r = 0; r < kMEPT; ++r) {
                const int i = r * kMB + threadIdx.x;
                if (i < cnt) {
                    sk[pad32(i)] = t[r];
                    if (PAIRS) sv[pad32(i)] = tv[PAIRS ? r : 0];
                }
            }
        }
        __syncthreads();
        const int q0 = threadIdx.x * kMEPT < cnt ? threadIdx.x * kMEPT : cnt;
        const int q1 = q0 + kMEPT < cnt ? q0 + kMEPT : cnt;
        if (q0 < q1) {
            int ia = (int)merge_path<U>([&](size_t i) { return sk[pad32((int)i)]; }, na,
                                        [&](size_t i) { return sk[pad32(na + (int)i)]; }, nb, (size_t)q0);
            int ib = q0 - ia;
            U ha = ia < na ? sk[pad32(ia)] : (U)0;
            U hb = ib < nb ? sk[pad32(na + ib)] : (U)0;
#pragma unroll 4
            for (int q = q0; q < q1; ++q) {
                // the right run's key goes first only when strictly smaller: stable
                const bool takeB = ia >= na || (ib < nb && hb < ha);
                if (takeB) {
                    so[pad32(q)] = hb;
                    if (PAIRS) sov[pad32(q)] = sv[pad32(na + ib)];
                    ++ib;
                    if (ib < nb) hb = sk[pad32(na + ib)];
                } else {
                    so[pad32(q)] = ha;
                    if (PAIRS) sov[pad32(q)] = sv[pad32(ia)];
                    ++ia;
                    if (ia < na) ha = sk[pad32(ia)];
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += kMB) {
            dst[o + i] = last ? map_inv(so[pad32(i)], map) : so[pad32(i)];
            if (PAIRS) vdst[o + i] = sov[pad32(i)];
        }
        __syncthreads();
        o = e;
        ++piece;
    }
}

template <typename U, bool PAIRS>
int merge_sort_t(const MergeArgs& a0, void* ws, cudaStream_t s, std::string* err) {
    MergeArgs a = a0;
    const size_t n = a.n;
    // global rounds after the block sort
    int rounds = 0;
    for (size_t w = (size_t)a.btile; w < n; w <<= 1) ++rounds;
    const size_t ntiles = (n + kMTile - 1) / kMTile;
    size_t* split = (size_t*)ws;
    const size_t smem_block = (size_t)2 * kMTilePad * (sizeof(U) + (PAIRS ? 4 : 0));
    const size_t smem_pass = smem_block;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(merge_block_sort<U, PAIRS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_block);
        cudaFuncSetAttribute(merge_pass<U, PAIRS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_pass);
        configured = true;
    }
    // block sort: destination chosen so the last round ends in out
    const int dst_sel = (rounds % 2 == 1) ? 1 : 0;   // 1 = tmp
    const size_t nblk = (n + a.btile - 1) / a.btile;
    const int call = prof_call_begin(nullptr, 0, s);
    {
        ProfScope ps(call, EVOSORT_K_MERGE_BLOCK, -1, 2.0 * n * (sizeof(U) + (PAIRS ? 4 : 0)), n, s);
        merge_block_sort<U, PAIRS><<<(unsigned)nblk, kMB, smem_block, s>>>(a, dst_sel, rounds == 0);
    }
    count_launches(1);
    const U* src = dst_sel ? (const U*)a.tmp : (const U*)a.out;
    U* dst = dst_sel ? (U*)a.out : (U*)a.tmp;
    const uint32_t* vsrc = dst_sel ? a.vtmp : a.vout;
    uint32_t* vdst = dst_sel ? a.vout : a.vtmp;
    int r = 0;
    for (size_t w = (size_t)a.btile; w < n; w <<= 1, ++r) {
        {
            ProfScope ps(call, EVOSORT_K_MERGE_PARTITION, r, 0.0, ntiles + 1, s);
            merge_partition<U><<<(unsigned)((ntiles + 1 + 255) / 256), 256, 0, s>>>(src, n, w, ntiles, split);
        }
        {
            ProfScope ps(call, EVOSORT_K_MERGE_PASS, r, 2.0 * n * (sizeof(U) + (PAIRS ? 4 : 0)), n, s);
            merge_pass<U, PAIRS><<<(unsigned)ntiles, kMB, smem_pass, s>>>(src, dst, vsrc, vdst, n, w, split, a.map,
                                                                          r == rounds - 1);
        }
        count_launches(2);
        const U* t = src; src = dst; dst = (U*)t;
        const uint32_t* tv = vsrc; vsrc = vdst; vdst = (uint32_t*)tv;
    }
    prof_call_end(call, s, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("merge launch: ") + cudaGetErrorString(e);
        return EVOSORT_ERR_CUDA;
    }
    return EVOSORT_OK;
}

}  // namespace

static size_t merge_split_bytes(size_t n) {
    return (((n + kMTile - 1) / kMTile + 2) * sizeof(size_t) + 255) / 256 * 256;
}

size_t merge_workspace_bytes(size_t n, int w, bool pairs, const Plan&) {
    return merge_split_bytes(n) + (n * w + 255) / 256 * 256 + (pairs ? (n * 4 + 255) / 256 * 256 : 0);
}

int merge_sort(const void* in, void* out, const uint32_t* vin, uint32_t* vout, size_t n, int dt, const Plan& pl,
               void* ws, size_t ws_bytes, cudaStream_t s, std::string* err) {
    const int w = dtype_bytes(dt);
    const bool pairs = vout != nullptr;
    if (ws_bytes < merge_workspace_bytes(n, w, pairs, pl)) {
        *err = "workspace too small";
        return EVOSORT_ERR_NOMEM;
    }
    MergeArgs a;
    a.in = in;
    a.out = out;
    char* base = (char*)ws + merge_split_bytes(n);
    a.tmp = base;
    a.vin = vin;
    a.vout = vout;
    a.vtmp = pairs ? (uint32_t*)(base + (n * w + 255) / 256 * 256) : nullptr;
    a.n = n;
    a.map = key_map_for(dt, pl.descending);
    a.tins = pl.insertion_threshold;
    int t = a.tins;
    while (t * 2 <= kMTile) t *= 2;
    a.btile = t;
    if (w == 4)
        return pairs ? merge_sort_t<uint32_t, true>(a, ws, s, err) : merge_sort_t<uint32_t, false>(a, ws, s, err);
    return pairs ? merge_sort_t<uint64_t, true>(a, ws, s, err) : merge_sort_t<uint64_t, false>(a, ws, s, err);
}

}  // namespace evosort
