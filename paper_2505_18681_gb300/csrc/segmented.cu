// Batched segmented sort: many independent arrays of uneven length sorted in
// one persistent launch.  Each segment is sorted with the method its length
// calls for:
//   warp tier   (len < warp cap)     one warp, keys in registers, bitonic
//                                    network across the warp's lanes (warp cap
//                                    32..256, a tuning parameter);
//   block tier  (len <= block cap)   one CTA, keys in shared memory, the
//                                    insertion-run + merge sort of Algorithm 3;
//   large tier  (len >  block cap)   one CTA runs the LSD radix sort of
//                                    Algorithms 4a/4b over the segment in global
//                                    memory: one read for all digit histograms,
//                                    then per 8-bit digit a stable tile-by-tile
//                                    scatter.  A single CTA walks the tiles in
//                                    order, so running digit offsets replace the
//                                    device-wide look-back;
//   giant tier  (len >= giant)       the device-wide radix sort, one segment at
//                                    a time, before the persistent launch (one
//                                    CTA per segment would leave the rest of the
//                                    GPU idle once the other segments are done).
// K7 seg_count / seg_scan / seg_fill put the segments in a work list, longest
// first (counting sort by floor(log2(len))); K8 seg_sort drains it.  Giant
// segments are the head of that list: the host reads the list's length
// histogram (one small synchronous copy), sorts the head segments with the
// device-wide path and has K8 start after them.
#include <algorithm>
#include <vector>

#include "evosort.h"
#include "api_internal.h"
#include "common.cuh"
#include "smem_sort.cuh"

namespace evosort {
namespace {

constexpr int kSB = 512;             // threads per CTA
constexpr int kSW = kSB / 32;        // warps per CTA
constexpr int kWKW = 8;              // keys per lane in the warp tier (at most 256 keys)
constexpr int kNB = 48;              // length buckets (floor log2)
constexpr int kLKPT = 8;             // keys per thread per large-tier tile
constexpr int kLTile = kSB * kLKPT;  // keys per large-tier tile

struct SegArgs {
    void* keys;
    const uint64_t* off;
    size_t nseg;
    size_t total;
    KeyMap map;
    void* tmp;          // scratch of total keys (large-tier ping-pong)
    uint32_t* hdr;      // [0..kNB) bucket counts, [kNB..2kNB) bucket cursors,
                        // [2kNB] single items, [2kNB+1] warp-tier segments, [2kNB+2] work counter
    uint32_t* order;    // nseg entries: segment ids, longest first
    uint32_t* status;
    int block_cap;      // keys one CTA sorts in shared memory
    int tins;           // base run of the shared-memory merge sort
    int warp_log2;      // warp tier: len < 2^warp_log2
    uint32_t skip;      // work items sorted before K8 (giant segments)
};

__device__ __forceinline__ int len_bucket(uint64_t len) { return 63 - __clzll((long long)len); }

// L2 prefetch of the 16-byte-aligned part of [p, p + bytes) by the TMA
// engine (no shared memory is written; nothing outside the range is read).
__device__ __forceinline__ void prefetch_l2_inner(const void* p, size_t bytes) {
    const uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    if (e > a) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(e - a)) : "memory");
}

// A segment is sorted only if it lies inside the array: lo <= hi <= total.
// Any other segment is reported (ST_BAD_OFFSETS) and left out of the work
// list, so no tier ever reads or writes outside [0, total).  total < 2^40 is
// checked on the host, so a valid length always has a bucket below kNB.
__device__ __forceinline__ bool seg_ok(const SegArgs& a, uint64_t lo, uint64_t hi) {
    return lo <= hi && hi <= a.total;
}

// K7a: validate offsets, count segments per length bucket.
__global__ void seg_count(SegArgs a) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (a.off[0] != 0 || a.off[a.nseg] != a.total)) atomicOr(a.status, ST_BAD_OFFSETS);
    if (i >= a.nseg) return;
    const uint64_t lo = a.off[i], hi = a.off[i + 1];
    if (!seg_ok(a, lo, hi)) {
        atomicOr(a.status, ST_BAD_OFFSETS);
        return;
    }
    const uint64_t len = hi - lo;
    if (len >= 2) atomicAdd(&a.hdr[len_bucket(len)], 1u);
}

// K7b: bucket cursors in descending length order, item counts.
__global__ void seg_scan(SegArgs a) {
    if (threadIdx.x != 0) return;
    uint32_t pos = 0, single = 0, warp = 0;
    for (int b = kNB - 1; b >= 1; --b) {
        a.hdr[kNB + b] = pos;
        pos += a.hdr[b];
        if (b >= a.warp_log2)
            single += a.hdr[b];
        else
            warp += a.hdr[b];
    }
    a.hdr[2 * kNB] = single;
    a.hdr[2 * kNB + 1] = warp;
    a.hdr[2 * kNB + 2] = 0;
}

// K7c: scatter segment ids into the work list.
__global__ void seg_fill(SegArgs a) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nseg) return;
    const uint64_t lo = a.off[i], hi = a.off[i + 1];
    if (!seg_ok(a, lo, hi) || hi - lo < 2) return;
    const uint32_t p = atomicAdd(&a.hdr[kNB + len_bucket(hi - lo)], 1u);
    a.order[p] = (uint32_t)i;
}

// ---------------------------------------------------------------------------
// Tiers.
// ---------------------------------------------------------------------------
template <typename U>
__device__ void warp_tier(const SegArgs& a, uint64_t lo, int len) {
    const int lane = threadIdx.x & 31;
    U* keys = (U*)a.keys + lo;
    U k[kWKW];
#pragma unroll
    for (int r = 0; r < kWKW; ++r) {
        const int i = lane * kWKW + r;
        k[r] = i < len ? map_fwd(keys[i], a.map) : ~(U)0;
    }
    warp_bitonic_sort<U, kWKW>(k);
#pragma unroll
    for (int r = 0; r < kWKW; ++r) {
        const int i = lane * kWKW + r;
        if (i < len) keys[i] = map_inv(k[r], a.map);
    }
}

template <typename U>
__device__ void block_tier(const SegArgs& a, unsigned char* smem, uint64_t lo, int len) {
    U* k0 = (U*)smem;
    U* k1 = k0 + a.block_cap;
    U* keys = (U*)a.keys + lo;
    for (int i = threadIdx.x; i < len; i += kSB) k0[i] = map_fwd(keys[i], a.map);
    __syncthreads();
    const int which = smem_merge_sort<U, false>(k0, k1, nullptr, nullptr, len, a.tins);
    const U* ks = which ? k1 : k0;
    for (int i = threadIdx.x; i < len; i += kSB) keys[i] = map_inv(ks[i], a.map);
    __syncthreads();
}

template <typename U>
__device__ void large_tier(const SegArgs& a, unsigned char* smem, uint64_t lo, uint64_t len) {
    constexpr int NP = sizeof(U);          // 8-bit digits
    constexpr int BINS = 256;
    uint32_t* s_hist = (uint32_t*)smem;                 // NP * BINS
    uint32_t* s_run = s_hist + NP * BINS;               // BINS running offsets
    uint32_t* s_excl = s_run + BINS;                    // BINS tile offsets
    uint32_t* s_tcnt = s_excl + BINS;                   // BINS tile counts
    uint32_t* s_match = s_tcnt + BINS;                  // kSW * BINS match masks
    uint16_t* s_whist = (uint16_t*)(s_match + kSW * BINS);   // kSW * BINS
    U* s_r = (U*)(s_whist + kSW * BINS);               // kLTile reorder buffer
    __shared__ uint32_t s_scr[kSW + 1];
    __shared__ int s_active[NP];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    U* keys = (U*)a.keys + lo;
    U* tmp = (U*)a.tmp + lo;
    for (int i = tid; i < NP * BINS; i += kSB) s_hist[i] = 0;
    if (tid < NP) s_active[tid] = 0;
    __syncthreads();
    // one read of the segment for every pass's digit counts (unrolled, so
    // several of a thread's loads are in flight)
#pragma unroll 4
    for (uint64_t i = tid; i < len; i += kSB) {
        const U k = map_fwd(keys[i], a.map);
#pragma unroll
        for (int p = 0; p < NP; ++p) atomicAdd(&s_hist[p * BINS + digit_of(k, 8 * p, 0xFFu)], 1u);
    }
    __syncthreads();
    // a pass is needed unless one digit value holds every key
    for (int i = tid; i < NP * BINS; i += kSB)
        if (s_hist[i] != 0 && s_hist[i] != (uint32_t)len) s_active[i / BINS] = 1;
    __syncthreads();
    int nact = 0;
    for (int p = 0; p < NP; ++p) nact += s_active[p];
    if (nact == 0) return;   // every key equal: already sorted

    const U* src = keys;
    U* dst = tmp;
    int done = 0;
    const uint32_t lt = lanemask_lt();
    for (int p = 0; p < NP; ++p) {
        if (!s_active[p]) continue;
        const bool first = done == 0, last = done == nact - 1;
        const int shift = 8 * p;
        // running offsets: exclusive prefix of this pass's digit counts
        {
            const uint32_t c = tid < BINS ? s_hist[p * BINS + tid] : 0u;
            uint32_t tot;
            const uint32_t ex = block_exclusive_scan<kSB>(c, s_scr, &tot);
            if (tid < BINS) s_run[tid] = ex;
        }
        __syncthreads();
        for (uint64_t t0 = 0; t0 < len; t0 += kLTile) {
            const int valid = (len - t0) < (uint64_t)kLTile ? (int)(len - t0) : kLTile;
            uint16_t* wh = s_whist + warp * BINS;
            uint32_t* wm = s_match + warp * BINS;
            for (int i = lane; i < BINS; i += 32) {
                wm[i] = 0u;
                if ((i & 1) == 0) ((uint32_t*)wh)[i >> 1] = 0u;
            }
            __syncwarp();
            U key[kLKPT];
            uint32_t dr[kLKPT];
            const int wofs = warp * 32 * kLKPT + lane;
            // the tile's keys are all loaded before the ranking starts, so a
            // warp waits for one round trip per tile, not one per column; the
            // next tile is pulled into L2 meanwhile
            if (tid == 0 && t0 + kLTile < len) {
                const uint64_t nv = (len - t0 - kLTile) < (uint64_t)kLTile ? (len - t0 - kLTile) : (uint64_t)kLTile;
                prefetch_l2_inner(src + t0 + kLTile, nv * sizeof(U));
            }
#pragma unroll
            for (int i = 0; i < kLKPT; ++i) {
                const int s = wofs + 32 * i;
                key[i] = s < valid ? src[t0 + s] : ~(U)0;
            }
#pragma unroll
            for (int i = 0; i < kLKPT; ++i) {
                const int s = wofs + 32 * i;
                U k = key[i];
                if (first && s < valid) k = map_fwd(k, a.map);
                key[i] = k;
                const uint32_t dig = digit_of(k, shift, 0xFFu);
                atomicOr(&wm[dig], 1u << lane);
                __syncwarp();
                const uint32_t peers = wm[dig];
                __syncwarp();
                const int leader = 31 - __clz(peers);
                uint32_t old = 0;
                if (lane == leader) {
                    old = wh[dig];
                    wh[dig] = (uint16_t)(old + __popc(peers));
                    wm[dig] = 0u;
                }
                old = __shfl_sync(0xffffffffu, old, leader);
                dr[i] = dig | ((old + __popc(peers & lt)) << 16);
                __syncwarp();
            }
            __syncthreads();
            // tile digit counts and exclusive prefixes over warps
            uint32_t tc = 0;
            if (tid < BINS) {
                for (int w = 0; w < kSW; ++w) {
                    const uint32_t c = s_whist[w * BINS + tid];
                    s_whist[w * BINS + tid] = (uint16_t)tc;
                    tc += c;
                }
                s_tcnt[tid] = tc;
            }
            {
                uint32_t tot;
                const uint32_t ex = block_exclusive_scan<kSB>(tc, s_scr, &tot);
                if (tid < BINS) s_excl[tid] = ex;
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kLKPT; ++i) {
                const int s = wofs + 32 * i;
                if (s < valid) {
                    const uint32_t dig = dr[i] & 0xFFFFu;
                    s_r[s_excl[dig] + wh[dig] + (dr[i] >> 16)] = key[i];
                }
            }
            __syncthreads();
            for (int s = tid; s < valid; s += kSB) {
                const U k = s_r[s];
                const uint32_t dig = digit_of(k, shift, 0xFFu);
                dst[s_run[dig] + (s - s_excl[dig])] = last ? map_inv(k, a.map) : k;
            }
            __syncthreads();
            if (tid < BINS) s_run[tid] += s_tcnt[tid];
            __syncthreads();
        }
        const U* t = src;
        src = dst;
        dst = (U*)t;
        ++done;
    }
    if (nact & 1) {   // result is in the scratch copy
        for (uint64_t i = tid; i < len; i += kSB) keys[i] = tmp[i];
        __syncthreads();
    }
}

template <typename U>
__global__ void __launch_bounds__(kSB, 2) seg_sort(SegArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_item;
    const uint32_t single = a.hdr[2 * kNB];
    const uint32_t nwarp = a.hdr[2 * kNB + 1];
    const uint32_t nbatch = (nwarp + kSW - 1) / kSW;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&a.hdr[2 * kNB + 2], 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= single + nbatch) break;
        if (item < a.skip) continue;   // sorted by the device-wide path
        if (item < single) {
            const uint32_t seg = a.order[item];
            const uint64_t lo = a.off[seg], len = a.off[seg + 1] - lo;
            if (len <= (uint64_t)a.block_cap)
                block_tier<U>(a, smem, lo, (int)len);
            else
                large_tier<U>(a, smem, lo, len);
        } else {
            const uint32_t j = (item - single) * kSW + (threadIdx.x >> 5);
            if (j < nwarp) {
                const uint32_t seg = a.order[single + j];
                const uint64_t lo = a.off[seg];
                warp_tier<U>(a, lo, (int)(a.off[seg + 1] - lo));
            }
        }
    }
}

// (lo, len) of the first `count` work items (the longest segments).
__global__ void seg_head(SegArgs a, uint32_t count, unsigned long long* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint32_t seg = a.order[i];
    out[2 * i] = a.off[seg];
    out[2 * i + 1] = a.off[seg + 1] - a.off[seg];
}

size_t seg_smem_bytes(int w, int block_cap) {
    const size_t large = (size_t)w * 256 * 4 + 3 * 256 * 4 + kSW * 256 * 4 + kSW * 256 * 2 + (size_t)kLTile * w;
    const size_t block = (size_t)2 * block_cap * w;
    return large > block ? large : block;
}

size_t seg_hdr_bytes() { return 256 * sizeof(uint32_t); }

}  // namespace

size_t segmented_workspace_bytes(size_t total, size_t nseg, int w) {
    return seg_hdr_bytes() + (nseg * 4 + 255) / 256 * 256 + (total * w + 255) / 256 * 256;
}

static int segmented_giant(SegArgs& a, int dt, const Plan& pl, int gb, cudaStream_t s, uint32_t* skip,
                           std::string* err);

int segmented_sort(void* keys, size_t total, const uint64_t* off, size_t nseg, int dt, const Plan& pl, void* ws,
                   size_t ws_bytes, bool caller_ws, cudaStream_t s, std::string* err) {
    const int w = dtype_bytes(dt);
    if (ws_bytes < segmented_workspace_bytes(total, nseg, w)) {
        *err = "workspace too small";
        return EVOSORT_ERR_NOMEM;
    }
    uint32_t* status = status_word(err);
    if (!status) return EVOSORT_ERR_CUDA;
    SegArgs a;
    a.keys = keys;
    a.off = off;
    a.nseg = nseg;
    a.total = total;
    a.map = key_map_for(dt, pl.descending);
    a.hdr = (uint32_t*)ws;
    a.order = (uint32_t*)((char*)ws + seg_hdr_bytes());
    a.tmp = (char*)ws + seg_hdr_bytes() + (nseg * 4 + 255) / 256 * 256;
    a.status = status;
    a.block_cap = pl.seg_block_cap;
    a.tins = pl.insertion_threshold > 64 ? 16 : pl.insertion_threshold;
    a.warp_log2 = 31 - __builtin_clz((unsigned)pl.seg_warp_cap);
    a.skip = 0;
    const size_t smem = seg_smem_bytes(w, a.block_cap);
    const int sms = sm_count();
    cudaError_t e = cudaMemsetAsync(ws, 0, seg_hdr_bytes(), s);
    const unsigned g = (unsigned)((nseg + 255) / 256);
    const int call = prof_call_begin(nullptr, 0, s);
    {
        ProfScope ps(call, EVOSORT_K_SEGMENTED, 0, 0.0, nseg, s);
        if (e == cudaSuccess && g) {
            seg_count<<<g, 256, 0, s>>>(a);
            seg_scan<<<1, 32, 0, s>>>(a);
            seg_fill<<<g, 256, 0, s>>>(a);
            e = cudaGetLastError();
        }
    }
    // giant tier: not while the stream is being captured (the length
    // histogram read would synchronise), nor with a caller workspace (the
    // device-wide path takes its own scratch)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (e == cudaSuccess && pl.seg_giant > 0 && !caller_ws && total >= (size_t)pl.seg_giant)
        e = cudaStreamIsCapturing(s, &cap);
    if (e == cudaSuccess && pl.seg_giant > 0 && !caller_ws && total >= (size_t)pl.seg_giant &&
        cap == cudaStreamCaptureStatusNone) {
        const int gb = 63 - __builtin_clzll((unsigned long long)pl.seg_giant);
        const int rc = segmented_giant(a, dt, pl, gb, s, &a.skip, err);
        if (rc != EVOSORT_OK) return rc;
    }
    {
        ProfScope ps(call, EVOSORT_K_SEGMENTED, 1, 2.0 * total * w, total, s);
        if (e == cudaSuccess) {
            static int resident[2] = {0, 0};
            const int wi = w == 4 ? 0 : 1;
            auto kern = w == 4 ? (void (*)(SegArgs))seg_sort<uint32_t> : (void (*)(SegArgs))seg_sort<uint64_t>;
            if (resident[wi] == 0) {
                // sized for the largest block tier allowed, so every seg_block_cap fits
                const size_t smax = seg_smem_bytes(w, w == 4 ? 8192 : 4096);
                e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
                int nb = 0;
                if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kSB, smax);
                resident[wi] = nb > 0 ? nb : 1;
            }
            if (e == cudaSuccess) {
                if (w == 4)
                    seg_sort<uint32_t><<<(unsigned)(sms * resident[wi]), kSB, smem, s>>>(a);
                else
                    seg_sort<uint64_t><<<(unsigned)(sms * resident[wi]), kSB, smem, s>>>(a);
                e = cudaGetLastError();
            }
        }
    }
    prof_call_end(call, s, nullptr);
    count_launches(4);
    if (e != cudaSuccess) {
        *err = std::string("segmented launch: ") + cudaGetErrorString(e);
        return EVOSORT_ERR_CUDA;
    }
    return EVOSORT_OK;
}

// Giant tier: after K7, count the segments of at least 2^gb keys from the
// length histogram, sort each with the device-wide radix path (scratch from
// the stream-ordered pool, sized for the longest), and return how many head
// items K8 must skip.  Returns 0 items when there are none.
static int segmented_giant(SegArgs& a, int dt, const Plan& pl, int gb, cudaStream_t s, uint32_t* skip,
                           std::string* err) {
    *skip = 0;
    uint32_t hist[kNB];
    cudaError_t e = cudaMemcpyAsync(hist, a.hdr, sizeof(hist), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        *err = std::string("segmented sort: length histogram read: ") + cudaGetErrorString(e);
        return EVOSORT_ERR_CUDA;
    }
    uint32_t k = 0;
    for (int b = gb; b < kNB; ++b) k += hist[b];
    if (k == 0) return EVOSORT_OK;
    std::vector<unsigned long long> head(2 * (size_t)k);
    unsigned long long* d_head = nullptr;
    e = cudaMallocAsync((void**)&d_head, head.size() * sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        seg_head<<<(k + 255) / 256, 256, 0, s>>>(a, k, d_head);
        count_launches(1);
        e = cudaMemcpyAsync(head.data(), d_head, head.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFreeAsync(d_head, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        *err = std::string("segmented sort: giant segment list: ") + cudaGetErrorString(e);
        return EVOSORT_ERR_CUDA;
    }
    const int w = dtype_bytes(dt);
    size_t longest = 0;
    for (uint32_t i = 0; i < k; ++i) longest = std::max<size_t>(longest, head[2 * i + 1]);
    Plan rp;
    default_radix_plan(dt, &rp, longest);
    rp.descending = pl.descending;
    const size_t need = radix_workspace_bytes(longest, w, false, rp);
    void* ws = nullptr;
    e = cudaMallocAsync(&ws, need, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *err = std::string("segmented sort: giant segment scratch: ") + cudaGetErrorString(e);
        return EVOSORT_ERR_NOMEM;
    }
    int rc = EVOSORT_OK;
    for (uint32_t i = 0; i < k && rc == EVOSORT_OK; ++i) {
        void* seg = (char*)a.keys + head[2 * i] * w;
        Plan sp;
        default_radix_plan(dt, &sp, head[2 * i + 1]);
        sp.descending = pl.descending;
        rc = radix_sort(seg, seg, nullptr, nullptr, head[2 * i + 1], dt, sp, ws, need, s, err);
    }
    cudaFreeAsync(ws, s);
    *skip = k;
    return rc;
}

}  // namespace evosort
