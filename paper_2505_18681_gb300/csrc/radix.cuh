// LSD radix sort kernels (Section 3.1; Algorithms 4a/4b of the paper).
//
// The paper's pass is: per-thread digit histograms, a global reduce and
// exclusive prefix sum over digit counts, thread-wise write offsets, a stable
// scatter into a temporary array, then a buffer swap.  On the GPU the pass
// becomes one "onesweep" kernel per digit:
//
//   K1 radix_histogram   one read of all keys counts the digits of every pass
//                        (the per-thread histograms of all passes at once);
//   K2 radix_scan_plan   exclusive prefix sum of each pass's digit counts; a
//                        pass whose digit is the same for every key is skipped,
//                        and the ping-pong buffer chain is planned on the device;
//   K3 radix_onesweep    per tile: stable digit ranking in the tile, tile digit
//                        histogram, decoupled look-back over preceding tiles for
//                        the per-digit write offsets (the "thread-wise offsets"
//                        of the paper, with tiles in place of threads), then a
//                        shared-memory reorder and a coalesced stable scatter;
//   K3b radix_fixup      copies the result into the output buffer when no pass
//                        ran (out-of-place) or an odd number of passes ran
//                        (in-place).
#pragma once

#include "common.cuh"

namespace evosort {

// Buffer selectors of the pass chain.
enum : int { BUF_IN = 0, BUF_OUT = 1, BUF_TMP = 2 };
enum : int { FIX_NONE = 0, FIX_IN_TO_OUT = 1, FIX_TMP_TO_OUT = 2, FIX_REVERSE = 3 };

// Order flags K1 records while it counts (words of RadixArgs::order): a pair
// of neighbours that descends, that ascends, that is equal (in the order the
// sort produces, i.e. on the mapped keys).
enum : int { ORD_DESCENT = 0, ORD_ASCENT = 1, ORD_EQUAL = 2 };
// Range words (64-bit, zeroed with the scratch): the largest complement of a
// mapped key (so ~word = the smallest key), the largest mapped key, the bias
// the passes subtract (0 unless rebased), and flags.
enum : int { RNG_NOTMIN = 0, RNG_MAX = 1, RNG_BIAS = 2, RNG_FLAGS = 3, RNG_WORDS = 4 };
enum : unsigned { RNG_RECORDED = 1u, RNG_REBASED = 2u };

struct PassDesc {
    int active;   // 0: the digit is constant over all keys, pass skipped
    int src, dst; // buffer selectors
    int xin;      // apply to_ordered on load (first active pass)
    int xout;     // apply from_ordered on store (last active pass)
    int fixup;    // used in the entry after the last pass
    int rank;     // adaptive ranking: the rank mode this pass runs with
    int pad1;
};

struct RadixArgs {
    const void* in;
    void* out;
    void* tmp;
    const uint32_t* vin;
    uint32_t* vout;
    uint32_t* vtmp;
    size_t n;
    int dt;
    KeyMap map;      // order-preserving key map of dt
    int d;           // digit bits
    int npass;       // ceil(8w / d)
    int lb64;        // look-back slots are 64-bit (n >= 2^30)
    int adapt;       // ranking chosen per pass by K2 (PassDesc::rank)
    double conc_later, conc_first;   // adaptive ranking thresholds (see radix_scan_plan)
    uint32_t spin_limit;             // polls of a look-back slot before a wait gives up
    size_t ntiles;   // tiles per pass
    PassDesc* desc;             // npass + 1 entries
    unsigned long long* counts; // npass << d digit counts, then exclusive offsets
    void* lookback;             // slots [pass][tile][digit]
    uint32_t* tile_counter;     // npass counters
    uint32_t* order;            // 3 order flags (ORD_*), zeroed with the counters
    unsigned long long* range;  // RNG_WORDS words (RNG_*), zeroed with the counters
    unsigned long long* counts2;   // npass << d digit counts of the rebased keys
    uint32_t* status;
};

// Range reduction ("rebase"): when the mapped keys span fewer 8-bit digits
// than the raw digits that vary (keys of both signs near zero differ in all
// their high bytes), the passes rank key - min instead of the key: the same
// order, with only ceil(bits(max - min) / 8) digits left to sort.  The
// smallest mapped key is subtracted on the first pass's load and added back
// on the last pass's store.
template <typename U>
__device__ __forceinline__ U rank_key(U raw, const KeyMap& m, U bias) {
    return map_fwd(raw, m) - bias;
}
template <typename U>
__device__ __forceinline__ U unrank_key(U k, const KeyMap& m, U bias) {
    return map_inv((U)(k + bias), m);
}
// The bias the pass kernels subtract (0 when the sort is not rebased).
template <typename U>
__device__ __forceinline__ U pass_bias(const RadixArgs& a) {
    return a.range ? (U)a.range[RNG_BIAS] : (U)0;
}

template <typename U>
__device__ __forceinline__ const U* sel_src(const RadixArgs& a, int s) {
    return s == BUF_IN ? (const U*)a.in : (s == BUF_OUT ? (const U*)a.out : (const U*)a.tmp);
}
template <typename U>
__device__ __forceinline__ U* sel_dst(const RadixArgs& a, int s) {
    return s == BUF_OUT ? (U*)a.out : (U*)a.tmp;
}
__device__ __forceinline__ const uint32_t* sel_vsrc(const RadixArgs& a, int s) {
    return s == BUF_IN ? a.vin : (s == BUF_OUT ? a.vout : a.vtmp);
}
__device__ __forceinline__ uint32_t* sel_vdst(const RadixArgs& a, int s) {
    return s == BUF_OUT ? a.vout : a.vtmp;
}

// ---------------------------------------------------------------------------
// K1: digit histograms of every pass in one read of the keys.
// Shared counters per CTA, replicated in `cols` columns (lane % cols): the
// counter of (pass, digit, column) sits at ((pass * bins + digit) * cols +
// column), so with 32 columns each lane only ever touches its own bank and
// the shared atomics never conflict.  Each thread reads a run of HC
// consecutive keys and merges consecutive equal digits before the atomic;
// when a whole warp ends its runs on one digit (sorted and low-entropy input)
// the warp adds one reduced count instead of 32.
// While it counts, K1 also compares every key with its successor and records
// whether any pair descends, ascends or is equal (ORD_* flags): K2 then
// turns an input that is already in order into a copy, and one in exactly
// reverse order into a reversed copy, instead of running the passes.
// ---------------------------------------------------------------------------
constexpr int kHistThreads = 1024;
constexpr size_t kHistSmem = 128 * 1024;

// columns of the histogram for a pass count and digit width (power of two)
__host__ __device__ constexpr int hist_cols(int npass, int d) {
    int c = 32;
    while (c > 1 && (size_t)npass * ((size_t)1 << d) * c * 4 > kHistSmem) c >>= 1;
    return c;
}

__device__ __forceinline__ void hist_add_run(uint32_t* h, int cols, uint32_t dig, uint32_t run, bool warp_full) {
    const int lane = threadIdx.x & 31;
    if (warp_full) {
        const uint32_t d0 = __shfl_sync(0xffffffffu, dig, 0);
        if (__all_sync(0xffffffffu, dig == d0)) {
            const uint32_t t = __reduce_add_sync(0xffffffffu, run);
            if (lane == 0) atomicAdd(&h[d0 * cols], t);
            return;
        }
    }
    atomicAdd(&h[dig * cols + (lane & (cols - 1))], run);
}

template <typename U>
__global__ void __launch_bounds__(kHistThreads) radix_histogram(RadixArgs a) {
    extern __shared__ uint32_t s_h[];
    const int bins = 1 << a.d;
    const int cols = hist_cols(a.npass, a.d);
    const int total = a.npass * bins;
    const uint32_t mask = (uint32_t)(bins - 1);
    for (int i = threadIdx.x; i < total * cols; i += blockDim.x) s_h[i] = 0;
    __syncthreads();

    constexpr int V = 16 / sizeof(U);   // keys per 128-bit load
    constexpr int HC = 16;              // keys per thread run
    const U* keys = (const U*)a.in;
    const size_t n = a.n;
    const KeyMap map = a.map;
    const int lane = threadIdx.x & 31;
    const int col = lane & (cols - 1);
    // 16-byte aligned body of whole warp chunks (32 runs of HC keys); the
    // head and the tail use scalar loads
    size_t head = ((16 - ((uintptr_t)keys & 15)) & 15) / sizeof(U);
    if (head > n) head = n;
    const size_t nchunks = (n - head) / (32 * HC);
    const size_t tail0 = head + nchunks * 32 * HC;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t gthreads = (size_t)gridDim.x * blockDim.x;

    bool dsc = false, asc = false, eq = false;   // order relations seen by this thread
    auto relate = [&](U x, U y) {   // x precedes y in memory (both mapped)
        dsc |= x > y;
        asc |= x < y;
        eq |= x == y;
    };
    auto count_key = [&](size_t i) {
        const U k = map_fwd(keys[i], map);
        for (int p = 0; p < a.npass; ++p)
            atomicAdd(&s_h[(p * bins + digit_of(k, p * a.d, mask)) * cols + col], 1u);
        if (i + 1 < n) relate(k, map_fwd(keys[i + 1], map));
    };
    if (gtid < head) count_key(gtid);
    if (gtid < n - tail0) count_key(tail0 + gtid);

    // warps take 32 runs (32 * HC consecutive keys) at a time; lane L reads
    // the 16-byte vectors L, L + 32, ... of the warp's chunk, so every load
    // instruction covers 512 contiguous bytes
    const size_t warp_id = gtid >> 5;
    const size_t nwarps = gthreads >> 5;
    for (size_t c = warp_id; c < nchunks; c += nwarps) {
        const bool warp_full = true;
        {
            U k[HC];
            const uint4* vp = (const uint4*)(keys + head + c * 32 * HC);
#pragma unroll
            for (int j = 0; j < HC / V; ++j) {
                const uint4 v = __ldcs(vp + j * 32 + lane);
                memcpy(&k[j * V], &v, 16);
            }
#pragma unroll
            for (int j = 0; j < HC; ++j) k[j] = map_fwd(k[j], map);
            // neighbours: inside a vector (this thread), from one vector to the
            // next (the next lane, or lane 0's next vector for lane 31), and
            // from the chunk's last key to the next key in memory
#pragma unroll
            for (int j = 0; j < HC / V; ++j) {
#pragma unroll
                for (int t = 0; t + 1 < V; ++t) relate(k[j * V + t], k[j * V + t + 1]);
                const U nx = __shfl_down_sync(0xffffffffu, k[j * V], 1);
                const U nx0 = __shfl_sync(0xffffffffu, k[(j + 1 < HC / V ? j + 1 : j) * V], 0);
                if (lane < 31) {
                    relate(k[j * V + V - 1], nx);
                } else if (j + 1 < HC / V) {
                    relate(k[j * V + V - 1], nx0);
                } else {
                    const size_t after = head + (c + 1) * 32 * HC;   // first key after this chunk
                    if (after < n) relate(k[j * V + V - 1], map_fwd(keys[after], map));
                }
            }
            for (int p = 0; p < a.npass; ++p) {
                const int sh = p * a.d;
                uint32_t* h = s_h + (size_t)p * bins * cols;
                uint32_t cur = digit_of(k[0], sh, mask);
                uint32_t run = 1;
#pragma unroll
                for (int j = 1; j < HC; ++j) {
                    const uint32_t dg = digit_of(k[j], sh, mask);
                    if (dg == cur) {
                        ++run;
                    } else {
                        atomicAdd(&h[cur * cols + col], run);
                        cur = dg;
                        run = 1;
                    }
                }
                hist_add_run(h, cols, cur, run, warp_full);
            }
        }
    }
    if (__any_sync(0xffffffffu, dsc) && lane == 0) atomicOr(&a.order[ORD_DESCENT], 1u);
    if (__any_sync(0xffffffffu, asc) && lane == 0) atomicOr(&a.order[ORD_ASCENT], 1u);
    if (__any_sync(0xffffffffu, eq) && lane == 0) atomicOr(&a.order[ORD_EQUAL], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        uint32_t sum = 0;
        for (int c = 0; c < cols; ++c) sum += s_h[i * cols + ((c + i) & (cols - 1))];
        if (sum) atomicAdd(&a.counts[i], (unsigned long long)sum);
    }
}

// K1 for 8-bit digits (the default): the pass count and every digit's shift
// are compile-time constants, and each key adds one to its lane's column of
// each pass's counters directly (no run merging: the columns already keep a
// warp's atomics apart, and merging costs a compare per digit on random
// keys).  Counters of 64-bit keys use 16 columns (2 lanes per column) to fit
// 128 KB.  The order relations are recorded as in the generic kernel, and so
// are the smallest and largest mapped keys (RNG_* words).
// With REBASE (K1b, launched after K1) the kernel first decides whether the
// sort is rebased: only when the span of the mapped keys needs fewer 8-bit
// digits than the passes whose raw digit varies.  If not, it returns at
// once; if so, it counts the digits of key - min into counts2 (and its first
// CTA publishes the bias), which K2 then uses in place of the raw counts.
template <typename U, bool REBASE>
__global__ void __launch_bounds__(kHistThreads) radix_histogram8(RadixArgs a) {
    extern __shared__ uint32_t s_h[];
    constexpr int NP = (int)sizeof(U);
    constexpr int BINS = 256;
    constexpr int COLS = hist_cols(NP, 8);
    __shared__ unsigned s_triv;
    __shared__ int s_go;
    __shared__ U s_bias;
    if (REBASE) {
        if (!(a.range[RNG_FLAGS] & RNG_RECORDED)) return;
        if (threadIdx.x == 0) s_triv = 0u;
        __syncthreads();
        // passes whose raw digit is constant (one digit holds every key)
        for (int i = threadIdx.x; i < NP * BINS; i += blockDim.x)
            if (a.counts[i] == (unsigned long long)a.n) atomicOr(&s_triv, 1u << (i / BINS));
        __syncthreads();
        if (threadIdx.x == 0) {
            const int varying = NP - __popc(s_triv);
            const U mn = (U)~(U)a.range[RNG_NOTMIN];
            const U span = (U)((U)a.range[RNG_MAX] - mn);
            const int bits = span ? 64 - __clzll((long long)(unsigned long long)span) : 0;
            s_go = (bits + 7) / 8 < varying ? 1 : 0;
            s_bias = mn;
            if (s_go && blockIdx.x == 0) {
                a.range[RNG_BIAS] = (unsigned long long)mn;
                atomicOr(&a.range[RNG_FLAGS], (unsigned long long)RNG_REBASED);
            }
        }
        __syncthreads();
        if (!s_go) return;
    }
    const U bias = REBASE ? s_bias : (U)0;
    unsigned long long* const cnt_out = REBASE ? a.counts2 : a.counts;
    for (int i = threadIdx.x; i < NP * BINS * COLS; i += blockDim.x) s_h[i] = 0;
    __syncthreads();

    constexpr int V = 16 / sizeof(U);
    constexpr int HC = 64 / sizeof(U);   // keys per thread per chunk (16 registers of keys)
    const U* keys = (const U*)a.in;
    const size_t n = a.n;
    const KeyMap map = a.map;
    const int lane = threadIdx.x & 31;
    uint32_t* hcol = s_h + (lane & (COLS - 1));
    size_t head = ((16 - ((uintptr_t)keys & 15)) & 15) / sizeof(U);
    if (head > n) head = n;
    const size_t nchunks = (n - head) / (32 * HC);
    const size_t tail0 = head + nchunks * 32 * HC;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t gthreads = (size_t)gridDim.x * blockDim.x;

    auto add = [&](U k) {
#pragma unroll
        for (int p = 0; p < NP; ++p)
            atomicAdd(&hcol[(p * BINS + (uint32_t)((k >> (8 * p)) & 0xFFu)) * COLS], 1u);
    };
    bool dsc = false, asc = false, eq = false;
    auto relate = [&](U x, U y) {
        if (REBASE) return;
        dsc |= x > y;
        asc |= x < y;
        eq |= x == y;
    };
    U notmin = 0, maxk = 0;   // largest ~key and largest key seen (0 = identity)
    auto extent = [&](U k) {
        if (REBASE) return;
        notmin = (U)~k > notmin ? (U)~k : notmin;
        maxk = k > maxk ? k : maxk;
    };
    auto count_key = [&](size_t i) {
        const U k = map_fwd(keys[i], map);
        extent(k);
        add((U)(k - bias));
        if (i + 1 < n) relate(k, map_fwd(keys[i + 1], map));
    };
    if (gtid < head) count_key(gtid);
    if (gtid < n - tail0) count_key(tail0 + gtid);

    const size_t warp_id = gtid >> 5;
    const size_t nwarps = gthreads >> 5;
    for (size_t c = warp_id; c < nchunks; c += nwarps) {
        U k[HC];
        const uint4* vp = (const uint4*)(keys + head + c * 32 * HC);
#pragma unroll
        for (int j = 0; j < HC / V; ++j) {
            const uint4 v = __ldcs(vp + j * 32 + lane);
            memcpy(&k[j * V], &v, 16);
        }
#pragma unroll
        for (int j = 0; j < HC; ++j) k[j] = map_fwd(k[j], map);
        if (!REBASE) {
#pragma unroll
        for (int j = 0; j < HC / V; ++j) {
#pragma unroll
            for (int t = 0; t + 1 < V; ++t) relate(k[j * V + t], k[j * V + t + 1]);
            const U nx = __shfl_down_sync(0xffffffffu, k[j * V], 1);
            const U nx0 = __shfl_sync(0xffffffffu, k[(j + 1 < HC / V ? j + 1 : j) * V], 0);
            if (lane < 31) {
                relate(k[j * V + V - 1], nx);
            } else if (j + 1 < HC / V) {
                relate(k[j * V + V - 1], nx0);
            } else {
                const size_t after = head + (c + 1) * 32 * HC;
                if (after < n) relate(k[j * V + V - 1], map_fwd(keys[after], map));
            }
        }
        }
#pragma unroll
        for (int j = 0; j < HC; ++j) {
            extent(k[j]);
            add((U)(k[j] - bias));
        }
    }
    if (!REBASE) {
        if (__any_sync(0xffffffffu, dsc) && lane == 0) atomicOr(&a.order[ORD_DESCENT], 1u);
        if (__any_sync(0xffffffffu, asc) && lane == 0) atomicOr(&a.order[ORD_ASCENT], 1u);
        if (__any_sync(0xffffffffu, eq) && lane == 0) atomicOr(&a.order[ORD_EQUAL], 1u);
        unsigned long long nm = notmin, mx = maxk;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y0 = __shfl_xor_sync(0xffffffffu, nm, o);
            const unsigned long long y1 = __shfl_xor_sync(0xffffffffu, mx, o);
            nm = y0 > nm ? y0 : nm;
            mx = y1 > mx ? y1 : mx;
        }
        if (lane == 0) {
            atomicMax(&a.range[RNG_NOTMIN], nm);
            atomicMax(&a.range[RNG_MAX], mx);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.range[RNG_FLAGS], (unsigned long long)RNG_RECORDED);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NP * BINS; i += blockDim.x) {
        uint32_t sum = 0;
        for (int c = 0; c < COLS; ++c) sum += s_h[i * COLS + ((c + i) & (COLS - 1))];
        if (sum) atomicAdd(&cnt_out[i], (unsigned long long)sum);
    }
}

// ---------------------------------------------------------------------------
// K2: exclusive prefix sum of each pass's digit counts, trivial-pass test and
// the buffer chain.  One CTA of 1024 threads.
// ---------------------------------------------------------------------------
// Adaptive ranking (rank mode 4): a pass ranks with match.any when its digit
// is concentrated, else with shared match masks.  Concentration is the sum
// over digits of (count / n)^2: when it is high, most lanes of a warp share a
// few digits, which serialises the match masks' shared atomics.  A later pass
// sees keys already grouped by the lower digits, so equal digits sit together
// and the threshold is low (default 1/32, a.conc_later); the first pass to run
// sees the input order, where match.any only pays once one digit holds most
// keys (default 1/4, a.conc_first).  Both thresholds are tunable.

static __global__ void __launch_bounds__(1024) radix_scan_plan(RadixArgs a, int inplace) {
    __shared__ unsigned long long s_scr[33];
    __shared__ int s_trivial[64];
    __shared__ int s_conc[64];
    __shared__ double s_sq[32];
    const int bins = 1 << a.d;
    const int per = (bins + 1023) / 1024;   // consecutive bins per thread (<= 2)
    // a rebased sort (K1b ran) plans from the digit counts of key - min
    if (a.range && (a.range[RNG_FLAGS] & RNG_REBASED)) {
        for (int i = threadIdx.x; i < (a.npass << a.d); i += blockDim.x) a.counts[i] = a.counts2[i];
        __syncthreads();
    }
    for (int p = 0; p < a.npass; ++p) {
        unsigned long long* c = a.counts + (size_t)p * bins;
        unsigned long long local[2] = {0, 0};
        unsigned long long sum = 0;
        int triv = 0;
        double sq = 0.0;
        for (int j = 0; j < per; ++j) {
            const int b = threadIdx.x * per + j;
            local[j] = b < bins ? c[b] : 0ull;
            if (local[j] == (unsigned long long)a.n) triv = 1;
            sum += local[j];
            sq += (double)local[j] * (double)local[j];
        }
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if ((threadIdx.x & 31) == 0) s_sq[threadIdx.x >> 5] = sq;
        const int any_triv = __syncthreads_or(triv);
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < 32; ++w) t += s_sq[w];
            const double nn = (double)a.n * (double)a.n;
            s_conc[p] = (t > a.conc_later * nn ? 1 : 0) | (t > a.conc_first * nn ? 2 : 0);
        }
        unsigned long long tot;
        unsigned long long ex = block_exclusive_scan<1024>(sum, s_scr, &tot);
        for (int j = 0; j < per; ++j) {
            const int b = threadIdx.x * per + j;
            if (b < bins) c[b] = ex;
            ex += local[j];
        }
        if (threadIdx.x == 0) s_trivial[p] = any_triv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int active[64];
        int e = 0;
        // already in order: no pass runs, the input is copied (or, in place,
        // left as it is); in exactly reverse order (for key/value sorts with
        // no two equal keys, so the result stays stable): a reversed copy
        const bool in_order = a.order[ORD_DESCENT] == 0;
        const bool reversed = !in_order && a.order[ORD_ASCENT] == 0 && (!a.vout || a.order[ORD_EQUAL] == 0);
        if (in_order || reversed) {
            for (int p = 0; p <= a.npass; ++p) {
                PassDesc z = {};
                a.desc[p] = z;
            }
            a.desc[a.npass].fixup = reversed ? FIX_REVERSE : (inplace ? FIX_NONE : FIX_IN_TO_OUT);
            return;
        }
        for (int p = 0; p < a.npass; ++p)
            if (!s_trivial[p]) active[e++] = p;
        for (int p = 0; p <= a.npass; ++p) {
            PassDesc z = {};
            a.desc[p] = z;
        }
        for (int k = 0; k < e; ++k) {
            PassDesc pd = {};
            pd.active = 1;
            if (inplace) {
                pd.src = k == 0 ? BUF_OUT : ((k - 1) % 2 == 0 ? BUF_TMP : BUF_OUT);
                pd.dst = (k % 2 == 0) ? BUF_TMP : BUF_OUT;
            } else {
                pd.dst = ((e - 1 - k) % 2 == 0) ? BUF_OUT : BUF_TMP;
                pd.src = k == 0 ? BUF_IN : (((e - k) % 2 == 0) ? BUF_OUT : BUF_TMP);
            }
            pd.xin = (k == 0);
            pd.xout = (k == e - 1);
            pd.rank = (s_conc[active[k]] & (k > 0 ? 1 : 2)) ? 1 : 3;
            a.desc[active[k]] = pd;
        }
        int fix = FIX_NONE;
        if (e == 0 && !inplace) fix = FIX_IN_TO_OUT;
        if (inplace && (e % 2 == 1)) fix = FIX_TMP_TO_OUT;
        a.desc[a.npass].fixup = fix;
    }
}

// ---------------------------------------------------------------------------
// K3: one onesweep pass.  RANK selects how a warp finds the lanes that share
// a digit: 1 = match.any, 2 = one ballot per digit bit, 3 = shared-memory
// match masks built with atomicOr (fewest instructions; serialises when many
// lanes share a digit, as in sorted or low-entropy input).  Under adaptive
// ranking both the RANK 1 and RANK 3 kernels are launched for every pass and
// the one the pass descriptor does not name returns at once.
//
// Persistent CTAs take tiles in order from an atomic counter, so every tile's
// predecessors are held by running CTAs and the look-back always progresses.
// A CTA claims its next tile once the current one's aggregates are published
// and has the TMA engine copy it (keys, and values for pairs) into the other
// half of a double input buffer; a third buffer receives the reordered tile.
// ---------------------------------------------------------------------------
template <int RANK, int D>
__device__ __forceinline__ uint32_t warp_peers(uint32_t dig) {
    if (RANK == 1) {
        return __match_any_sync(0xffffffffu, dig);
    } else {
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int bit = 0; bit < D; ++bit) {
            const bool set = (dig >> bit) & 1u;
            const uint32_t b = __ballot_sync(0xffffffffu, set);
            peers &= set ? b : ~b;
        }
        return peers;
    }
}

// Dynamic shared memory of one onesweep CTA: three tile buffers (two TMA
// input buffers, one reorder buffer), per-virtual-warp digit counters, the
// tile's digit offsets, counts, partial sums and global bases (64- and 32-bit),
// two mbarriers.  (Rank mode 3 keeps its
// per-warp match masks in the reorder buffer.)
// Largest dynamic shared memory a CTA may use on sm_100-class GPUs (227 KB),
// less room for the kernel's static shared variables.
constexpr size_t kMaxDynSmem = 232448 - 1024;

// Each warp ranks its keys as vw independent "virtual warps" (vw = 2: the
// first and second half of its keys, interleaved for instruction-level
// parallelism), each with its own digit counters.
__host__ __device__ constexpr size_t onesweep_smem_vw(int block, int kpt, int w, bool pairs, int d, int vw) {
    return 3 * (size_t)block * kpt * (w + (pairs ? 4 : 0)) + (size_t)(block / 32) * vw * ((size_t)1 << d) * 2 +
           ((size_t)1 << d) * 20 + ((2 << d) <= block ? ((size_t)1 << d) * 16 : 0) + 16;
}
// two virtual warps per warp where their counters fit, else one
// (Rank mode 3, and 4 which launches it, also needs the match masks of the
// virtual warps, one 32-bit word per digit each, to fit in the reorder buffer.)
__host__ __device__ constexpr int onesweep_vw(int block, int kpt, int w, bool pairs, int d, int rank = 0) {
    return (kpt % 2 == 0 && onesweep_smem_vw(block, kpt, w, pairs, d, 2) <= kMaxDynSmem &&
            ((rank != 3 && rank != 4) ||
             (size_t)(block / 32) * 2 * ((size_t)1 << d) * 4 <= (size_t)block * kpt * w))
               ? 2
               : 1;
}
__host__ __device__ constexpr size_t onesweep_smem_bytes(int block, int kpt, int w, bool pairs, int d, int rank) {
    return onesweep_smem_vw(block, kpt, w, pairs, d, onesweep_vw(block, kpt, w, pairs, d, rank));
}

// Decoupled look-back for one digit: sums the counts of the preceding tiles
// back to the nearest inclusive prefix.  LBW slots are read per L2 round trip.
template <typename S, int LBW>
__device__ __forceinline__ uint64_t lookback_digit(const S* slot0, size_t stride, long long tile,
                                                   uint32_t* status, uint32_t limit) {
    constexpr int FB = sizeof(S) * 8 - 2;   // flag bits: 01 aggregate, 10 inclusive prefix
    const S cmask = ((S)1 << FB) - 1;
    uint64_t excl = 0;
    long long t = tile - 1;
    uint32_t polls = 0;
    while (t >= 0) {
        S v[LBW];
#pragma unroll
        for (int k = 0; k < LBW; ++k)
            v[k] = (t - k >= 0) ? ld_relaxed(slot0 + (size_t)(t - k) * stride) : ((S)2 << FB);
        int adv = 0;
        bool fin = false, blocked = false;
#pragma unroll
        for (int k = 0; k < LBW; ++k) {
            if (!fin && !blocked) {
                const uint32_t f = (uint32_t)(v[k] >> FB);
                if (f == 0) {
                    blocked = true;
                } else {
                    excl += (uint64_t)(v[k] & cmask);
                    ++adv;
                    if (f == 2) fin = true;
                }
            }
        }
        if (fin) break;
        t -= adv;
        if (blocked) {
            if (++polls > limit) {
                atomicOr(status, ST_TIMEOUT);
                break;
            }
            if ((polls & 255u) == 0 && ld_relaxed(status) != 0) break;
            __nanosleep(32);
        }
    }
    return excl;
}

// CTAs per SM the register budget is tuned for: about 40 registers plus one
// per key of the thread.
constexpr int onesweep_min_blocks(int block, int kpt) {
    return 65536 / (block * (kpt + 40)) < 1 ? 1 : (65536 / (block * (kpt + 40)) > 4 ? 4 : 65536 / (block * (kpt + 40)));
}

template <typename U, bool PAIRS, int BLOCK, int KPT, int D, int RANK>
__global__ void __launch_bounds__(BLOCK, onesweep_min_blocks(BLOCK, KPT)) radix_onesweep(RadixArgs a, int pass) {
    constexpr int WARPS = BLOCK / 32;
    constexpr int TILE = BLOCK * KPT;
    constexpr int PER_MAX = ((1 << D) + BLOCK - 1) / BLOCK;
    constexpr size_t KB = (size_t)TILE * sizeof(U);
    constexpr size_t VB = PAIRS ? (size_t)TILE * 4 : 0;
    const PassDesc desc = a.desc[pass];
    if (!desc.active || (a.adapt && desc.rank != RANK)) return;

    constexpr int bins = 1 << D;
    const int shift = pass * D;
    constexpr uint32_t mask = (uint32_t)(bins - 1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const KeyMap map = a.map;
    const U bias = pass_bias<U>(a);   // smallest mapped key when rebased, else 0

    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* bufs = smem;   // two input tile buffers of KB + VB bytes
    U* s_rkeys = (U*)(smem + 2 * (KB + VB));                  // reorder buffer
    uint32_t* s_rvals = (uint32_t*)(smem + 2 * (KB + VB) + KB);
    constexpr int kVW = onesweep_vw(BLOCK, KPT, (int)sizeof(U), PAIRS, D, RANK);
    constexpr int NVW = WARPS * kVW;   // virtual warps, in input order
    uint16_t* s_whist = (uint16_t*)(smem + 3 * (KB + VB));
    uint32_t* s_excl = (uint32_t*)(s_whist + NVW * bins);
    uint32_t* s_tcnt = s_excl + bins;
    uint32_t* s_part = s_tcnt + bins;   // 4 x bins partial sums (only when 2 * bins <= BLOCK)
    unsigned long long* s_gbase = (unsigned long long*)(s_part + (2 * bins <= BLOCK ? 4 * bins : 0));
    uint32_t* s_gbase32 = (uint32_t*)(s_gbase + bins);   // low words, used when n < 2^32
    const bool small_n = a.n < (1ull << 32);
    uint64_t* s_bar = (uint64_t*)(s_gbase32 + bins);
    // RANK 3 match masks (NVW x bins words) live in the reorder buffer,
    // which is idle while a tile is ranked
    uint32_t* s_match = (uint32_t*)s_rkeys;
    __shared__ uint32_t s_tile[2];
    __shared__ uint32_t s_scr[WARPS + 1];
    __shared__ uint32_t s_bad;   // this tile's offsets left the array

    const size_t n = a.n;
    const U* src = sel_src<U>(a, desc.src);
    U* dst = sel_dst<U>(a, desc.dst);
    const uint32_t* vsrc = PAIRS ? sel_vsrc(a, desc.src) : nullptr;
    uint32_t* vdst = PAIRS ? sel_vdst(a, desc.dst) : nullptr;
    const bool use_tma = (((uintptr_t)src & 15) == 0) && (!PAIRS || (((uintptr_t)vsrc & 15) == 0));
    const size_t full_tiles = n / TILE;

    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_mbar_init();
        const uint32_t t0 = atomicAdd(a.tile_counter + pass, 1u);
        s_tile[0] = t0;
        if (use_tma && t0 < full_tiles) {
            mbar_arrive_expect_tx(&s_bar[0], (uint32_t)(KB + VB));
            bulk_load(bufs, src + (size_t)t0 * TILE, (uint32_t)KB, &s_bar[0]);
            if (PAIRS) bulk_load(bufs + KB, vsrc + (size_t)t0 * TILE, (uint32_t)VB, &s_bar[0]);
        }
    }
    __syncthreads();

    uint32_t ph0 = 0, ph1 = 0;   // mbarrier phase of each buffer
    const uint32_t FA32 = 1u << 30, FP32 = 2u << 30;
    const uint64_t FA64 = 1ull << 62, FP64 = 2ull << 62;

    for (int it = 0;; ++it) {
        const int cur = it & 1;
        const uint32_t tile = s_tile[cur];
        if (tile >= a.ntiles) break;
        const size_t base = (size_t)tile * TILE;
        const bool full = tile < full_tiles;
        if (tid == 0) s_bad = 0;
        unsigned char* kb = bufs + cur * (KB + VB);
        U* s_keys = (U*)kb;
        uint32_t* s_vals = (uint32_t*)(kb + KB);
        uint16_t* wh = s_whist + warp * kVW * bins;   // kVW rows, one per virtual warp
        uint32_t* wm = s_match + warp * kVW * bins;
        for (int i = lane; i < kVW * bins / 2; i += 32) ((uint32_t*)wh)[i] = 0;
        if (RANK == 3)
            for (int i = lane; i < kVW * bins; i += 32) wm[i] = 0u;

        // ---- keys of the tile, warp-striped (warp w owns a contiguous run of
        // 32*KPT keys; key i of a lane sits at w*32*KPT + 32*i + lane).  The
        // keys stay in the tile buffer until the reorder; registers keep only
        // (rank << 16 | digit) per key.
        uint32_t dr[KPT];
        const int wofs = warp * 32 * KPT + lane;
        if (use_tma && full) {
            const uint32_t ph = cur ? ph1 : ph0;
            mbar_wait_bounded(&s_bar[cur], ph, a.status);
            if (cur) ph1 ^= 1u; else ph0 ^= 1u;
#pragma unroll
            for (int i = 0; i < KPT; ++i) {
                U k = s_keys[wofs + 32 * i];
                if (desc.xin) k = rank_key(k, map, bias);
                dr[i] = digit_of(k, shift, mask);
            }
        } else {
#pragma unroll
            for (int i = 0; i < KPT; ++i) {
                const size_t idx = base + wofs + 32 * i;
                U k = ~(U)0;   // pad: ranks after every real key of the tile
                if (idx < n) {
                    const U raw = ld_stream(src + idx);
                    s_keys[wofs + 32 * i] = raw;
                    if (PAIRS) s_vals[wofs + 32 * i] = ld_stream(vsrc + idx);
                    k = desc.xin ? rank_key(raw, map, bias) : raw;
                }
                dr[i] = digit_of(k, shift, mask);
            }
        }
        __syncwarp();

        // ---- stable rank of each key among the equal digits of its virtual
        // warp: keys [0, KPT/2) of a lane belong to the warp's first virtual
        // warp, [KPT/2, KPT) to its second; the two chains are independent
        const uint32_t lt = lanemask_lt();
        constexpr int H = KPT / kVW;
        uint16_t* wh1 = wh + (kVW == 2 ? bins : 0);
        uint32_t* wm1 = wm + (kVW == 2 ? bins : 0);
        if (kVW == 1) {
#pragma unroll
            for (int i = 0; i < KPT; ++i) {
                const uint32_t d0 = dr[i];
                uint32_t p0;
                if (RANK == 3) {
                    atomicOr(&wm[d0], 1u << lane);
                    __syncwarp();
                    p0 = wm[d0];
                    __syncwarp();
                } else {
                    p0 = warp_peers<RANK, D>(d0);
                }
                const int l0 = 31 - __clz(p0);
                uint32_t o0 = 0;
                if (lane == l0) {
                    o0 = wh[d0];
                    wh[d0] = (uint16_t)(o0 + __popc(p0));
                    if (RANK == 3) wm[d0] = 0u;
                }
                o0 = __shfl_sync(0xffffffffu, o0, l0);
                dr[i] = d0 | ((o0 + __popc(p0 & lt)) << 16);
                __syncwarp();
            }
        }
#pragma unroll
        for (int i = 0; i < (kVW == 2 ? H : 0); ++i) {
            const uint32_t d0 = dr[i], d1 = dr[i + H];
            uint32_t p0, p1;
            if (RANK == 3) {
                // peers from shared match masks: every lane ORs its bit into
                // its digit's word and reads the word back
                atomicOr(&wm[d0], 1u << lane);
                atomicOr(&wm1[d1], 1u << lane);
                __syncwarp();
                p0 = wm[d0];
                p1 = wm1[d1];
                __syncwarp();
            } else {
                p0 = warp_peers<RANK, D>(d0);
                p1 = warp_peers<RANK, D>(d1);
            }
            const int l0 = 31 - __clz(p0), l1 = 31 - __clz(p1);
            uint32_t o0 = 0, o1 = 0;
            if (lane == l0) {
                o0 = wh[d0];
                wh[d0] = (uint16_t)(o0 + __popc(p0));
                if (RANK == 3) wm[d0] = 0u;
            }
            if (lane == l1) {
                o1 = wh1[d1];
                wh1[d1] = (uint16_t)(o1 + __popc(p1));
                if (RANK == 3) wm1[d1] = 0u;
            }
            o0 = __shfl_sync(0xffffffffu, o0, l0);
            o1 = __shfl_sync(0xffffffffu, o1, l1);
            dr[i] = d0 | ((o0 + __popc(p0 & lt)) << 16);
            dr[i + H] = d1 | ((o1 + __popc(p1 & lt)) << 16);
            __syncwarp();
        }
        __syncthreads();

        // ---- tile digit counts; virtual-warp counts -> exclusive prefix over
        // virtual warps (in input order); publish each digit's tile aggregate
        // (tile 0: its inclusive prefix)
        constexpr int per = PER_MAX;
        const int b0 = tid * per;
        uint32_t mysum = 0;
        constexpr int G = (BLOCK >= 2 * bins) ? ((BLOCK / bins) < 4 ? (BLOCK / bins) : 4) : 1;
        constexpr int VPG = NVW / G;   // virtual warps per group
        if (G > 1) {
            // thread (g, b) = tid (g-major, so a warp reads consecutive digits)
            const int g = tid / bins, b = tid % bins;
            if (g < G) {
                uint32_t sum = 0;
#pragma unroll 8
                for (int v = 0; v < VPG; ++v) sum += s_whist[(g * VPG + v) * bins + b];
                s_part[g * bins + b] = sum;
            }
            __syncthreads();
            if (tid < bins) {
                uint32_t t = 0;
#pragma unroll
                for (int q = 0; q < G; ++q) t += s_part[q * bins + tid];
                mysum = t;
                s_tcnt[tid] = t;
                const size_t slot = ((size_t)pass * a.ntiles + tile) * bins + tid;
                if (a.lb64)
                    st_relaxed((uint64_t*)a.lookback + slot, (tile == 0 ? FP64 : FA64) | t);
                else
                    st_relaxed((uint32_t*)a.lookback + slot, (tile == 0 ? FP32 : FA32) | t);
            }
        } else {
#pragma unroll
            for (int j = 0; j < PER_MAX; ++j) {
                const int b = b0 + j;
                if (j < per && b < bins) {
                    uint32_t t = 0;
#pragma unroll 8
                    for (int v = 0; v < NVW; ++v) t += s_whist[v * bins + b];
                    mysum += t;
                    s_tcnt[b] = t;
                    const size_t slot = ((size_t)pass * a.ntiles + tile) * bins + b;
                    if (a.lb64)
                        st_relaxed((uint64_t*)a.lookback + slot, (tile == 0 ? FP64 : FA64) | t);
                    else
                        st_relaxed((uint32_t*)a.lookback + slot, (tile == 0 ? FP32 : FA32) | t);
                }
            }
        }
        // Claim the next tile only now, once this tile's aggregates are out:
        // a claimed tile blocks the look-back of every later tile until its
        // holder ranks it, so claims are made as late as the prefetch allows.
        // The TMA engine copies it into the other input buffer meanwhile.
        if (tid == 0) {
            const uint32_t nx = atomicAdd(a.tile_counter + pass, 1u);
            s_tile[cur ^ 1] = nx;
            if (use_tma && nx < full_tiles) {
                unsigned char* nb = bufs + (cur ^ 1) * (KB + VB);
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&s_bar[cur ^ 1], (uint32_t)(KB + VB));
                bulk_load(nb, src + (size_t)nx * TILE, (uint32_t)KB, &s_bar[cur ^ 1]);
                if (PAIRS) bulk_load(nb + KB, vsrc + (size_t)nx * TILE, (uint32_t)VB, &s_bar[cur ^ 1]);
            }
        }
        {
            uint32_t ex = 0;
            constexpr bool kWarpScan = G > 1 && bins >= 32 && BLOCK >= 1024;
            if (kWarpScan) {
                // the tile counts are in s_tcnt: one warp scans them (each
                // lane a run of bins / 32 digits) instead of a block-wide scan
                // with its three barriers (faster with 32 warps; with 16 the
                // block-wide scan measured faster)
                __syncthreads();
                if (warp == 0) {
                    constexpr int PL = bins >= 32 ? bins / 32 : 1;
                    uint32_t c[PL];
                    uint32_t sum = 0;
#pragma unroll
                    for (int j = 0; j < PL; ++j) {
                        c[j] = s_tcnt[lane * PL + j];
                        sum += c[j];
                    }
                    uint32_t inc = sum;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += y;
                    }
                    uint32_t run = inc - sum;
#pragma unroll
                    for (int j = 0; j < PL; ++j) {
                        s_excl[lane * PL + j] = run;
                        run += c[j];
                    }
                }
            } else {
                uint32_t tot;
                ex = block_exclusive_scan<BLOCK>(mysum, s_scr, &tot);
            }
            if (G > 1) {
                if (!kWarpScan && tid < bins) s_excl[tid] = ex;
                __syncthreads();
                // prefixes biased by the digit's offset in the tile, so the
                // reorder needs one lookup per key
                const int g = tid / bins, b = tid % bins;
                if (g < G) {
                    uint32_t run = s_excl[b];
                    for (int q = 0; q < g; ++q) run += s_part[q * bins + b];
#pragma unroll 8
                    for (int v = 0; v < VPG; ++v) {
                        const int i = (g * VPG + v) * bins + b;
                        const uint32_t c = s_whist[i];
                        s_whist[i] = (uint16_t)run;
                        run += c;
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < PER_MAX; ++j) {
                    const int b = b0 + j;
                    if (j < per && b < bins) {
                        s_excl[b] = ex;
                        uint32_t run = ex;
                        ex += s_tcnt[b];
#pragma unroll 8
                        for (int v = 0; v < NVW; ++v) {
                            const uint32_t c = s_whist[v * bins + b];
                            s_whist[v * bins + b] = (uint16_t)run;
                            run += c;
                        }
                    }
                }
            }
        }
        __syncthreads();   // s_excl and the warp prefixes are complete
        // ---- decoupled look-back for the owned digits.  No barrier follows:
        // threads without digits to resolve go straight on to the reorder,
        // which overlaps the look-back's L2 round trips.
        {
            const unsigned long long* boff = a.counts + (size_t)pass * bins;
#pragma unroll
            for (int j = 0; j < PER_MAX; ++j) {
                const int b = b0 + j;
                if (j < per && b < bins) {
                    uint64_t excl = 0;
                    const size_t slot0 = (size_t)pass * a.ntiles * bins + b;
                    if (tile > 0) {
                        if (a.lb64) {
                            excl = lookback_digit<uint64_t, 16>((const uint64_t*)a.lookback + slot0, bins,
                                                               tile, a.status, a.spin_limit);
                            st_relaxed((uint64_t*)a.lookback + slot0 + (size_t)tile * bins,
                                       FP64 | (excl + s_tcnt[b]));
                        } else {
                            excl = lookback_digit<uint32_t, 16>((const uint32_t*)a.lookback + slot0, bins,
                                                               tile, a.status, a.spin_limit);
                            st_relaxed((uint32_t*)a.lookback + slot0 + (size_t)tile * bins,
                                       FP32 | (uint32_t)(excl + s_tcnt[b]));
                        }
                    }
                    const unsigned long long gb = boff[b] + excl - s_excl[b];
                    s_gbase[b] = gb;
                    s_gbase32[b] = (uint32_t)gb;
                    // the digit's keys land in [boff + excl, boff + excl +
                    // count): past n only after an inconsistent look-back (a
                    // timed-out wait); the tile's stores are then skipped.
                    // (A partial tile's padding keys count under the digit of
                    // an all-ones key but are never stored.)
                    const uint32_t pad = (!full && b == (int)digit_of(~(U)0, shift, mask))
                                             ? (uint32_t)(TILE - (n - base)) : 0u;
                    if (boff[b] + excl + (s_tcnt[b] - pad) > n) {
                        s_bad = 1;
                        atomicOr(a.status, ST_RANGE);
                    }
                }
            }
        }

        // ---- reorder the tile by digit into the reorder buffer (stable)
        {
            const int valid_in = full ? TILE : (int)(n - base);
#pragma unroll
            for (int i = 0; i < KPT; ++i) {
                const int s = wofs + 32 * i;
                if (full || s < valid_in) {
                    U k = s_keys[s];
                    if (desc.xin) k = rank_key(k, map, bias);
                    const uint32_t dig = dr[i] & 0xFFFFu;
                    const uint32_t pos = ((kVW == 2 && i >= H) ? wh1 : wh)[dig] + (dr[i] >> 16);
                    s_rkeys[pos] = k;
                    if (PAIRS) s_rvals[pos] = s_vals[s];
                }
            }
        }
        __syncthreads();

        // ---- coalesced stable scatter to the global digit buckets
        const int valid = s_bad ? 0 : (full ? TILE : (int)(n - base));
#pragma unroll
        for (int i = 0; i < KPT; ++i) {
            const int s = i * BLOCK + tid;
            if ((full && valid) || s < valid) {
                const U k = s_rkeys[s];
                const uint32_t dig = digit_of(k, shift, mask);
                const size_t g = small_n ? (size_t)(uint32_t)(s_gbase32[dig] + (uint32_t)s)
                                         : (size_t)(s_gbase[dig] + (unsigned long long)s);
                st_stream(dst + g, desc.xout ? unrank_key(k, map, bias) : k);
                if (PAIRS) st_stream(vdst + g, s_rvals[s]);
            }
        }
        __syncthreads();   // the tile buffers are reused by later iterations
    }
}
// ---------------------------------------------------------------------------
// K3b: result copy when the pass chain did not end in the output buffer.
// ---------------------------------------------------------------------------
// Copies in 16-byte vectors where both sides are aligned; the reversed copy
// reads each vector's keys with coalesced scalar loads (descending addresses)
// and stores them as one vector.
template <typename T>
__device__ __forceinline__ void copy_forward(const T* s, T* o, size_t n, size_t t0, size_t stride) {
    constexpr int V = 16 / sizeof(T);
    if (((uintptr_t)s & 15) == 0 && ((uintptr_t)o & 15) == 0) {
        const size_t nv = n / V;
        for (size_t q = t0; q < nv; q += stride) __stcs((uint4*)o + q, __ldcs((const uint4*)s + q));
        for (size_t i = nv * V + t0; i < n; i += stride) o[i] = s[i];
    } else {
        for (size_t i = t0; i < n; i += stride) o[i] = s[i];
    }
}

template <typename T>
__device__ __forceinline__ void copy_reversed(const T* s, T* o, size_t n, size_t t0, size_t stride) {
    constexpr int V = 16 / sizeof(T);
    if (((uintptr_t)o & 15) == 0) {
        const size_t nv = n / V;
        for (size_t q = t0; q < nv; q += stride) {
            T v[V];
#pragma unroll
            for (int t = 0; t < V; ++t) v[t] = __ldcs(s + (n - 1 - (q * V + t)));
            uint4 u;
            memcpy(&u, v, 16);
            __stcs((uint4*)o + q, u);
        }
        for (size_t i = nv * V + t0; i < n; i += stride) o[i] = s[n - 1 - i];
    } else {
        for (size_t i = t0; i < n; i += stride) o[i] = s[n - 1 - i];
    }
}

template <typename U>
__global__ void __launch_bounds__(256) radix_fixup(RadixArgs a) {
    const int fix = a.desc[a.npass].fixup;
    if (fix == FIX_NONE) return;
    U* o = (U*)a.out;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n = a.n;
    if (fix == FIX_REVERSE) {
        const U* s = (const U*)a.in;
        if ((const void*)s == (const void*)o) {   // in place: swap mirror pairs
            for (size_t i = t0; i < n / 2; i += stride) {
                const U x = o[i];
                o[i] = o[n - 1 - i];
                o[n - 1 - i] = x;
                if (a.vout) {
                    const uint32_t v = a.vout[i];
                    a.vout[i] = a.vout[n - 1 - i];
                    a.vout[n - 1 - i] = v;
                }
            }
        } else {
            copy_reversed(s, o, n, t0, stride);
            if (a.vout) copy_reversed(a.vin, a.vout, n, t0, stride);
        }
        return;
    }
    const U* s = fix == FIX_IN_TO_OUT ? (const U*)a.in : (const U*)a.tmp;
    const uint32_t* vs = fix == FIX_IN_TO_OUT ? a.vin : a.vtmp;
    copy_forward(s, o, n, t0, stride);
    if (a.vout) copy_forward(vs, a.vout, n, t0, stride);
}

}  // namespace evosort

namespace evosort {
// The rank-3 match masks must fit in the reorder buffer.
constexpr bool match_masks_fit(int block, int kpt, int w, bool pairs, int d) {
    return (size_t)(block / 32) * onesweep_vw(block, kpt, w, pairs, d, 3) * ((size_t)1 << d) * 4 <=
           (size_t)block * kpt * w;
}
}  // namespace evosort
