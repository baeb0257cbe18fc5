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
enum : int { FIX_NONE = 0, FIX_IN_TO_OUT = 1, FIX_TMP_TO_OUT = 2 };

struct PassDesc {
    int active;   // 0: the digit is constant over all keys, pass skipped
    int src, dst; // buffer selectors
    int xin;      // apply to_ordered on load (first active pass)
    int xout;     // apply from_ordered on store (last active pass)
    int fixup;    // used in the entry after the last pass
    int pad0, pad1;
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
    int d;           // digit bits
    int npass;       // ceil(8w / d)
    int lb64;        // look-back slots are 64-bit (n >= 2^30)
    size_t ntiles;   // tiles per pass
    PassDesc* desc;             // npass + 1 entries
    unsigned long long* counts; // npass << d digit counts, then exclusive offsets
    void* lookback;             // npass * ntiles << d slots
    uint32_t* tile_counter;     // npass counters
    uint32_t* status;
};

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
// Shared counters per CTA (npass << d of them); consecutive equal digits of a
// thread's keys are merged before the shared atomic, which keeps sorted and
// low-entropy inputs from serialising on one counter.
// ---------------------------------------------------------------------------
template <typename U>
__global__ void __launch_bounds__(512) radix_histogram(RadixArgs a) {
    extern __shared__ uint32_t s_h[];
    const int bins = 1 << a.d;
    const int total = a.npass * bins;
    const U mask = (U)(bins - 1);
    for (int i = threadIdx.x; i < total; i += blockDim.x) s_h[i] = 0;
    __syncthreads();

    constexpr int V = 16 / sizeof(U);   // keys per 128-bit load
    const U* keys = (const U*)a.in;
    const size_t n = a.n;
    // 16-byte aligned body; the head and tail are read with scalar loads
    size_t head = ((16 - ((uintptr_t)keys & 15)) & 15) / sizeof(U);
    if (head > n) head = n;
    const size_t nvec = (n - head) / V;
    const size_t tail0 = head + nvec * V;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t gthreads = (size_t)gridDim.x * blockDim.x;

    auto count_key = [&](U k) {
        k = to_ordered(k, a.dt);
        for (int p = 0; p < a.npass; ++p) {
            const uint32_t dig = (uint32_t)((k >> (p * a.d)) & mask);
            atomicAdd(&s_h[p * bins + dig], 1u);
        }
    };
    if (gtid < head) count_key(keys[gtid]);
    if (gtid < n - tail0) count_key(keys[tail0 + gtid]);

    using Vec = uint4;
    const Vec* vp = (const Vec*)(keys + head);
    for (size_t i = gtid; i < nvec; i += gthreads) {
        Vec v = __ldcs(vp + i);
        U k[V];
        memcpy(k, &v, 16);
#pragma unroll
        for (int j = 0; j < V; ++j) k[j] = to_ordered(k[j], a.dt);
        for (int p = 0; p < a.npass; ++p) {
            const int sh = p * a.d;
            uint32_t prev = (uint32_t)((k[0] >> sh) & mask);
            uint32_t run = 1;
#pragma unroll
            for (int j = 1; j < V; ++j) {
                const uint32_t dig = (uint32_t)((k[j] >> sh) & mask);
                if (dig == prev) {
                    ++run;
                } else {
                    atomicAdd(&s_h[p * bins + prev], run);
                    prev = dig;
                    run = 1;
                }
            }
            atomicAdd(&s_h[p * bins + prev], run);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < total; i += blockDim.x)
        if (s_h[i]) atomicAdd(&a.counts[i], (unsigned long long)s_h[i]);
}

// ---------------------------------------------------------------------------
// K2: exclusive prefix sum of each pass's digit counts, trivial-pass test and
// the buffer chain.  One CTA of 1024 threads.
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(1024) radix_scan_plan(RadixArgs a, int inplace) {
    __shared__ unsigned long long s_scr[33];
    __shared__ int s_trivial[64];
    const int bins = 1 << a.d;
    const int per = (bins + 1023) / 1024;   // consecutive bins per thread (<= 2)
    for (int p = 0; p < a.npass; ++p) {
        unsigned long long* c = a.counts + (size_t)p * bins;
        unsigned long long local[2] = {0, 0};
        unsigned long long sum = 0;
        int triv = 0;
        for (int j = 0; j < per; ++j) {
            const int b = threadIdx.x * per + j;
            local[j] = b < bins ? c[b] : 0ull;
            if (local[j] == (unsigned long long)a.n) triv = 1;
            sum += local[j];
        }
        const int any_triv = __syncthreads_or(triv);
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
// a digit: 1 = match.any, 2 = one ballot per digit bit.
// ---------------------------------------------------------------------------
template <int RANK>
__device__ __forceinline__ uint32_t warp_peers(uint32_t dig, int d) {
    if (RANK == 1) {
        return __match_any_sync(0xffffffffu, dig);
    } else {
        uint32_t peers = 0xffffffffu;
        for (int bit = 0; bit < d; ++bit) {
            const uint32_t b = __ballot_sync(0xffffffffu, (dig >> bit) & 1u);
            peers &= ((dig >> bit) & 1u) ? b : ~b;
        }
        return peers;
    }
}

template <int BLOCK, int KPT, int MAXB, bool PAIRS, typename U>
constexpr size_t onesweep_smem_bytes(int d) {
    return (size_t)BLOCK * KPT * sizeof(U) + (PAIRS ? (size_t)BLOCK * KPT * 4 : 0) +
           (size_t)(BLOCK / 32) * (1u << d) * 2 + (size_t)(1u << d) * 4 + (size_t)(1u << d) * 8;
}

template <typename U, bool PAIRS, int BLOCK, int KPT, int MAXB, int RANK>
__global__ void __launch_bounds__(BLOCK) radix_onesweep(RadixArgs a, int pass) {
    constexpr int WARPS = BLOCK / 32;
    constexpr int TILE = BLOCK * KPT;
    constexpr int PER_MAX = ((1 << MAXB) + BLOCK - 1) / BLOCK;
    const PassDesc desc = a.desc[pass];
    if (!desc.active) return;

    const int d = a.d;
    const int bins = 1 << d;
    const int shift = pass * d;
    const U mask = (U)(bins - 1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    extern __shared__ __align__(16) unsigned char smem[];
    U* s_keys = (U*)smem;
    uint32_t* s_vals = (uint32_t*)(smem + (size_t)TILE * sizeof(U));
    uint16_t* s_whist = (uint16_t*)(smem + (size_t)TILE * sizeof(U) + (PAIRS ? (size_t)TILE * 4 : 0));
    uint32_t* s_excl = (uint32_t*)(s_whist + WARPS * bins);
    unsigned long long* s_gbase = (unsigned long long*)(s_excl + bins);
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_scr[WARPS + 1];

    const size_t n = a.n;
    const U* src = sel_src<U>(a, desc.src);
    U* dst = sel_dst<U>(a, desc.dst);

    // Persistent CTAs: tiles are taken in order from an atomic counter, so a
    // tile's predecessors are always held by running CTAs (forward progress
    // of the look-back does not depend on CTA scheduling order).
    for (;;) {
    if (tid == 0) s_tile = atomicAdd(a.tile_counter + pass, 1u);
    {
        uint32_t* z = (uint32_t*)s_whist;
        for (int i = tid; i < WARPS * bins / 2; i += BLOCK) z[i] = 0;
    }
    __syncthreads();
    const size_t tile = s_tile;
    if (tile >= a.ntiles) break;
    const size_t base = tile * TILE;

    // ---- load (warp-striped: each warp reads a contiguous run of 32*KPT keys)
    U key[KPT];
    uint32_t val[PAIRS ? KPT : 1];
    const size_t wbase = base + (size_t)warp * 32 * KPT + lane;
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
        const size_t idx = wbase + (size_t)i * 32;
        if (idx < n) {
            U k = ld_stream(src + idx);
            key[i] = desc.xin ? to_ordered(k, a.dt) : k;
        } else {
            key[i] = ~(U)0;   // pad: ranks after every real key of the tile
        }
    }
    if (PAIRS) {
        const uint32_t* vsrc = sel_vsrc(a, desc.src);
#pragma unroll
        for (int i = 0; i < KPT; ++i) {
            const size_t idx = wbase + (size_t)i * 32;
            val[i] = idx < n ? ld_stream(vsrc + idx) : 0u;
        }
    }

    // ---- stable rank of each key among equal digits of its warp
    uint16_t* wh = s_whist + warp * bins;
    uint32_t rank[KPT];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
        const uint32_t dig = (uint32_t)((key[i] >> shift) & mask);
        const uint32_t peers = warp_peers<RANK>(dig, d);
        const int leader = 31 - __clz(peers);
        uint32_t old = 0;
        if (lane == leader) {
            old = wh[dig];
            wh[dig] = (uint16_t)(old + __popc(peers));
        }
        old = __shfl_sync(0xffffffffu, old, leader);
        rank[i] = old + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();

    // ---- tile digit counts; warp counts -> exclusive prefix over warps
    const int per = (bins + BLOCK - 1) / BLOCK;
    const int b0 = tid * per;
    uint32_t cnt[PER_MAX];
    uint32_t mysum = 0;
#pragma unroll
    for (int j = 0; j < PER_MAX; ++j) {
        cnt[j] = 0;
        const int b = b0 + j;
        if (j < per && b < bins) {
            uint32_t s = 0;
#pragma unroll 4
            for (int w = 0; w < WARPS; ++w) {
                const uint32_t c = s_whist[w * bins + b];
                s_whist[w * bins + b] = (uint16_t)s;
                s += c;
            }
            cnt[j] = s;
            mysum += s;
        }
    }
    // publish this tile's aggregate (tile 0 publishes its inclusive prefix)
    const uint32_t FA32 = 1u << 30, FP32 = 2u << 30, M32 = FA32 - 1;
    const uint64_t FA64 = 1ull << 62, FP64 = 2ull << 62, M64 = FA64 - 1;
#pragma unroll
    for (int j = 0; j < PER_MAX; ++j) {
        const int b = b0 + j;
        if (j < per && b < bins) {
            const size_t slot = ((size_t)pass * a.ntiles + tile) * bins + b;
            if (a.lb64)
                st_relaxed((uint64_t*)a.lookback + slot, (tile == 0 ? FP64 : FA64) | cnt[j]);
            else
                st_relaxed((uint32_t*)a.lookback + slot, (tile == 0 ? FP32 : FA32) | cnt[j]);
        }
    }
    // exclusive scan of the tile counts over digits
    {
        uint32_t tot;
        uint32_t ex = block_exclusive_scan<BLOCK>(mysum, s_scr, &tot);
#pragma unroll
        for (int j = 0; j < PER_MAX; ++j) {
            const int b = b0 + j;
            if (j < per && b < bins) s_excl[b] = ex;
            ex += cnt[j];
        }
    }
    // ---- decoupled look-back over preceding tiles, all owned digits at once
    {
        uint64_t excl[PER_MAX];
        long long t[PER_MAX];
        bool done[PER_MAX];
        int left = 0;
#pragma unroll
        for (int j = 0; j < PER_MAX; ++j) {
            excl[j] = 0;
            t[j] = (long long)tile - 1;
            done[j] = !(j < per && b0 + j < bins) || tile == 0;
            left += done[j] ? 0 : 1;
        }
        uint32_t polls = 0;
        while (left > 0) {
#pragma unroll
            for (int j = 0; j < PER_MAX; ++j) {
                if (done[j]) continue;
                const size_t slot = ((size_t)pass * a.ntiles + (size_t)t[j]) * bins + b0 + j;
                uint64_t v, flag, c;
                if (a.lb64) {
                    v = ld_relaxed((const uint64_t*)a.lookback + slot);
                    flag = v >> 62;
                    c = v & M64;
                } else {
                    const uint32_t v32 = ld_relaxed((const uint32_t*)a.lookback + slot);
                    flag = v32 >> 30;
                    c = v32 & M32;
                }
                if (flag == 0) continue;
                excl[j] += c;
                if (flag == 2 || t[j] == 0) {
                    done[j] = true;
                    --left;
                } else {
                    --t[j];
                }
            }
            if (left > 0 && ++polls > kSpinLimit) {
                atomicOr(a.status, ST_TIMEOUT);
                break;
            }
            if (left > 0 && (polls & 1023u) == 0 && ld_relaxed(a.status) != 0) break;
        }
        const unsigned long long* boff = a.counts + (size_t)pass * bins;
#pragma unroll
        for (int j = 0; j < PER_MAX; ++j) {
            const int b = b0 + j;
            if (j < per && b < bins) {
                if (tile > 0) {
                    const size_t slot = ((size_t)pass * a.ntiles + tile) * bins + b;
                    if (a.lb64)
                        st_relaxed((uint64_t*)a.lookback + slot, FP64 | (excl[j] + cnt[j]));
                    else
                        st_relaxed((uint32_t*)a.lookback + slot, FP32 | (uint32_t)(excl[j] + cnt[j]));
                }
                s_gbase[b] = boff[b] + excl[j] - s_excl[b];
            }
        }
    }
    __syncthreads();

    // ---- reorder the tile by digit in shared memory (stable)
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
        const uint32_t dig = (uint32_t)((key[i] >> shift) & mask);
        const uint32_t pos = s_excl[dig] + wh[dig] + rank[i];
        s_keys[pos] = key[i];
        if (PAIRS) s_vals[pos] = val[i];
    }
    __syncthreads();

    // ---- coalesced stable scatter to the global digit buckets
    const size_t valid = (n - base) < (size_t)TILE ? (n - base) : (size_t)TILE;
    uint32_t* vdst = PAIRS ? sel_vdst(a, desc.dst) : nullptr;
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
        const int s = i * BLOCK + tid;
        if ((size_t)s < valid) {
            const U k = s_keys[s];
            const uint32_t dig = (uint32_t)((k >> shift) & mask);
            const size_t g = (size_t)(s_gbase[dig] + (unsigned long long)s);
            st_stream(dst + g, desc.xout ? from_ordered(k, a.dt) : k);
            if (PAIRS) st_stream(vdst + g, s_vals[s]);
        }
    }
    __syncthreads();   // shared tile buffers are reused by the next tile
    }
}

// ---------------------------------------------------------------------------
// K3b: result copy when the pass chain did not end in the output buffer.
// ---------------------------------------------------------------------------
template <typename U>
__global__ void __launch_bounds__(256) radix_fixup(RadixArgs a) {
    const int fix = a.desc[a.npass].fixup;
    if (fix == FIX_NONE) return;
    const U* s = fix == FIX_IN_TO_OUT ? (const U*)a.in : (const U*)a.tmp;
    const uint32_t* vs = fix == FIX_IN_TO_OUT ? a.vin : a.vtmp;
    U* o = (U*)a.out;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        o[i] = s[i];
        if (a.vout) a.vout[i] = vs[i];
    }
}

}  // namespace evosort
