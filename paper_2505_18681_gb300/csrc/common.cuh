// Shared device helpers for the sort kernels: key types, the order-preserving
// key transform, memory-model helpers and small block-wide scans.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace evosort {

// dtype codes, identical to evosort_dtype in include/evosort.h
enum : int { DT_I32 = 0, DT_I64 = 1, DT_U32 = 2, DT_U64 = 3, DT_F32 = 4, DT_F64 = 5 };

// device status word bits (evosort_sync maps them to evosort_status)
enum : uint32_t { ST_TIMEOUT = 1u, ST_BAD_OFFSETS = 2u, ST_RANGE = 4u };

// Bounded waits: polls before a kernel gives up, records ST_TIMEOUT and
// proceeds (its output is then invalid but the context lives).  Look-back
// waits take their limit from the launch (evosort_set_wait_limit, default
// this value); mbarrier waits for the kernel's own bulk copies always use it.
constexpr uint32_t kSpinLimit = 1u << 22;

inline int dtype_bytes(int dt) { return (dt == DT_I32 || dt == DT_U32 || dt == DT_F32) ? 4 : 8; }

// ---------------------------------------------------------------------------
// Order-preserving map of key bits onto unsigned integers (the sign flip of
// Algorithms 4a/4b; for floats the sign-magnitude flip, then a rotation by
// 2^m - 1 that moves both NaN blocks above +inf).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t to_ordered(uint32_t u, int dt) {
    if (dt == DT_I32) return u ^ 0x80000000u;
    if (dt == DT_F32) {
        uint32_t t = (u & 0x80000000u) ? ~u : (u ^ 0x80000000u);
        return t - 0x007FFFFFu;
    }
    return u;
}
__device__ __forceinline__ uint64_t to_ordered(uint64_t u, int dt) {
    if (dt == DT_I64) return u ^ 0x8000000000000000ull;
    if (dt == DT_F64) {
        uint64_t t = (u >> 63) ? ~u : (u ^ 0x8000000000000000ull);
        return t - 0x000FFFFFFFFFFFFFull;
    }
    return u;
}
__device__ __forceinline__ uint32_t from_ordered(uint32_t t, int dt) {
    if (dt == DT_I32) return t ^ 0x80000000u;
    if (dt == DT_F32) {
        uint32_t x = t + 0x007FFFFFu;
        return (x & 0x80000000u) ? (x ^ 0x80000000u) : ~x;
    }
    return t;
}
__device__ __forceinline__ uint64_t from_ordered(uint64_t t, int dt) {
    if (dt == DT_I64) return t ^ 0x8000000000000000ull;
    if (dt == DT_F64) {
        uint64_t x = t + 0x000FFFFFFFFFFFFFull;
        return (x >> 63) ? (x ^ 0x8000000000000000ull) : ~x;
    }
    return t;
}

// The same maps without branches, for kernels that apply them per key:
//   forward  t = ((x ^ ((sar(x) & F) | S)) - R) ^ X
//   inverse  x = u ^ ((~sar(u) & F) | S),  u = (t ^ X) + R
// with (F, S, R) = (0, 0, 0) unsigned, (0, signbit, 0) signed and
// (all-ones, signbit, 2^m - 1) float; sar is the arithmetic shift by w-1.
// X is 0 for an ascending sort and all ones for a descending one (the
// complement reverses the order, and equal keys stay equal, so a stable
// ascending sort of the complemented keys is the stable descending sort).
struct KeyMap {
    unsigned long long f, s, r, x;
};
inline KeyMap key_map_for(int dt, bool descending = false) {
    KeyMap m{0, 0, 0, 0};
    if (dt == DT_I32) m.s = 0x80000000ull;
    if (dt == DT_I64) m.s = 0x8000000000000000ull;
    if (dt == DT_F32) m = {0xFFFFFFFFull, 0x80000000ull, 0x007FFFFFull, 0};
    if (dt == DT_F64) m = {~0ull, 0x8000000000000000ull, 0x000FFFFFFFFFFFFFull, 0};
    if (descending) m.x = dtype_bytes(dt) == 4 ? 0xFFFFFFFFull : ~0ull;
    return m;
}
__device__ __forceinline__ uint32_t map_fwd(uint32_t x, const KeyMap& m) {
    const uint32_t sar = (uint32_t)((int32_t)x >> 31);
    return ((x ^ ((sar & (uint32_t)m.f) | (uint32_t)m.s)) - (uint32_t)m.r) ^ (uint32_t)m.x;
}
__device__ __forceinline__ uint64_t map_fwd(uint64_t x, const KeyMap& m) {
    const uint64_t sar = (uint64_t)((int64_t)x >> 63);
    return ((x ^ ((sar & m.f) | m.s)) - m.r) ^ m.x;
}
__device__ __forceinline__ uint32_t map_inv(uint32_t t, const KeyMap& m) {
    const uint32_t u = (t ^ (uint32_t)m.x) + (uint32_t)m.r;
    const uint32_t sar = (uint32_t)((int32_t)u >> 31);
    return u ^ ((~sar & (uint32_t)m.f) | (uint32_t)m.s);
}
__device__ __forceinline__ uint64_t map_inv(uint64_t t, const KeyMap& m) {
    const uint64_t u = (t ^ m.x) + m.r;
    const uint64_t sar = (uint64_t)((int64_t)u >> 63);
    return u ^ ((~sar & m.f) | m.s);
}

// ---------------------------------------------------------------------------
// Relaxed GPU-scope loads/stores for the decoupled look-back slots.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Streaming loads/stores: data touched once per pass, kept out of L1.
template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) { return __ldcs(p); }
template <typename T>
__device__ __forceinline__ void st_stream(T* p, T v) { __stcs(p, v); }

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA engine, non-tensor form) with mbarrier
// completion.  Global source and shared destination must be 16-byte aligned
// and the size a multiple of 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of an mbarrier; records ST_TIMEOUT on
// expiry.  Returns false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t* status) {
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
    }
    atomicOr(status, ST_TIMEOUT);
    return false;
}

// Digit `shift .. shift+d` of a key, with 64-bit keys split into words so the
// shift is one funnel shift.
__device__ __forceinline__ uint32_t digit_of(uint32_t k, int shift, uint32_t mask) {
    return (k >> shift) & mask;
}
__device__ __forceinline__ uint32_t digit_of(uint64_t k, int shift, uint32_t mask) {
    const uint32_t lo = (uint32_t)k, hi = (uint32_t)(k >> 32);
    const uint32_t v = shift >= 32 ? (hi >> (shift - 32)) : __funnelshift_r(lo, hi, shift);
    return v & mask;
}

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of one value per thread (any integer type).
// scratch: at least BLOCK/32 elements of shared memory.  Returns the
// exclusive prefix; *total receives the block sum.
// ---------------------------------------------------------------------------
template <int BLOCK, typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* scratch, T* total) {
    constexpr int WARPS = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < WARPS ? scratch[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < WARPS) scratch[lane] = wi - w;   // exclusive warp offsets
        if (lane == WARPS - 1) scratch[WARPS] = wi; // block total
    }
    __syncthreads();
    T r = scratch[warp] + inc - v;
    *total = scratch[WARPS];
    __syncthreads();
    return r;
}

}  // namespace evosort
