// Register-tile onesweep pass (K3r): the stable scatter pass of Algorithms
// 4a/4b with the tile held in registers instead of a shared-memory copy.
//
// The pass computes exactly what radix_onesweep (radix.cuh) computes: the
// keys of each tile are ranked stably among equal digits, the tile's digit
// counts are published for the decoupled look-back, and the keys are
// reordered by digit in shared memory and written to their global digit
// buckets.  It spends shared-memory bandwidth and barriers differently,
// because on this GPU the pass is bound by shared-memory wavefronts, barrier
// stalls and look-back waits, not by DRAM:
//   - keys go from global memory straight into registers (warp-striped,
//     coalesced) and stay there until the reorder: no staging copy of the
//     tile and no second read of it (one shared-memory wavefront per 32 keys
//     fewer, and no re-applied key map);
//   - a warp ranks one column of 32 keys at a time: the lanes sharing a
//     digit come from shared-memory match masks (atomicOr, then a read) or,
//     for concentrated digits, from match.any; the running count of each digit
//     in the warp is a 32-bit shared counter that only the column's leader
//     lane for that digit updates, with one atomic add that also returns the
//     old count (one access where a read and a write were);
//   - after the ranking, threads 256..511 (scanners) sum each digit's count
//     over the warps and hand it to threads 0..255 (owners, one digit each)
//     through a named barrier; the owners publish the counts and walk the
//     look-back while the scanners scan the counts and turn the warp counters
//     into reorder offsets, then release the other warps to reorder through
//     another named barrier and the owners through a third, so the
//     look-back's L2 round trips overlap the scan and most of the reorder
//     (two CTA-wide barriers per tile);
//   - the next tile is claimed only after this tile's look-back is done (and
//     prefetched into L2 by one bulk prefetch): a claimed tile blocks the
//     look-back of every later tile until its counts are published, so the
//     shorter the time from claim to counts, the shorter every walk.
// Measured on 1e9 uniform int32 keys (8-bit digits, 1024 x 16 tiles): 3.94 ms
// per pass against 4.85 ms for the staged kernel at its best tile.
#pragma once

#include "radix.cuh"

namespace evosort {

// L2 prefetch of a global range by the TMA engine (no shared memory is
// written).  Address 16-byte aligned, size a multiple of 16 bytes.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Barrier over `nthreads` threads (whole warps) that use barrier `id`; id 0
// is the one __syncthreads uses.
__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Look-back slots read per L2 round trip: 8 keeps the owner threads' look-back
// window in registers next to their keys (16 spilled; measured slower).
constexpr int kRegLookback = 8;

// Shared memory of one register-tile CTA: reorder buffer (keys, then values),
// per-warp digit counters, match masks (rank mode 3), and per-digit tile
// offsets, tile counts and global bases.
__host__ __device__ constexpr size_t reg_smem_bytes(int block, int kpt, int w, bool pairs, int d, int rank) {
    return (size_t)block * kpt * (w + (pairs ? 4 : 0)) +                                 // reorder buffer
           (size_t)(block / 32) * ((size_t)1 << d) * 4 * (rank == 3 ? 2 : 1) +          // counters (+ masks)
           ((size_t)1 << d) * (4 + 4 + 8 + 4) + 64;                                      // excl, cnt, gbase, gbase32
}

// The register tile needs at least two threads per digit (digit owners and
// scanners are disjoint halves).
__host__ __device__ constexpr bool reg_shape_ok(int block, int d) { return block >= (2 << d); }

template <typename U, bool PAIRS, int BLOCK, int KPT, int D, int RANK>
__global__ void __launch_bounds__(BLOCK, (BLOCK >= 1024 ? 1 : 1024 / BLOCK))
    radix_onesweep_reg(RadixArgs a, int pass) {
    constexpr int WARPS = BLOCK / 32;
    constexpr int TILE = BLOCK * KPT;
    constexpr int bins = 1 << D;
    static_assert(reg_shape_ok(BLOCK, D), "register tile needs BLOCK >= 2 * bins");
    static_assert(RANK != 2, "ranking");
    const PassDesc desc = a.desc[pass];
    if (!desc.active || (a.adapt && desc.rank != RANK)) return;

    const int shift = pass * D;
    constexpr uint32_t mask = (uint32_t)(bins - 1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const KeyMap map = a.map;
    const U bias = pass_bias<U>(a);   // smallest mapped key when rebased, else 0

    extern __shared__ __align__(16) unsigned char smem[];
    U* s_r = (U*)smem;
    uint32_t* s_rv = (uint32_t*)(smem + (size_t)TILE * sizeof(U));
    uint32_t* s_wc = (uint32_t*)(smem + (size_t)TILE * (sizeof(U) + (PAIRS ? 4 : 0)));
    uint32_t* s_wm = s_wc + WARPS * bins;                                  // rank mode 3 only
    uint32_t* s_excl = s_wm + (RANK == 3 ? WARPS * bins : 0);              // tile offset of each digit
    uint32_t* s_cnt = s_excl + bins;                                       // tile count of each digit
    unsigned long long* s_gbase = (unsigned long long*)(s_cnt + bins);     // global start - tile offset
    uint32_t* s_gbase32 = (uint32_t*)(s_gbase + bins);
    __shared__ uint32_t s_tile[2];
    __shared__ uint32_t s_wtot[WARPS];
    __shared__ uint32_t s_bad;

    const size_t n = a.n;
    const U* src = sel_src<U>(a, desc.src);
    U* dst = sel_dst<U>(a, desc.dst);
    const uint32_t* vsrc = PAIRS ? sel_vsrc(a, desc.src) : nullptr;
    uint32_t* vdst = PAIRS ? sel_vdst(a, desc.dst) : nullptr;
    const bool can_prefetch = (((uintptr_t)src & 15) == 0) && (!PAIRS || (((uintptr_t)vsrc & 15) == 0));
    const size_t full_tiles = n / TILE;
    const bool small_n = n < (1ull << 32);
    const uint32_t FA32 = 1u << 30, FP32 = 2u << 30;
    const uint64_t FA64 = 1ull << 62, FP64 = 2ull << 62;
    const unsigned long long* boff = a.counts + (size_t)pass * bins;

    auto claim = [&](int slot) {
        const uint32_t t = atomicAdd(a.tile_counter + pass, 1u);
        s_tile[slot] = t;
        if (can_prefetch && t < full_tiles) {
            prefetch_l2(src + (size_t)t * TILE, (uint32_t)(TILE * sizeof(U)));
            if (PAIRS) prefetch_l2(vsrc + (size_t)t * TILE, (uint32_t)(TILE * 4));
        }
    };
    if (tid == 0) claim(0);
    // match masks start at zero; each column's leader clears the words it used
    if (RANK == 3)
        for (int i = tid; i < WARPS * bins; i += BLOCK) s_wm[i] = 0u;
    __syncthreads();

    for (int it = 0;; ++it) {
        const int cur = it & 1;
        const uint32_t tile = s_tile[cur];
        if (tile >= a.ntiles) break;
        const size_t base = (size_t)tile * TILE;
        const bool full = tile < full_tiles;
        const int valid = full ? TILE : (int)(n - base);

        // ---- keys of the tile into registers, warp-striped: warp w owns a
        // run of 32*KPT keys; key i of a lane sits at w*32*KPT + 32*i + lane
        U key[KPT];
        uint32_t val[PAIRS ? KPT : 1];
        uint32_t rk[(KPT + 1) / 2];   // rank in the warp, two 16-bit fields per register
        const int wofs = warp * 32 * KPT + lane;
        if (full) {
#pragma unroll
            for (int i = 0; i < KPT; ++i) key[i] = ld_stream(src + base + wofs + 32 * i);
            if (PAIRS) {
#pragma unroll
                for (int i = 0; i < KPT; ++i) val[PAIRS ? i : 0] = ld_stream(vsrc + base + wofs + 32 * i);
            }
        } else {
#pragma unroll
            for (int i = 0; i < KPT; ++i) {
                const int s = wofs + 32 * i;
                key[i] = s < valid ? ld_stream(src + base + s) : ~(U)0;   // pad: ranks after every real key
                if (PAIRS) val[PAIRS ? i : 0] = s < valid ? ld_stream(vsrc + base + s) : 0u;
            }
        }
        // this warp's counters start at zero; no other warp touches them
        // between this warp's scatter of the previous tile and B1
        uint32_t* wc = s_wc + warp * bins;
        uint32_t* wm = s_wm + warp * bins;
        for (int i = lane; i < bins / 4; i += 32) ((uint4*)wc)[i] = make_uint4(0u, 0u, 0u, 0u);
        if (desc.xin) {
#pragma unroll
            for (int i = 0; i < KPT; ++i)
                if (full || wofs + 32 * i < valid) key[i] = rank_key(key[i], map, bias);
        }
#pragma unroll
        for (int i = 0; i < (KPT + 1) / 2; ++i) rk[i] = 0u;
        __syncwarp();

        // ---- stable rank among equal digits of the warp: columns in input
        // order, lanes in order inside a column
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int i = 0; i < KPT; ++i) {
            const uint32_t d0 = digit_of(key[i], shift, mask);
            uint32_t p0;
            if (RANK == 1) {
                p0 = __match_any_sync(0xffffffffu, d0);
            } else {
                atomicOr(&wm[d0], 1u << lane);
                __syncwarp();
                p0 = wm[d0];
                __syncwarp();
            }
            const int l0 = 31 - __clz(p0);
            uint32_t o0 = 0;
            if (lane == l0) {
                o0 = atomicAdd(&wc[d0], (uint32_t)__popc(p0));
                if (RANK == 3) wm[d0] = 0u;
            }
            o0 = __shfl_sync(0xffffffffu, o0, l0);
            rk[i / 2] |= (o0 + __popc(p0 & lt)) << (16 * (i & 1));
            __syncwarp();
        }
        __syncthreads();   // B1: every warp's digit counts are final

        if (tid < bins) {
            // digit owners: publish the tile's count of digit b (summed over
            // the warps), walk the look-back to the digit's global start
            const int b = tid;
            if (tid == 0) s_bad = 0;   // set again only after barrier 4
            named_barrier(2, 2 * bins);   // the scanners' digit counts
            const uint32_t cnt = s_cnt[b];
            const size_t slot0 = (size_t)pass * a.ntiles * bins + b;
            const size_t slot = slot0 + (size_t)tile * bins;
            if (a.lb64)
                st_relaxed((uint64_t*)a.lookback + slot, (tile == 0 ? FP64 : FA64) | cnt);
            else
                st_relaxed((uint32_t*)a.lookback + slot, (tile == 0 ? FP32 : FA32) | cnt);
            uint64_t excl = 0;
            if (tile > 0) {
                if (a.lb64) {
                    excl = lookback_digit<uint64_t, kRegLookback>((const uint64_t*)a.lookback + slot0, bins, tile,
                                                                  a.status, a.spin_limit);
                    st_relaxed((uint64_t*)a.lookback + slot, FP64 | (excl + cnt));
                } else {
                    excl = lookback_digit<uint32_t, kRegLookback>((const uint32_t*)a.lookback + slot0, bins, tile,
                                                                  a.status, a.spin_limit);
                    st_relaxed((uint32_t*)a.lookback + slot, FP32 | (uint32_t)(excl + cnt));
                }
            }
            const unsigned long long glb = boff[b] + excl;
            // the digit's keys land in [glb, glb + count): past n only after an
            // inconsistent look-back (a timed-out wait); the tile's stores are
            // then skipped.  (A partial tile's padding keys count under the
            // digit of an all-ones key but are never stored.)
            const uint32_t pad = (!full && b == (int)digit_of(~(U)0, shift, mask)) ? (uint32_t)(TILE - valid) : 0u;
            // the owners' own reorder needs the scanners' offsets
            __syncwarp();   // the look-back diverged per lane: whole warps at the barrier
            named_barrier(4, 2 * bins);
            if (glb + (cnt - pad) > n) {
                s_bad = 1;
                atomicOr(a.status, ST_RANGE);
            }
            const unsigned long long gb = glb - s_excl[b];
            s_gbase[b] = gb;
            s_gbase32[b] = (uint32_t)gb;
            // claim the next tile now that this one's look-back is done, and
            // have the TMA engine pull it into L2 while this tile is reordered
            // and scattered
            if (tid == 0) claim(cur ^ 1);
        } else if (tid < 2 * bins) {
            // scanners: exclusive scan of the tile's digit counts, then the
            // warp counters become reorder offsets (digit offset in the tile
            // + count of the digit in earlier warps)
            const int b = tid - bins;
            uint32_t cnt = 0;
#pragma unroll 8
            for (int v = 0; v < WARPS; ++v) cnt += s_wc[v * bins + b];
            s_cnt[b] = cnt;
            asm volatile("bar.arrive 2, %0;" ::"n"(2 * bins) : "memory");
            uint32_t inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            constexpr int SW = bins / 32;   // scanner warps
            if (SW > 1) {
                if (lane == 31) s_wtot[b >> 5] = inc;
                named_barrier(1, bins);
                uint32_t before = 0;
                for (int q = 0; q < (b >> 5); ++q) before += s_wtot[q];
                inc += before;
            }
            uint32_t run = inc - cnt;
            s_excl[b] = run;
#pragma unroll 8
            for (int v = 0; v < WARPS; ++v) {
                const uint32_t c = s_wc[v * bins + b];
                s_wc[v * bins + b] = run;
                run += c;
            }
            // offsets ready: release the other warps (3) and the owners (4);
            // every scanner wrote a column of every warp's counters, so the
            // scanners wait for each other before their own reorder
            if (BLOCK > 2 * bins) asm volatile("bar.arrive 3, %0;" ::"n"(BLOCK - bins) : "memory");
            asm volatile("bar.arrive 4, %0;" ::"n"(2 * bins) : "memory");
            named_barrier(1, bins);
        } else {
            // the remaining warps reorder as soon as the offsets are ready,
            // while the owners are still walking the look-back
            asm volatile("bar.sync 3, %0;" ::"n"(BLOCK - bins) : "memory");
        }

        // ---- reorder the tile by digit into the reorder buffer (stable)
#pragma unroll
        for (int i = 0; i < KPT; ++i) {
            const uint32_t dig = digit_of(key[i], shift, mask);
            const uint32_t pos = wc[dig] + ((rk[i / 2] >> (16 * (i & 1))) & 0xFFFFu);
            if (full || wofs + 32 * i < valid) {
                s_r[pos] = key[i];
                if (PAIRS) s_rv[pos] = val[PAIRS ? i : 0];
            }
        }
        __syncthreads();   // B3: tile reordered, bases and next tile ready

        // ---- coalesced stable scatter to the global digit buckets
        const int nv = s_bad ? 0 : valid;
#pragma unroll
        for (int i = 0; i < KPT; ++i) {
            const int s = i * BLOCK + tid;
            if (s < nv) {
                const U k = s_r[s];
                const uint32_t dig = digit_of(k, shift, mask);
                const size_t g = small_n ? (size_t)(uint32_t)(s_gbase32[dig] + (uint32_t)s)
                                         : (size_t)(s_gbase[dig] + (unsigned long long)s);
                st_stream(dst + g, desc.xout ? unrank_key(k, map, bias) : k);
                if (PAIRS) st_stream(vdst + g, s_rv[s]);
            }
        }
        // no barrier: the next tile writes the reorder buffer, bases and
        // tile offsets only after its B1, which every thread reaches
        // after finishing this scatter
    }
}

template <typename U, bool PAIRS, int BLOCK, int KPT, int D, int RANK>
cudaError_t launch_reg_inst(size_t grid, int sms, cudaStream_t s, const RadixArgs& a, int pass) {
    auto kern = radix_onesweep_reg<U, PAIRS, BLOCK, KPT, D, RANK>;
    const size_t smem = reg_smem_bytes(BLOCK, KPT, (int)sizeof(U), PAIRS, D, RANK);
    static int resident = 0;   // resident CTAs per SM
    if (resident == 0) {
        cudaError_t e = cudaSuccess;
        if (smem > 48 * 1024)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BLOCK, smem);
        if (e != cudaSuccess) return e;
        resident = nb > 0 ? nb : 1;
    }
    // persistent grid: every SM full, never more CTAs than tiles
    size_t g = (size_t)sms * resident;
    if (g > grid) g = grid;
    if (g < 1) g = 1;
    kern<<<(unsigned)g, BLOCK, smem, s>>>(a, pass);
    return cudaGetLastError();
}

// Rank modes of the register tile: 1 (match.any) and 3 (match masks); rank
// mode 4 launches both per pass, as for the staged tile.
template <typename U, bool PAIRS, int B, int K>
cudaError_t launch_reg_rank(int rank, size_t grid, int sms, cudaStream_t s, const RadixArgs& a, int pass) {
    if (a.d != 8) return cudaErrorInvalidConfiguration;
    if (rank == 1) return launch_reg_inst<U, PAIRS, B, K, 8, 1>(grid, sms, s, a, pass);
    if (rank == 3) return launch_reg_inst<U, PAIRS, B, K, 8, 3>(grid, sms, s, a, pass);
    return cudaErrorInvalidConfiguration;
}

}  // namespace evosort
