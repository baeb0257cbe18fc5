// Genetic-algorithm autotuner (Algorithm 2 of the paper, RunGATuning) and the
// tuned-parameter table used by the dispatcher (Algorithm 5).
//
// The genome holds the knobs that act on the sort this library runs:
//   algo        radix or merge (the paper's A_code: 4 = radix, 3 = merge)
//   digit_bits  radix digit width d in [4, 11] (the paper fixes 8)
//   kern        radix pass kernel: staged tile or register tile
//   shape       radix CTA tile shape (threads x keys per thread)
//   rank        radix tile ranking variant
//   tins        mergesort insertion threshold T_insertion in [2, 2048],
//               first generation drawn from [2, 256] (Section 4.2 bounds)
//   alater, afirst  the adaptive ranking's two thresholds
//   small       the one-CTA small-array cut-over, the GPU form of the
//               paper's T_numpy (a library sort below a size, Algorithm 5)
//   sblock, swarp, sgiant  the segmented sort's tier cut-overs (tuned in the
//               segmented mode only)
// Fitness f(x) = device time of one sort of the sample with genome x (median
// of `reps` CUDA-event timings); a genome whose output is wrong or whose
// configuration is rejected gets +infinity.
// Operators (the paper names them but not their details; this library's
// reading): tournament selection of size 3, elitism of the best `elite`
// genomes, uniform crossover applied to a pair with probability 0.7 (each gene
// from either parent with probability 1/2), uniform mutation applied to an
// individual with probability 0.3 (each gene redrawn with probability 0.2),
// re-evaluation of changed genomes only (identical genomes share a cached
// fitness), SplitMix64 random numbers from a seed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "evosort.h"
#include "api_internal.h"
#include "common.cuh"

namespace evosort {
namespace {

struct Rng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double unit() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
    int range(int lo, int hi) { return lo + (int)(next() % (uint64_t)(hi - lo + 1)); }
};

// Staged-tile shapes; register-tile shapes come from the library's
// preference list for the key width (reg_shape_for).
const int kShapes[][2] = {{256, 16}, {512, 16}, {512, 32}, {1024, 8}, {1024, 16}, {512, 8}};
constexpr int kNShapes = 6;
const int kSmallCaps[] = {1, 1024, 2048, 4096, 8192};   // 1 = off
const int kBlockCaps[] = {256, 512, 1024, 2048, 4096, 8192};
const int kWarpCaps[] = {32, 64, 128, 256};
const long long kGiants[] = {-1, 1ll << 20, 1ll << 22, 1ll << 24, 1ll << 26};   // -1 = off

// Tuning modes: one array (the sort of a sample), or a segmented batch.
enum { MODE_ARRAY = 0, MODE_SEGMENTED = 1 };

struct Genome {
    int algo, d, kern, shape, rank, tins, alater, afirst, small, sblock, swarp, sgiant;
    auto key() const { return std::tie(algo, d, kern, shape, rank, tins, alater, afirst, small, sblock, swarp, sgiant); }
    bool operator<(const Genome& o) const { return key() < o.key(); }
    // genes that do not act in this mode, for this algorithm or at this size
    // are normalised away, so equivalent genomes share one fitness evaluation
    Genome canon(int mode, size_t n, int w) const {
        Genome g = *this;
        if (mode == MODE_SEGMENTED) {
            g.algo = g.d = g.kern = g.shape = g.rank = g.alater = g.afirst = g.small = 0;
            if (g.tins > 64) g.tins = 16;   // the block tier's base runs
            return g;
        }
        g.sblock = g.swarp = g.sgiant = 0;
        if ((size_t)kSmallCaps[g.small] >= n && g.small != 0) {   // the one-CTA path takes the whole sort
            g = Genome{};
            g.algo = this->algo;   // kept: an explicit algorithm plus a cut-over selects the path
            g.small = 4;           // every cap >= n behaves the same
            g.tins = std::min(this->tins, 32);
            return g;
        }
        g.small = 0;   // every cap < n is "off"
        if (g.algo == EVOSORT_ALGO_RADIX) {
            g.tins = 0;
            if (g.kern == 2) g.shape %= (w == 4 ? 2 : 3);   // register shapes: a shorter list
            if (g.rank != 4 || n < kAdaptMinKeys) g.alater = g.afirst = 0;
        } else {
            g.d = g.kern = g.shape = g.rank = g.alater = g.afirst = 0;
        }
        return g;
    }
};

Genome random_genome(Rng& r, int tins_hi) {
    Genome g;
    g.algo = r.unit() < 0.5 ? EVOSORT_ALGO_RADIX : EVOSORT_ALGO_MERGE;
    g.d = r.range(4, 11);
    g.kern = r.range(1, 2);
    g.shape = r.range(0, kNShapes - 1);
    g.rank = r.range(1, 4);
    g.tins = r.range(2, tins_hi);
    g.alater = r.range(3, 8);
    g.afirst = r.range(1, 4);
    g.small = r.range(0, 4);
    g.sblock = r.range(0, 5);
    g.swarp = r.range(0, 3);
    g.sgiant = r.range(0, 4);
    return g;
}

// The library's defaults as a genome (seeded into the first generation).
Genome default_genome(int w) {
    Genome g;
    g.algo = EVOSORT_ALGO_RADIX;
    g.d = 8;
    g.kern = 2;
    g.shape = 0;
    g.rank = 4;
    g.tins = 32;
    g.alater = 5;
    g.afirst = 2;
    g.small = 3;                  // 4096
    g.sblock = w == 4 ? 5 : 4;    // 8192 / 4096
    g.swarp = 3;                  // 256
    g.sgiant = 3;                 // 2^24
    return g;
}

// Register-tile shape `i` of the preference list for the key width.
void reg_shape_for(int w, int i, int* block, int* kpt) {
    static const int k4[][2] = {{1024, 16}, {512, 16}};
    static const int k8[][2] = {{1024, 12}, {1024, 8}, {512, 8}};
    if (w == 4) {
        *block = k4[i % 2][0];
        *kpt = k4[i % 2][1];
    } else {
        *block = k8[i % 3][0];
        *kpt = k8[i % 3][1];
    }
}

void to_params(const Genome& g, int w, evosort_params* p, void* stream) {
    evosort_default_params(p);
    p->algo = g.algo;
    p->digit_bits = g.d;
    p->pass_kernel = g.kern;
    if (g.kern == 2) {
        reg_shape_for(w, g.shape, &p->block_size, &p->keys_per_thread);
    } else if (g.kern == 1) {
        p->block_size = kShapes[g.shape][0];
        p->keys_per_thread = kShapes[g.shape][1];
    }
    p->rank_mode = g.rank;
    p->insertion_threshold = g.tins;
    p->adapt_later = g.alater;
    p->adapt_first = g.afirst;
    p->small_cap = g.small ? kSmallCaps[g.small] : 1;
    p->seg_block_cap = g.sblock || g.swarp || g.sgiant ? kBlockCaps[g.sblock] : 0;
    p->seg_warp_cap = g.sblock || g.swarp || g.sgiant ? kWarpCaps[g.swarp] : 0;
    p->seg_giant = g.sblock || g.swarp || g.sgiant ? kGiants[g.sgiant] : 0;
    p->stream = stream;
}

// ---- device-side checks of a candidate's output ----------------------------
__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// flags[0] |= 1 on any mismatch with the reference
template <typename U>
__global__ void check_equal(const U* a, const U* b, size_t n, uint32_t* flags) {
    bool bad = false;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        bad |= a[i] != b[i];
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 1u);
}

// flags[0] |= 2 if out is not non-decreasing under the key map; sums[0..1]
// accumulate an order-independent fingerprint of in, sums[2..3] of out
template <typename U>
__global__ void check_sorted_fingerprint(const U* in, const U* out, size_t n, KeyMap map, uint32_t* flags,
                                         unsigned long long* sums) {
    bool bad = false;
    unsigned long long s_in = 0, x_in = 0, s_out = 0, x_out = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint64_t hi = fmix64((uint64_t)in[i]), ho = fmix64((uint64_t)out[i]);
        s_in += hi;
        x_in ^= hi;
        s_out += ho;
        x_out ^= ho;
        if (i + 1 < n && map_fwd(out[i], map) > map_fwd(out[i + 1], map)) bad = true;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 2u);
    atomicAdd(&sums[0], s_in);
    atomicXor(&sums[1], x_in);
    atomicAdd(&sums[2], s_out);
    atomicXor(&sums[3], x_out);
}

struct Scratch {
    uint32_t* flags = nullptr;
    unsigned long long* sums = nullptr;
};

bool verify(const void* sample, const void* out, const void* expected, size_t n, int dt, Scratch& sc,
            cudaStream_t s) {
    const int w = dtype_bytes(dt);
    cudaMemsetAsync(sc.flags, 0, 4, s);
    cudaMemsetAsync(sc.sums, 0, 32, s);
    const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, (size_t)sm_count() * 8);
    const KeyMap m = key_map_for(dt);
    if (expected) {
        if (w == 4) check_equal<uint32_t><<<grid, 256, 0, s>>>((const uint32_t*)out, (const uint32_t*)expected, n, sc.flags);
        else check_equal<uint64_t><<<grid, 256, 0, s>>>((const uint64_t*)out, (const uint64_t*)expected, n, sc.flags);
    } else {
        if (w == 4)
            check_sorted_fingerprint<uint32_t><<<grid, 256, 0, s>>>((const uint32_t*)sample, (const uint32_t*)out,
                                                                   n, m, sc.flags, sc.sums);
        else
            check_sorted_fingerprint<uint64_t><<<grid, 256, 0, s>>>((const uint64_t*)sample, (const uint64_t*)out,
                                                                   n, m, sc.flags, sc.sums);
    }
    count_launches(1);
    uint32_t f = 0;
    unsigned long long h[4] = {0, 0, 0, 0};
    cudaMemcpyAsync(&f, sc.flags, 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h, sc.sums, 32, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return false;
    if (f) return false;
    if (!expected && (h[0] != h[2] || h[1] != h[3])) return false;
    return true;
}

}  // namespace
}  // namespace evosort

using namespace evosort;

extern "C" {

void evosort_default_ga_config(evosort_ga_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->population = 30;
    c->generations = 10;
    c->crossover_p = 0.7;
    c->mutation_p = 0.3;
    c->gene_mutation_p = 0.2;
    c->elite = 2;
    c->tournament = 3;
    c->reps = 3;
    c->tins_init_max = 256;
    c->seed = 42;
    c->allow_merge = 1;
}

evosort_status evosort_ga_search(const evosort_ga_config* cfg, int key_bytes, evosort_fitness_fn fitness_cb,
                                 void* ctx, evosort_params* best, float* best_ms, evosort_ga_log* log,
                                 int log_cap) {
    set_error("");
    evosort_ga_config c;
    if (cfg) c = *cfg;
    else evosort_default_ga_config(&c);
    if (!fitness_cb || !best || (key_bytes != 4 && key_bytes != 8) || c.population < 4 || c.generations < 1 ||
        c.reps < 1 || c.tournament < 1 || c.elite < 0 || c.elite >= c.population || c.tins_init_max < 2 ||
        c.tins_init_max > 2048 || (c.mode != MODE_ARRAY && c.mode != MODE_SEGMENTED)) {
        set_error("evosort_ga_search: bad GA configuration");
        return EVOSORT_ERR_INVALID;
    }
    const int w = key_bytes;
    const size_t n = c.sample_keys ? (size_t)c.sample_keys : ~(size_t)0;
    Rng rng{c.seed};
    std::map<Genome, float> cache;
    Genome champion = default_genome(w);
    float champion_f = INFINITY;
    auto fitness = [&](const Genome& g0) -> float {
        const Genome g = g0.canon(c.mode, n, w);
        auto it = cache.find(g);
        if (it != cache.end()) return it->second;
        evosort_params p;
        to_params(g0, w, &p, nullptr);
        float f = fitness_cb(&p, std::isfinite(champion_f) ? champion_f : -1.f, ctx);
        if (!(f >= 0.f)) f = INFINITY;   // negative or NaN: failed genome
        cache[g] = f;
        return f;
    };
    auto restrict_genes = [&](Genome& g) {
        if (!c.allow_merge) g.algo = EVOSORT_ALGO_RADIX;
    };
    // initial population (the paper draws T_insertion from [2, 256] first)
    std::vector<Genome> pop(c.population);
    for (auto& g : pop) {
        g = random_genome(rng, c.tins_init_max);
        restrict_genes(g);
    }
    // seed the defaults so the tuned result is never worse than the plain path
    pop[0] = default_genome(w);
    std::vector<float> fit(c.population);
    for (int gen = 0; gen < c.generations; ++gen) {
        for (int i = 0; i < c.population; ++i) {
            fit[i] = fitness(pop[i]);
            if (fit[i] < champion_f) {
                champion_f = fit[i];
                champion = pop[i];
            }
        }
        std::vector<int> idx(c.population);
        for (int i = 0; i < c.population; ++i) idx[i] = i;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return fit[a] < fit[b]; });
        if (log && gen < log_cap) {
            float worst = 0, sum = 0;
            int nfin = 0;
            for (float f : fit)
                if (std::isfinite(f)) {
                    worst = std::max(worst, f);
                    sum += f;
                    ++nfin;
                }
            log[gen].generation = gen;
            log[gen].best_ms = fit[idx[0]];
            log[gen].mean_ms = nfin ? sum / nfin : INFINITY;
            log[gen].worst_ms = nfin ? worst : INFINITY;
            log[gen].evaluations = (int)cache.size();
            to_params(pop[idx[0]].canon(c.mode, n, w), w, &log[gen].best, nullptr);
        }
        if (gen == c.generations - 1) break;
        // next generation: elites, then tournament-selected parents with
        // uniform crossover and uniform mutation
        std::vector<Genome> next;
        for (int i = 0; i < c.elite; ++i) next.push_back(pop[idx[i]]);
        auto select = [&]() {
            int b = rng.range(0, c.population - 1);
            for (int t = 1; t < c.tournament; ++t) {
                const int o = rng.range(0, c.population - 1);
                if (fit[o] < fit[b] || (fit[o] == fit[b] && o < b)) b = o;
            }
            return pop[b];
        };
        while ((int)next.size() < c.population) {
            Genome a = select(), b = select();
            if (rng.unit() < c.crossover_p) {
                // uniform crossover: each gene from either parent
                int* ga[] = {&a.algo, &a.d, &a.kern, &a.shape, &a.rank, &a.tins, &a.alater, &a.afirst, &a.small,
                             &a.sblock, &a.swarp, &a.sgiant};
                int* gb[] = {&b.algo, &b.d, &b.kern, &b.shape, &b.rank, &b.tins, &b.alater, &b.afirst, &b.small,
                             &b.sblock, &b.swarp, &b.sgiant};
                for (int k = 0; k < 12; ++k)
                    if (rng.unit() < 0.5) std::swap(*ga[k], *gb[k]);
            }
            for (Genome* g : {&a, &b}) {
                if (rng.unit() < c.mutation_p) {
                    // uniform mutation: each gene redrawn with gene_mutation_p
                    const Genome r = random_genome(rng, 2048);
                    int* gg[] = {&g->algo, &g->d, &g->kern, &g->shape, &g->rank, &g->tins, &g->alater, &g->afirst,
                                 &g->small, &g->sblock, &g->swarp, &g->sgiant};
                    const int* rr[] = {&r.algo, &r.d, &r.kern, &r.shape, &r.rank, &r.tins, &r.alater, &r.afirst,
                                       &r.small, &r.sblock, &r.swarp, &r.sgiant};
                    for (int k = 0; k < 12; ++k)
                        if (rng.unit() < c.gene_mutation_p) *gg[k] = *rr[k];
                }
                restrict_genes(*g);
            }
            next.push_back(a);
            if ((int)next.size() < c.population) next.push_back(b);
        }
        pop.swap(next);
    }
    if (!std::isfinite(champion_f)) {
        set_error("evosort_ga_search: no genome produced a verified sort");
        return EVOSORT_ERR_CUDA;
    }
    // reported with the genes that had no effect set to the defaults
    to_params(champion.canon(c.mode, n, w), w, best, nullptr);
    if (best_ms) *best_ms = champion_f;
    return EVOSORT_OK;
}

namespace {
struct DeviceFitness {
    const void* sample;
    const void* expected;
    void* out;
    size_t n;
    evosort_dtype dt;
    cudaStream_t s;
    int reps;
    Scratch sc;
    cudaEvent_t e0, e1;
};

// fitness of one genome: verified device time of a sort of the sample
float device_fitness(const evosort_params* p0, float champion_ms, void* ctx) {
    DeviceFitness& F = *(DeviceFitness*)ctx;
    evosort_params p = *p0;
    p.stream = F.s;
    cudaEventRecord(F.e0, F.s);
    const bool ran = evosort_sort_to(F.sample, F.out, F.n, F.dt, &p) == EVOSORT_OK;
    cudaEventRecord(F.e1, F.s);
    float f = -1.f;
    if (ran && evosort_sync(F.s) == EVOSORT_OK && verify(F.sample, F.out, F.expected, F.n, F.dt, F.sc, F.s)) {
        float first = 0;
        cudaEventElapsedTime(&first, F.e0, F.e1);
        std::vector<float> t;
        // a genome far slower than the best so far is not timed again
        const int reps = (champion_ms > 0.f && first > 4.f * champion_ms) ? 0 : F.reps;
        if (reps == 0) t.push_back(first);
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(F.e0, F.s);
            evosort_sort_to(F.sample, F.out, F.n, F.dt, &p);
            cudaEventRecord(F.e1, F.s);
            cudaEventSynchronize(F.e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, F.e0, F.e1);
            t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        f = t[t.size() / 2];
        if (evosort_sync(F.s) != EVOSORT_OK) f = -1.f;
    }
    cudaGetLastError();
    return f;
}
}  // namespace

evosort_status evosort_tune(const void* sample, size_t n, evosort_dtype dt, const void* expected,
                            const evosort_ga_config* cfg, void* stream, evosort_params* best, float* best_ms,
                            evosort_ga_log* log, int log_cap) {
    set_error("");
    if (!sample || !best || n < 2) {
        set_error("evosort_tune: need a device sample of at least 2 keys and an output params struct");
        return EVOSORT_ERR_INVALID;
    }
    if (dt < EVOSORT_I32 || dt > EVOSORT_F64) {
        set_error("unknown dtype");
        return EVOSORT_ERR_INVALID;
    }
    evosort_ga_config c;
    if (cfg) c = *cfg;
    else evosort_default_ga_config(&c);
    c.mode = MODE_ARRAY;
    c.sample_keys = n;
    DeviceFitness F;
    F.sample = sample;
    F.expected = expected;
    F.n = n;
    F.dt = dt;
    F.s = (cudaStream_t)stream;
    F.reps = c.reps;
    const int w = dtype_bytes(dt);
    cudaError_t e = cudaMallocAsync(&F.out, n * w, F.s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&F.sc.flags, 64, F.s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&F.sc.sums, 64, F.s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("evosort_tune: allocation: ") + cudaGetErrorString(e));
        return EVOSORT_ERR_NOMEM;
    }
    cudaEventCreate(&F.e0);
    cudaEventCreate(&F.e1);
    const evosort_status st = evosort_ga_search(&c, w, device_fitness, &F, best, best_ms, log, log_cap);
    cudaEventDestroy(F.e0);
    cudaEventDestroy(F.e1);
    cudaFreeAsync(F.out, F.s);
    cudaFreeAsync(F.sc.flags, F.s);
    cudaFreeAsync(F.sc.sums, F.s);
    cudaStreamSynchronize(F.s);
    if (st == EVOSORT_OK) best->stream = stream;
    return st;
}

}  // extern "C"
