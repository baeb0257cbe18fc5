// Dispatcher of Algorithm 5 (AdaptivePartitionSort): picks the algorithm and
// its parameters for one call from a table of tuned parameters, keyed by key
// type, size bucket (floor(log2 n)) and a distribution class read off a small
// strided sample of the keys.  The paper keys its parameters on n alone (one
// GA run per size); the class adds what the data itself changes on a GPU:
// which digits are constant, how many lanes of a warp share a digit.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "evosort.h"
#include "api_internal.h"
#include "common.cuh"

namespace evosort {
namespace {

struct Entry {
    int dt, bucket, cls;
    evosort_params p;
    float ms;
};
std::mutex g_tab_mu;
std::vector<Entry> g_tab;

constexpr int kSample = 4096;

uint64_t host_map(uint64_t u, int dt, bool descending) {
    // order-preserving map of key bits, host copy (same definition as the kernels')
    const int w = dtype_bytes(dt);
    const KeyMap m = key_map_for(dt, descending);
    if (w == 4) {
        const uint32_t x = (uint32_t)u;
        const uint32_t sar = (x & 0x80000000u) ? 0xFFFFFFFFu : 0u;
        return (uint32_t)(((x ^ ((sar & (uint32_t)m.f) | (uint32_t)m.s)) - (uint32_t)m.r) ^ (uint32_t)m.x);
    }
    const uint64_t sar = (u >> 63) ? ~0ull : 0ull;
    return ((u ^ ((sar & m.f) | m.s)) - m.r) ^ m.x;
}

}  // namespace

// Class of a sample of m keys (raw bytes, m x key width), taken at stride
// n / m from an array of n keys, read in the order of the sort's direction.
// With info, the distinct sampled keys (mapped, ascending) when there are at
// most kDictMax of them, and the sample's order (1: no pair falls, -1: no
// pair rises, 0: both happen).
int classify_sample(const unsigned char* buf, size_t m, int dt, bool descending, SampleInfo* info) {
    const int w = dtype_bytes(dt);
    std::vector<uint64_t> raw(m, 0);
    for (size_t i = 0; i < m; ++i) {
        uint64_t u = 0;
        std::memcpy(&u, buf + i * w, w);
        raw[i] = host_map(u, dt, descending);
    }
    // strict rises and falls between neighbours: equal neighbours say
    // nothing about order (90% zeros would otherwise read as both sorted and
    // reverse sorted)
    size_t up = 0, down = 0;
    uint64_t vary = 0;
    for (size_t i = 0; i + 1 < m; ++i) {
        up += raw[i] < raw[i + 1];
        down += raw[i] > raw[i + 1];
    }
    for (size_t i = 0; i < m; ++i) vary |= raw[i] ^ raw[0];
    std::vector<uint64_t> sorted(raw);
    std::sort(sorted.begin(), sorted.end());
    const size_t distinct = std::unique(sorted.begin(), sorted.end()) - sorted.begin();
    if (info) {
        info->dict.clear();
        if (distinct <= (size_t)kDictMax) info->dict.assign(sorted.begin(), sorted.begin() + distinct);
        info->order = down == 0 ? 1 : (up == 0 ? -1 : 0);
    }
    // top-byte concentration: share of the sample in the most common top byte
    size_t top[256] = {0};
    for (size_t i = 0; i < m; ++i) top[(raw[i] >> (8 * w - 8)) & 0xFF] += 1;
    const size_t topmax = *std::max_element(top, top + 256);
    int bits = 0;
    while (bits < 64 && (vary >> bits)) ++bits;
    if (distinct == 1) return EVOSORT_CLASS_CONSTANT;
    if (distinct <= 64) return EVOSORT_CLASS_FEW;          // few values, whatever their order
    const size_t moves = up + down;
    if (up >= 0.9 * (double)moves) return EVOSORT_CLASS_SORTED;
    if (down >= 0.9 * (double)moves) return EVOSORT_CLASS_REVERSE;
    if (bits <= 16) return EVOSORT_CLASS_NARROW16;
    if (bits <= 4 * w) return EVOSORT_CLASS_NARROW;          // at most half the key bits vary
    if (topmax * 4 > m) return EVOSORT_CLASS_SKEWED;         // a quarter in one top byte
    return EVOSORT_CLASS_RANDOM;
}

// Class of n keys in host memory, from the same strided sample the device
// path copies (read here directly, no CUDA call).
int classify_host(const void* keys, size_t n, int dt, bool descending) {
    if (n < 2) return EVOSORT_CLASS_CONSTANT;
    const int w = dtype_bytes(dt);
    const size_t m = n < (size_t)kSample ? n : (size_t)kSample;
    const size_t stride = n / m;
    std::vector<unsigned char> buf(m * w);
    for (size_t i = 0; i < m; ++i) std::memcpy(buf.data() + i * w, (const unsigned char*)keys + i * stride * w, w);
    return classify_sample(buf.data(), m, dt, descending);
}

// Table entry for (dt, n, cls): the class itself at the nearest size bucket,
// else the random class; false (and *out untouched) when neither is present.
bool table_lookup(int dt, size_t n, int cls, evosort_params* out) {
    int bucket = 0;
    while (bucket < 63 && (n >> (bucket + 1))) ++bucket;
    std::lock_guard<std::mutex> lk(g_tab_mu);
    const Entry* best = nullptr;
    int bestd = 1 << 30;
    for (int pass = 0; pass < (cls == EVOSORT_CLASS_SEGMENTED ? 1 : 2) && !best; ++pass) {
        const int want = pass == 0 ? cls : EVOSORT_CLASS_RANDOM;
        for (const auto& x : g_tab)
            if (x.dt == dt && x.cls == want && std::abs(x.bucket - bucket) < bestd) {
                best = &x;
                bestd = std::abs(x.bucket - bucket);
            }
    }
    if (!best) return false;
    *out = best->p;
    return true;
}

bool table_nonempty() {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    return !g_tab.empty();
}

// Class of keys[0..n) (a device array) from a strided sample, read in the
// order of the sort's direction (synchronises the stream).
evosort_status classify_device(const void* keys, size_t n, int dt, void* stream, bool descending,
                                        int* cls, SampleInfo* info = nullptr) {
    set_error("");
    if (!cls || (n && !keys) || dt < EVOSORT_I32 || dt > EVOSORT_F64) {
        set_error("evosort_classify: bad argument");
        return EVOSORT_ERR_INVALID;
    }
    const int w = dtype_bytes(dt);
    if (n < 2) {
        *cls = EVOSORT_CLASS_CONSTANT;
        return EVOSORT_OK;
    }
    const size_t m = n < (size_t)kSample ? n : (size_t)kSample;
    const size_t stride = n / m;
    std::vector<unsigned char> buf(m * w);
    // one strided device-to-host copy of m keys
    cudaError_t e = cudaMemcpy2DAsync(buf.data(), w, keys, stride * w, w, m, cudaMemcpyDeviceToHost,
                                      (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error(std::string("evosort_classify: sample copy: ") + cudaGetErrorString(e));
        return EVOSORT_ERR_CUDA;
    }
    *cls = classify_sample(buf.data(), m, dt, descending, info);
    return EVOSORT_OK;
}

evosort_status plan_for(const void* keys, size_t n, int dt, void* stream, bool descending,
                                 evosort_params* out, int* cls_out, SampleInfo* info) {
    set_error("");
    if (!out) {
        set_error("evosort_plan: null output");
        return EVOSORT_ERR_INVALID;
    }
    evosort_default_params(out);
    out->stream = stream;
    int cls = EVOSORT_CLASS_RANDOM;
    if (table_nonempty() && n >= 2) {
        const evosort_status st = classify_device(keys, n, dt, stream, descending, &cls, info);
        if (st != EVOSORT_OK) return st;
        if (table_lookup(dt, n, cls, out)) out->stream = stream;
        out->descending = descending ? 1 : 0;
    }
    if (cls_out) *cls_out = cls;
    return EVOSORT_OK;
}

}  // namespace evosort

using namespace evosort;

extern "C" {


evosort_status evosort_classify(const void* keys, size_t n, evosort_dtype dt, void* stream, int* cls) {
    return classify_device(keys, n, dt, stream, false, cls);
}

evosort_status evosort_table_set(evosort_dtype dt, int size_bucket, int cls, const evosort_params* p, float ms) {
    if (!p || dt < EVOSORT_I32 || dt > EVOSORT_F64 || size_bucket < 0 || size_bucket > 63 || cls < 0 ||
        cls > EVOSORT_CLASS_SEGMENTED) {
        set_error("evosort_table_set: bad argument");
        return EVOSORT_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_tab_mu);
    Entry en{dt, size_bucket, cls, *p, ms};
    en.p.stream = nullptr;
    en.p.workspace = nullptr;
    en.p.workspace_bytes = 0;
    for (auto& x : g_tab)
        if (x.dt == dt && x.bucket == size_bucket && x.cls == cls) {
            x = en;
            return EVOSORT_OK;
        }
    g_tab.push_back(en);
    return EVOSORT_OK;
}

void evosort_table_clear(void) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    g_tab.clear();
}

size_t evosort_table_size(void) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    return g_tab.size();
}

evosort_status evosort_table_save(const char* path) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    std::ofstream f(path ? path : "");
    if (!f) {
        set_error("evosort_table_save: cannot open file");
        return EVOSORT_ERR_INVALID;
    }
    f << "# evosort tuned table: dtype size_bucket class algo digit_bits block_size keys_per_thread "
         "rank_mode insertion_threshold seg_block_cap ms [pass_kernel adapt_later adapt_first seg_warp_cap "
         "small_cap seg_giant]\n";
    for (const auto& x : g_tab)
        f << x.dt << ' ' << x.bucket << ' ' << x.cls << ' ' << x.p.algo << ' ' << x.p.digit_bits << ' '
          << x.p.block_size << ' ' << x.p.keys_per_thread << ' ' << x.p.rank_mode << ' '
          << x.p.insertion_threshold << ' ' << x.p.seg_block_cap << ' ' << x.ms << ' ' << x.p.pass_kernel << ' '
          << x.p.adapt_later << ' ' << x.p.adapt_first << ' ' << x.p.seg_warp_cap << ' ' << x.p.small_cap << ' '
          << x.p.seg_giant << '\n';
    return f ? EVOSORT_OK : EVOSORT_ERR_INVALID;
}

evosort_status evosort_table_load(const char* path) {
    std::ifstream f(path ? path : "");
    if (!f) {
        set_error("evosort_table_load: cannot open file");
        return EVOSORT_ERR_INVALID;
    }
    std::string line;
    int lineno = 0;
    while (std::getline(f, line)) {
        ++lineno;
        if (line.empty() || line[0] == '#') continue;
        std::istringstream is(line);
        int dt, bucket, cls;
        evosort_params p;
        evosort_default_params(&p);
        float ms = 0;
        if (!(is >> dt >> bucket >> cls >> p.algo >> p.digit_bits >> p.block_size >> p.keys_per_thread >>
              p.rank_mode >> p.insertion_threshold >> p.seg_block_cap >> ms)) {
            set_error("evosort_table_load: malformed line " + std::to_string(lineno));
            return EVOSORT_ERR_INVALID;
        }
        // optional later columns (0 = default when absent)
        int extra[5] = {0, 0, 0, 0, 0};
        long long giant = 0;
        int got = 0;
        while (got < 5 && (is >> extra[got])) ++got;
        if (got == 5) is >> giant;
        if (!is.eof() && is.fail() && got > 0 && got < 5) {
            set_error("evosort_table_load: malformed optional columns on line " + std::to_string(lineno));
            return EVOSORT_ERR_INVALID;
        }
        p.pass_kernel = extra[0];
        p.adapt_later = extra[1];
        p.adapt_first = extra[2];
        p.seg_warp_cap = extra[3];
        p.small_cap = extra[4];
        p.seg_giant = giant;
        const evosort_status st = evosort_table_set((evosort_dtype)dt, bucket, cls, &p, ms);
        if (st != EVOSORT_OK) return st;
    }
    return EVOSORT_OK;
}

evosort_status evosort_plan(const void* keys, size_t n, evosort_dtype dt, void* stream, evosort_params* out,
                            int* cls_out) {
    return plan_for(keys, n, dt, stream, false, out, cls_out);
}

evosort_status evosort_plan_host(const void* keys, size_t n, evosort_dtype dt, int descending, evosort_params* out,
                                 int* cls_out) {
    set_error("");
    if (!out || (n && !keys) || dt < EVOSORT_I32 || dt > EVOSORT_F64) {
        set_error("evosort_plan_host: bad argument");
        return EVOSORT_ERR_INVALID;
    }
    evosort_default_params(out);
    int cls = EVOSORT_CLASS_RANDOM;
    if (table_nonempty() && n >= 2) {
        cls = classify_host(keys, n, dt, descending != 0);
        table_lookup(dt, n, cls, out);
        out->stream = nullptr;
    }
    out->descending = descending ? 1 : 0;
    if (cls_out) *cls_out = cls;
    return EVOSORT_OK;
}

}  // extern "C"
