// C ABI of the sort library: argument checks, parameter resolution, scratch
// memory and the dispatcher of Algorithm 5 (AdaptivePartitionSort).
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "evosort.h"
#include "api_internal.h"
#include "closed_form.h"
#include "radix_launch.cuh"

namespace evosort {

// Device status word: kernels OR error bits into it; evosort_sync reads and
// clears it.
__device__ uint32_t g_status_word;

static thread_local std::string t_err;
static std::atomic<uint64_t> g_launches{0};
static std::atomic<uint32_t> g_wait_limit{0};

uint32_t wait_limit() {
    const uint32_t v = g_wait_limit.load(std::memory_order_relaxed);
    return v ? v : kSpinLimit;
}

void set_error(const std::string& msg) { t_err = msg; }
void count_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static std::mutex g_dev_mu;
struct DevInfo {
    bool init = false;
    int sms = 0;
    uint32_t* status = nullptr;
};
static DevInfo g_dev[64];

const DevInfo* device_info(std::string* err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        *err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DevInfo& di = g_dev[dev];
    if (!di.init) {
        e = cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&di.status, g_status_word);
        if (e == cudaSuccess) {
            // keep freed scratch in the stream-ordered pool instead of returning
            // it to the CUDA driver after every call
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t thr = ~0ull;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
        }
        if (e != cudaSuccess) {
            *err = std::string("device set-up: ") + cudaGetErrorString(e);
            return nullptr;
        }
        di.init = true;
    }
    return &di;
}

int sm_count() {
    std::string err;
    const DevInfo* di = device_info(&err);
    return di ? di->sms : 148;
}

uint32_t* status_word(std::string* err) {
    const DevInfo* di = device_info(err);
    return di ? di->status : nullptr;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// Instrumentation: CUDA events around every launch while enabled.  Each sort
// call also copies its radix pass descriptors to pinned host memory so a
// record can say whether the pass ran or was skipped.
// ---------------------------------------------------------------------------
struct ProfRecord {
    int kind, pass, call;
    int rank;   // adaptive ranking: the variant this launch runs (0: not adaptive)
    double bytes;
    uint64_t items;
    cudaEvent_t e0, e1;
};
struct ProfCall {
    PassDesc* host_desc;   // pinned copy, npass + 1 entries (radix calls)
    int ndesc;
    cudaEvent_t copied;    // recorded after the copy into host_desc
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRecord> g_prof;
static std::vector<ProfCall> g_prof_calls;
// pinned arena for the descriptor copies (allocated when profiling is enabled,
// so nothing is allocated while a measured region runs)
constexpr size_t kArenaDescs = 1 << 14;
static PassDesc* g_arena = nullptr;
static size_t g_arena_used = 0;

bool prof_enabled() { return g_prof_on; }

int prof_call_begin(const PassDesc* dev_desc, int ndesc, cudaStream_t) {
    if (!g_prof_on) return -1;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfCall c{nullptr, 0, nullptr};
    if (dev_desc && ndesc > 0 && g_arena && g_arena_used + ndesc <= kArenaDescs) {
        c.host_desc = g_arena + g_arena_used;
        c.ndesc = ndesc;
        g_arena_used += ndesc;
    }
    g_prof_calls.push_back(c);
    return (int)g_prof_calls.size() - 1;
}

void prof_call_end(int call, cudaStream_t s, const PassDesc* dev_desc) {
    if (call < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfCall& c = g_prof_calls[call];
    if (c.host_desc && dev_desc) {
        cudaMemcpyAsync(c.host_desc, dev_desc, sizeof(PassDesc) * c.ndesc, cudaMemcpyDeviceToHost, s);
        // the copy comes after the call's last launch event: the reader waits
        // for this event, not only for the launches, before it uses the copy
        if (cudaEventCreateWithFlags(&c.copied, cudaEventDisableTiming) == cudaSuccess)
            cudaEventRecord(c.copied, s);
        else
            c.copied = nullptr;
    }
}

ProfScope::ProfScope(int call, int kind, int pass, double bytes, uint64_t items, cudaStream_t s, int rank)
    : call_(call), idx_(-1), s_(s) {
    if (!g_prof_on || call < 0) return;
    ProfRecord r{kind, pass, call, rank, bytes, items, nullptr, nullptr};
    cudaEventCreate(&r.e0);
    cudaEventCreate(&r.e1);
    cudaEventRecord(r.e0, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back(r);
    idx_ = (int)g_prof.size() - 1;
}

ProfScope::~ProfScope() {
    if (idx_ < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(g_prof[idx_].e1, s_);
}


// ---------------------------------------------------------------------------
// Radix sort: scratch layout and launch sequence.
// ---------------------------------------------------------------------------
struct RadixLayout {
    int npass;
    size_t ntiles;
    int lb64;
    size_t off_desc, off_tiles, off_counts, off_range, off_counts2, off_cbins, off_lookback, zero_end, off_tmp, off_vtmp,
        total;
};

static RadixLayout radix_layout(size_t n, int w, bool pairs, const Plan& pl) {
    RadixLayout L;
    L.npass = (8 * w + pl.digit_bits - 1) / pl.digit_bits;
    const size_t tile = (size_t)pl.block_size * pl.keys_per_thread;
    L.ntiles = (n + tile - 1) / tile;
    L.lb64 = n >= (1ull << 30) ? 1 : 0;
    const size_t bins = (size_t)1 << pl.digit_bits;
    size_t off = 0;
    L.off_desc = off;
    off = align_up(off + (L.npass + 1) * sizeof(PassDesc), 256);
    L.off_tiles = off;
    off = align_up(off + (L.npass + 4) * sizeof(uint32_t), 256);   // tile counters, then the order flags
    L.off_counts = off;
    off = align_up(off + L.npass * bins * sizeof(unsigned long long), 256);
    L.off_range = off;   // RNG_WORDS range words (smallest / largest key, bias, flags)
    off = align_up(off + RNG_WORDS * sizeof(unsigned long long), 256);
    L.off_counts2 = off;   // digit counts of the rebased keys (8-bit digits only)
    off = align_up(off + (pl.digit_bits == 8 ? L.npass * bins * sizeof(unsigned long long) : 0), 256);
    L.off_cbins = off;   // value bins of the narrow-range counting sort (keys only, 8-bit digits)
    off = align_up(off + (pl.digit_bits == 8 && !pairs ? counting_bins_bytes() : 0), 256);
    L.off_lookback = off;
    off = align_up(off + (size_t)L.npass * L.ntiles * bins * (L.lb64 ? 8 : 4), 256);
    L.zero_end = off;
    L.off_tmp = off;
    off = align_up(off + n * w, 256);
    L.off_vtmp = off;
    if (pairs) off = align_up(off + n * sizeof(uint32_t), 256);
    L.total = off;
    return L;
}

size_t radix_workspace_bytes(size_t n, int w, bool pairs, const Plan& pl) {
    return radix_layout(n, w, pairs, pl).total;
}

int radix_sort(const void* in, void* out, const uint32_t* vin, uint32_t* vout, size_t n, int dt,
               const Plan& pl, void* ws, size_t ws_bytes, cudaStream_t s, std::string* err) {
    const int w = dtype_bytes(dt);
    const bool pairs = vout != nullptr;
    RadixLayout L = radix_layout(n, w, pairs, pl);
    if (ws_bytes < L.total) {
        *err = "workspace too small";
        return EVOSORT_ERR_NOMEM;
    }
    uint32_t* status = status_word(err);
    if (!status) return EVOSORT_ERR_CUDA;
    char* base = (char*)ws;
    RadixArgs a;
    a.in = in;
    a.out = out;
    a.tmp = base + L.off_tmp;
    a.vin = vin;
    a.vout = vout;
    a.vtmp = pairs ? (uint32_t*)(base + L.off_vtmp) : nullptr;
    a.n = n;
    a.dt = dt;
    a.map = key_map_for(dt, pl.descending);
    a.d = pl.digit_bits;
    a.npass = L.npass;
    a.lb64 = L.lb64;
    // adaptive ranking pays one extra (empty) launch per pass; below a few
    // million keys the match-mask ranking alone runs
    const bool adapt = pl.rank_mode == 4 && n >= kAdaptMinKeys;
    const int rank = pl.rank_mode == 4 ? 3 : pl.rank_mode;
    a.adapt = adapt ? 1 : 0;
    a.conc_later = std::ldexp(1.0, -pl.adapt_later);
    a.conc_first = std::ldexp(1.0, -pl.adapt_first);
    a.spin_limit = wait_limit();
    a.ntiles = L.ntiles;
    a.desc = (PassDesc*)(base + L.off_desc);
    a.counts = (unsigned long long*)(base + L.off_counts);
    a.lookback = base + L.off_lookback;
    a.tile_counter = (uint32_t*)(base + L.off_tiles);
    a.order = a.tile_counter + L.npass;
    a.range = (unsigned long long*)(base + L.off_range);
    a.counts2 = (unsigned long long*)(base + L.off_counts2);
    a.status = status;
    const int inplace = (in == out) ? 1 : 0;

    cudaError_t e = cudaMemsetAsync(base, 0, L.zero_end, s);
    const int sms = sm_count();
    const size_t hist_smem = (size_t)L.npass * ((size_t)1 << pl.digit_bits) * sizeof(uint32_t);
    size_t hist_grid = (n + 1024 * 16 - 1) / (1024 * 16);
    if (hist_grid > (size_t)sms) hist_grid = (size_t)sms;   // one 1024-thread CTA per SM (128 KB counters)
    if (hist_grid < 1) hist_grid = 1;
    const int vb = pairs ? 4 : 0;
    const double pass_bytes = 2.0 * (double)n * (w + vb);
    const int call = prof_call_begin(a.desc, L.npass + 1, s);
    {
        ProfScope ps(call, EVOSORT_K_RADIX_HISTOGRAM, -1, (double)n * w, n, s);
        if (e == cudaSuccess) e = launch_radix_aux(w, 0, hist_grid, hist_smem, s, a, inplace);
    }
    if (pl.digit_bits == 8) {
        // K1b: recount the digits of key - min when that leaves fewer passes
        // (it returns at once otherwise; whether it ran is decided on the
        // device, so its record carries no bytes)
        ProfScope ps(call, EVOSORT_K_RADIX_HISTOGRAM, -2, 0.0, n, s);
        if (e == cudaSuccess) e = launch_radix_aux(w, 3, hist_grid, hist_smem, s, a, inplace);
    }
    {
        ProfScope ps(call, EVOSORT_K_RADIX_SCAN, -1, 0.0, 0, s);
        if (e == cudaSuccess) e = launch_radix_aux(w, 1, 1, 0, s, a, inplace);
    }
    if (pl.digit_bits == 8 && !pairs) {
        // narrow key range: counting sort in place of the passes (decided on
        // the device; the two kernels return at once otherwise)
        ProfScope ps(call, EVOSORT_K_RADIX_COUNT, -1, 0.0, n, s);
        if (e == cudaSuccess)
            e = launch_radix_counting(w, a, (unsigned long long*)(base + L.off_cbins), s);
    }
    const bool reg = pl.pass_kernel == 2;
    for (int p = 0; p < L.npass && e == cudaSuccess; ++p) {
        for (int v = 0; v < (adapt ? 2 : 1) && e == cudaSuccess; ++v) {
            const int r = v == 0 ? rank : 1;
            ProfScope ps(call, EVOSORT_K_RADIX_ONESWEEP, p, pass_bytes, n, s, adapt ? r : 0);
            if (reg && w == 4)
                e = launch_onesweep_reg_u32(pairs, pl.block_size, pl.keys_per_thread, r, L.ntiles, sms, s, a, p);
            else if (reg)
                e = launch_onesweep_reg_u64(pairs, pl.block_size, pl.keys_per_thread, r, L.ntiles, sms, s, a, p);
            else if (w == 4)
                e = launch_onesweep_u32(pairs, pl.block_size, pl.keys_per_thread, r, L.ntiles, sms, s, a, p);
            else
                e = launch_onesweep_u64(pairs, pl.block_size, pl.keys_per_thread, r, L.ntiles, sms, s, a, p);
        }
    }
    size_t fix_grid = (n + 256 * 8 - 1) / (256 * 8);
    if (fix_grid > (size_t)sms * 8) fix_grid = (size_t)sms * 8;
    {
        ProfScope ps(call, EVOSORT_K_RADIX_FIXUP, L.npass, pass_bytes, n, s);
        if (e == cudaSuccess) e = launch_radix_aux(w, 2, fix_grid, 0, s, a, inplace);
    }
    prof_call_end(call, s, a.desc);
    count_launches(3 + (pl.digit_bits == 8 ? 1 : 0) + (pl.digit_bits == 8 && !pairs ? 2 : 0) +
                   (adapt ? 2 : 1) * L.npass);
    if (e != cudaSuccess) {
        *err = std::string("radix launch: ") + cudaGetErrorString(e);
        return EVOSORT_ERR_CUDA;
    }
    return EVOSORT_OK;
}

}  // namespace evosort

using namespace evosort;

// ---------------------------------------------------------------------------
// Parameter resolution.
// ---------------------------------------------------------------------------
static void defaults_for(int w, Plan* pl) {
    pl->algo = EVOSORT_ALGO_RADIX;
    pl->digit_bits = 8;
    pl->block_size = 0;        // chosen by default_tile_shape once pairs/d are known
    pl->keys_per_thread = 0;
    pl->insertion_threshold = 32;
    pl->rank_mode = 4;
    pl->seg_block_cap = w == 4 ? 8192 : 4096;
    pl->descending = false;
    pl->pass_kernel = 0;   // chosen with the tile shape
    pl->adapt_later = 5;   // 1/32
    pl->adapt_first = 2;   // 1/4
    pl->seg_warp_cap = 256;
    pl->small_cap = kSmallDefault;
    pl->seg_giant = (long long)1 << 24;
}

// Register-tile shapes in order of preference per key width and form, and
// whether the register tile is the default pass kernel for that form (where
// it measured faster than the staged tile).
static const int kRegPref32k[][2] = {{1024, 16}, {512, 16}};
static const int kRegPref32p[][2] = {{1024, 12}, {1024, 8}};
static const int kRegPref64k[][2] = {{1024, 12}, {1024, 8}, {512, 8}};
static const int kRegPref64p[][2] = {{1024, 12}, {1024, 8}, {512, 8}};

// Measured at 1e9 int64 / 5e8 key-value sorts: 5.30 vs 6.54 ms per int64 pass,
// 29.9 vs 43.9 ms for float64 + uint32 pairs, 12.3 vs 14.4 ms for int32 pairs.
static bool reg_by_default(int, bool) { return true; }

static void reg_prefs(int w, bool pairs, const int (**pref)[2], int* np) {
    if (w == 4 && !pairs) { *pref = kRegPref32k; *np = 2; }
    else if (w == 4) { *pref = kRegPref32p; *np = 2; }
    else if (!pairs) { *pref = kRegPref64k; *np = 3; }
    else { *pref = kRegPref64p; *np = 3; }
}

// Default radix tile shape and pass kernel.  The register tile is tried first
// when it is requested (pass_kernel 2) or is the default for the form
// (pass_kernel 0); the staged tile otherwise, or when no register tile gives
// at least half of the SMs a tile of a small input.  Within a kernel the
// first shape of the preference list (largest tiles first, so fewer tiles
// are in flight in the look-back) that fits is taken; with n known (n > 0), a
// shape is skipped while it would leave more than half of the SMs without a
// tile (n / tile < SMs / 2) and a smaller preferred shape fits: small sorts
// then fill the GPU.  (The GA's winners at 2^20 keys follow this rule: 8K-key
// tiles for 32-bit keys, against 16K above 2^22.)
// Fitted log2 tile size at n (the closed form of the tuned tables, L = log10 n
// clamped to the tuned range).
static double fitted_log2_tile(int w, size_t n) {
    const double* f = w == 4 ? kTileFit32 : kTileFit64;
    double L = std::log10((double)(n < 2 ? 2 : n));
    L = L < f[3] ? f[3] : (L > f[4] ? f[4] : L);
    return f[0] + f[1] * L + f[2] * L * L;
}

static void default_tile_shape(int w, bool pairs, Plan* pl, size_t n = 0) {
    const bool given = pl->block_size && pl->keys_per_thread;
    const size_t half = (size_t)(sm_count() / 2);
    if (pl->pass_kernel == 2 || (pl->pass_kernel == 0 && reg_by_default(w, pairs))) {
        const int(*pref0)[2];
        int np = 0;
        reg_prefs(w, pairs, &pref0, &np);
        // with n known, the preference order is by distance from the fitted
        // tile size (nearest first, ties to the larger tile); the "fills half
        // the SMs" rule below still guards small inputs
        int pref[4][2];
        for (int i = 0; i < np; ++i) {
            pref[i][0] = pref0[i][0];
            pref[i][1] = pref0[i][1];
        }
        if (n > 0 && !given) {
            const double t = fitted_log2_tile(w, n);
            for (int i = 1; i < np; ++i)
                for (int j = i; j > 0; --j) {
                    const double da = std::fabs(std::log2((double)pref[j][0] * pref[j][1]) - t);
                    const double db = std::fabs(std::log2((double)pref[j - 1][0] * pref[j - 1][1]) - t);
                    const bool larger = pref[j][0] * pref[j][1] > pref[j - 1][0] * pref[j - 1][1];
                    if (da < db - 1e-9 || (std::fabs(da - db) <= 1e-9 && larger)) {
                        std::swap(pref[j][0], pref[j - 1][0]);
                        std::swap(pref[j][1], pref[j - 1][1]);
                    } else {
                        break;
                    }
                }
        }
        int chosen = -1;
        for (int i = 0; i < np; ++i) {
            const int b = pl->block_size ? pl->block_size : pref[i][0];
            const int k = pl->keys_per_thread ? pl->keys_per_thread : pref[i][1];
            if (!reg_config_fits(w, pairs, b, k, pl->digit_bits, pl->rank_mode)) continue;
            chosen = i;
            if (given || n == 0 || n / ((size_t)b * k) >= half) break;
            chosen = -2 - i;   // fits, but leaves SMs idle: keep looking
        }
        if (chosen >= 0 || (pl->pass_kernel == 2 && chosen != -1)) {
            const int i = chosen >= 0 ? chosen : -2 - chosen;
            if (!pl->block_size) pl->block_size = pref[i][0];
            if (!pl->keys_per_thread) pl->keys_per_thread = pref[i][1];
            pl->pass_kernel = 2;
            return;
        }
        if (pl->pass_kernel == 2) return;   // nothing fits: reported by the caller's check
    }
    pl->pass_kernel = 1;
    static const int pref4[][2] = {{512, 32}, {1024, 16}, {512, 16}, {1024, 8}, {256, 16}, {256, 8}};
    static const int pref8[][2] = {{1024, 8}, {512, 16}, {1024, 4}, {512, 8}, {256, 16}, {256, 8}};
    const int(*pref)[2] = w == 4 ? pref4 : pref8;
    int chosen = -1;
    for (int i = 0; i < 6; ++i) {
        const int b = pl->block_size ? pl->block_size : pref[i][0];
        const int k = pl->keys_per_thread ? pl->keys_per_thread : pref[i][1];
        if (onesweep_config_fits(w, pairs, b, k, pl->digit_bits, pl->rank_mode) &&
            onesweep_rank_fits(pl->rank_mode, b, k, w, pairs, pl->digit_bits)) {
            chosen = i;
            const bool fills = n == 0 || n / ((size_t)b * k) >= half;
            if (fills || given) break;
        }
    }
    if (chosen >= 0) {
        if (!pl->block_size) pl->block_size = pref[chosen][0];
        if (!pl->keys_per_thread) pl->keys_per_thread = pref[chosen][1];
        return;
    }
    if (!pl->block_size) pl->block_size = 256;
    if (!pl->keys_per_thread) pl->keys_per_thread = 16;
}

static int resolve(const evosort_params* p, int dt, bool pairs, Plan* pl, std::string* err, size_t n = 0) {
    const int w = dtype_bytes(dt);
    defaults_for(w, pl);
    if (!p) {
        default_tile_shape(w, pairs, pl, n);
        return EVOSORT_OK;
    }
    pl->descending = p->descending != 0;
    if (p->algo != EVOSORT_ALGO_AUTO) pl->algo = p->algo;
    if (p->digit_bits) pl->digit_bits = p->digit_bits;
    if (p->block_size) pl->block_size = p->block_size;
    if (p->keys_per_thread) pl->keys_per_thread = p->keys_per_thread;
    if (p->insertion_threshold) pl->insertion_threshold = p->insertion_threshold;
    if (p->seg_block_cap) pl->seg_block_cap = p->seg_block_cap;
    if (pl->seg_block_cap < 256 || pl->seg_block_cap > (w == 4 ? 8192 : 4096)) {
        *err = "params.seg_block_cap must be in [256, 8192] (32-bit keys) or [256, 4096] (64-bit keys)";
        return EVOSORT_ERR_INVALID;
    }
    pl->pass_kernel = p->pass_kernel;
    if (pl->pass_kernel < 0 || pl->pass_kernel > 2) {
        *err = "params.pass_kernel must be 0, 1 or 2";
        return EVOSORT_ERR_INVALID;
    }
    if (p->adapt_later) pl->adapt_later = p->adapt_later;
    if (p->adapt_first) pl->adapt_first = p->adapt_first;
    if (pl->adapt_later < 1 || pl->adapt_later > 10 || pl->adapt_first < 1 || pl->adapt_first > 10) {
        *err = "params.adapt_later / adapt_first must be in [1, 10]";
        return EVOSORT_ERR_INVALID;
    }
    if (p->seg_warp_cap) pl->seg_warp_cap = p->seg_warp_cap;
    if (pl->seg_warp_cap != 32 && pl->seg_warp_cap != 64 && pl->seg_warp_cap != 128 && pl->seg_warp_cap != 256) {
        *err = "params.seg_warp_cap must be 32, 64, 128 or 256";
        return EVOSORT_ERR_INVALID;
    }
    if (p->small_cap) pl->small_cap = p->small_cap;
    if (pl->small_cap < 1 || pl->small_cap > kSmallMax) {
        *err = "params.small_cap must be 0 (default), 1 (off) or at most 8192";
        return EVOSORT_ERR_INVALID;
    }
    if (p->seg_giant) pl->seg_giant = p->seg_giant;
    if (pl->seg_giant != -1 && (pl->seg_giant < 1024 || (pl->seg_giant & (pl->seg_giant - 1)))) {
        *err = "params.seg_giant must be 0 (default), -1 (off) or a power of two of at least 1024";
        return EVOSORT_ERR_INVALID;
    }
    if (p->rank_mode) pl->rank_mode = p->rank_mode;
    else if (pl->digit_bits > 8) pl->rank_mode = 2;   // match masks are compiled for d <= 8
    else if (pl->digit_bits < 8) pl->rank_mode = 3;   // match.any is compiled for d = 8
    if (pl->algo != EVOSORT_ALGO_RADIX && pl->algo != EVOSORT_ALGO_MERGE) {
        *err = "params.algo must be -1, 0 or 1";
        return EVOSORT_ERR_INVALID;
    }
    if (pl->digit_bits < 4 || pl->digit_bits > 11) {
        *err = "params.digit_bits must be in [4, 11]";
        return EVOSORT_ERR_INVALID;
    }
    if (pl->rank_mode < 1 || pl->rank_mode > 4) {
        *err = "params.rank_mode must be 1, 2, 3 or 4";
        return EVOSORT_ERR_INVALID;
    }
    if (pl->insertion_threshold < 2 || pl->insertion_threshold > 2048) {
        *err = "params.insertion_threshold must be in [2, 2048]";
        return EVOSORT_ERR_INVALID;
    }
    if (pl->algo == EVOSORT_ALGO_RADIX && !onesweep_rank_supported(pl->rank_mode, pl->digit_bits)) {
        *err = "params.rank_mode: 1 (match.any) and 4 (adaptive) need digit_bits 8, 3 (match masks) needs "
               "digit_bits <= 8";
        return EVOSORT_ERR_INVALID;
    }
    if (pl->algo == EVOSORT_ALGO_RADIX && (!pl->block_size || !pl->keys_per_thread || !pl->pass_kernel))
        default_tile_shape(dtype_bytes(dt), pairs, pl, n);
    if (pl->algo == EVOSORT_ALGO_RADIX && pl->pass_kernel != 2 &&
        !onesweep_shape_supported(pl->block_size, pl->keys_per_thread)) {
        *err = "params.block_size/keys_per_thread: unsupported radix tile shape";
        return EVOSORT_ERR_INVALID;
    }
    return EVOSORT_OK;
}

static bool valid_dtype(int dt) { return dt >= EVOSORT_I32 && dt <= EVOSORT_F64; }

namespace evosort {
// The built-in parameters of a keys-only radix sort of n keys of dtype dt
// (n = 0: the tile shape for large inputs).
void default_radix_plan(int dt, Plan* pl, size_t n) {
    std::string err;
    resolve(nullptr, dt, false, pl, &err, n);
    pl->algo = EVOSORT_ALGO_RADIX;
}
}  // namespace evosort

static bool overlaps(const void* a, const void* b, size_t bytes) {
    const char* x = (const char*)a;
    const char* y = (const char*)b;
    return x != y && x < y + bytes && y < x + bytes;
}

static evosort_status finish(int rc, const std::string& err) {
    if (rc != EVOSORT_OK) set_error(err);
    return (evosort_status)rc;
}

static evosort_status sort_common(const void* in, void* out, const uint32_t* vin, uint32_t* vout, size_t n,
                                  evosort_dtype dt, const evosort_params* p) {
    std::string err;
    set_error("");
    if (!valid_dtype(dt)) return finish(EVOSORT_ERR_INVALID, "unknown dtype");
    if (n == 0) return EVOSORT_OK;
    const int w = dtype_bytes(dt);
    if (!in || !out) return finish(EVOSORT_ERR_INVALID, "null key pointer");
    if (((uintptr_t)in % w) || ((uintptr_t)out % w)) return finish(EVOSORT_ERR_INVALID, "misaligned key pointer");
    const bool pairs = vout != nullptr || vin != nullptr;
    if (pairs && (!vin || !vout)) return finish(EVOSORT_ERR_INVALID, "null value pointer");
    if (pairs && (((uintptr_t)vin % 4) || ((uintptr_t)vout % 4)))
        return finish(EVOSORT_ERR_INVALID, "misaligned value pointer");
    if (overlaps(in, out, n * w)) return finish(EVOSORT_ERR_INVALID, "keys_in and keys_out overlap");
    if (pairs && overlaps(vin, vout, n * 4)) return finish(EVOSORT_ERR_INVALID, "values_in and values_out overlap");
    if (pairs && (in == out) != ((const void*)vin == (const void*)vout))
        return finish(EVOSORT_ERR_INVALID, "keys and values must both be in place or both out of place");
    if (n >= (1ull << 40)) return finish(EVOSORT_ERR_UNSUPPORTED, "n >= 2^40");
    if (n == 1) {   // one key is sorted: in place nothing to do, else one copy
        cudaStream_t s1 = p ? (cudaStream_t)p->stream : nullptr;
        cudaError_t e1 = cudaSuccess;
        if (in != out) e1 = cudaMemcpyAsync(out, in, w, cudaMemcpyDeviceToDevice, s1);
        if (e1 == cudaSuccess && pairs && vin != vout) e1 = cudaMemcpyAsync(vout, vin, 4, cudaMemcpyDeviceToDevice, s1);
        if (e1 != cudaSuccess) return finish(EVOSORT_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e1));
        return EVOSORT_OK;
    }
    if (pairs && n > 0xFFFFFFFFull) return finish(EVOSORT_ERR_UNSUPPORTED, "key/value sorts need n < 2^32");
    // Algorithm 5's small-array branch: when the caller leaves the choice to
    // the dispatcher, arrays of at most small_cap keys are sorted by one CTA
    // in shared memory (one launch, no scratch, no sample of the keys)
    if (!p || p->algo == EVOSORT_ALGO_AUTO || p->small_cap > 1) {
        Plan sp;
        int rc0 = resolve(p, dt, pairs, &sp, &err, n);
        if (rc0) return finish(rc0, err);
        if (sp.small_cap > 1 && n <= (size_t)sp.small_cap) {
            rc0 = small_sort(in, out, vin, vout, n, dt, sp, p ? (cudaStream_t)p->stream : nullptr, &err);
            return finish(rc0, err);
        }
    }
    // dispatcher: tuned parameters for this input when the caller leaves the choice open
    evosort_params planned;
    if ((!p || p->algo == EVOSORT_ALGO_AUTO) && table_nonempty()) {
        void* st = p ? p->stream : nullptr;
        const bool desc = p && p->descending;
        int cls = EVOSORT_CLASS_RANDOM;
        SampleInfo info;
        const evosort_status ps = plan_for(in, n, dt, st, desc, &planned, &cls, &info);
        if (ps != EVOSORT_OK) return finish(ps, evosort_last_error());
        // a few distinct keys in the sample (keys only): counting sort over
        // those values, unless some key is not among them
        if (!pairs && cls == EVOSORT_CLASS_FEW && !info.dict.empty() && n >= kDictMinKeys) {
            bool done = false;
            const int rcd = dict_sort(in, out, n, dt, desc, info.dict, (cudaStream_t)st, &done, &err);
            if (rcd) return finish(rcd, err);
            if (done) return EVOSORT_OK;
        }
        // a sample in order (or in reverse order): copy checked on the way,
        // unless some key is out of order
        if (info.order != 0 && n >= kDictMinKeys) {
            bool done = false;
            const int rco = ordered_sort(in, out, vin, vout, n, dt, desc, info.order, (cudaStream_t)st, &done, &err);
            if (rco) return finish(rco, err);
            if (done) return EVOSORT_OK;
        }
        if (p) {
            planned.stream = p->stream;
            planned.workspace = p->workspace;
            planned.workspace_bytes = p->workspace_bytes;
            planned.descending = p->descending;
        }
        p = &planned;
    }
    Plan pl;
    int rc = resolve(p, dt, pairs, &pl, &err, n);
    if (rc) return finish(rc, err);
    auto tile_fits = [&](const Plan& q) {
        if (q.algo != EVOSORT_ALGO_RADIX) return true;
        if (q.pass_kernel == 2)
            return reg_config_fits(w, pairs, q.block_size, q.keys_per_thread, q.digit_bits, q.rank_mode);
        return onesweep_config_fits(w, pairs, q.block_size, q.keys_per_thread, q.digit_bits, q.rank_mode) &&
               onesweep_rank_fits(q.rank_mode, q.block_size, q.keys_per_thread, w, pairs, q.digit_bits);
    };
    if (p == &planned && !tile_fits(pl)) {
        // the tables are tuned on keys alone: a tile that cannot also hold the
        // values gives way to the default tile rule for this sort
        planned.block_size = planned.keys_per_thread = 0;
        planned.pass_kernel = 0;
        rc = resolve(p, dt, pairs, &pl, &err, n);
        if (rc) return finish(rc, err);
    }
    if (pl.algo == EVOSORT_ALGO_RADIX && pl.pass_kernel == 2 &&
        !reg_config_fits(w, pairs, pl.block_size, pl.keys_per_thread, pl.digit_bits, pl.rank_mode))
        return finish(EVOSORT_ERR_INVALID, "register-tile radix pass (pass_kernel 2): needs 8-bit digits, rank mode "
                                           "1, 3 or 4 and a compiled tile shape for this key width");
    if (pl.algo == EVOSORT_ALGO_RADIX && pl.pass_kernel != 2 &&
        (!onesweep_config_fits(w, pairs, pl.block_size, pl.keys_per_thread, pl.digit_bits, pl.rank_mode) ||
         !onesweep_rank_fits(pl.rank_mode, pl.block_size, pl.keys_per_thread, w, pairs, pl.digit_bits)))
        return finish(EVOSORT_ERR_INVALID, "radix tile does not fit in shared memory (block_size x "
                                           "keys_per_thread too large for this key width and digit width)");
    cudaStream_t s = p ? (cudaStream_t)p->stream : nullptr;

    size_t need = 0;
    if (pl.algo == EVOSORT_ALGO_MERGE) {
        need = merge_workspace_bytes(n, w, pairs, pl);
    } else {
        need = radix_workspace_bytes(n, w, pairs, pl);
    }
    void* ws = p ? p->workspace : nullptr;
    size_t ws_bytes = p ? p->workspace_bytes : 0;
    bool owned = false;
    if (!ws) {
        const DevInfo* di = device_info(&err);
        if (!di) return finish(EVOSORT_ERR_CUDA, err);
        cudaError_t e = cudaMallocAsync(&ws, need, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return finish(EVOSORT_ERR_NOMEM, std::string("scratch allocation: ") + cudaGetErrorString(e));
        }
        ws_bytes = need;
        owned = true;
    } else if ((uintptr_t)ws % 256) {
        return finish(EVOSORT_ERR_INVALID, "workspace must be 256-byte aligned");
    }
    if (pl.algo == EVOSORT_ALGO_MERGE)
        rc = merge_sort(in, out, vin, vout, n, dt, pl, ws, ws_bytes, s, &err);
    else
        rc = radix_sort(in, out, vin, vout, n, dt, pl, ws, ws_bytes, s, &err);
    if (owned) cudaFreeAsync(ws, s);
    return finish(rc, err);
}

extern "C" {

void evosort_default_params(evosort_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->algo = EVOSORT_ALGO_RADIX;
}

size_t evosort_workspace_bytes(size_t n, evosort_dtype dt, int with_values, const evosort_params* p) {
    std::string err;
    if (!valid_dtype(dt)) return 0;
    Plan pl;
    if (resolve(p, dt, with_values != 0, &pl, &err, n)) return 0;
    const int w = dtype_bytes(dt);
    if (pl.algo == EVOSORT_ALGO_MERGE) return merge_workspace_bytes(n, w, with_values != 0, pl);
    return radix_workspace_bytes(n, w, with_values != 0, pl);
}

evosort_status evosort_resolve(size_t n, evosort_dtype dt, int with_values, const evosort_params* p,
                               evosort_params* out) {
    std::string err;
    set_error("");
    if (!valid_dtype(dt) || !out) return finish(EVOSORT_ERR_INVALID, "evosort_resolve: bad argument");
    Plan pl;
    const int rc = resolve(p, dt, with_values != 0, &pl, &err, n);
    if (rc) return finish(rc, err);
    evosort_default_params(out);
    out->algo = pl.algo;
    out->digit_bits = pl.digit_bits;
    out->keys_per_thread = pl.keys_per_thread;
    out->block_size = pl.block_size;
    out->insertion_threshold = pl.insertion_threshold;
    out->rank_mode = pl.rank_mode;
    out->seg_block_cap = pl.seg_block_cap;
    out->descending = pl.descending ? 1 : 0;
    out->pass_kernel = pl.pass_kernel;
    out->adapt_later = pl.adapt_later;
    out->adapt_first = pl.adapt_first;
    out->seg_warp_cap = pl.seg_warp_cap;
    // the one-CTA path is considered only when the choice is left to the
    // dispatcher or a cut-over is given (sort_common); otherwise it is off
    out->small_cap = (p && p->algo != EVOSORT_ALGO_AUTO && p->small_cap <= 1) ? 1 : pl.small_cap;
    out->seg_giant = pl.seg_giant;
    if (p) {
        out->stream = p->stream;
        out->workspace = p->workspace;
        out->workspace_bytes = p->workspace_bytes;
    }
    return EVOSORT_OK;
}

evosort_status evosort_sort(void* keys, size_t n, evosort_dtype dt, const evosort_params* p) {
    return sort_common(keys, keys, nullptr, nullptr, n, dt, p);
}

evosort_status evosort_sort_to(const void* keys_in, void* keys_out, size_t n, evosort_dtype dt,
                               const evosort_params* p) {
    return sort_common(keys_in, keys_out, nullptr, nullptr, n, dt, p);
}

evosort_status evosort_sort_pairs(void* keys, uint32_t* values, size_t n, evosort_dtype dt,
                                  const evosort_params* p) {
    if (n && !values) return finish(EVOSORT_ERR_INVALID, "null value pointer");
    return sort_common(keys, keys, values, values, n, dt, p);
}

evosort_status evosort_sort_pairs_to(const void* keys_in, const uint32_t* values_in, void* keys_out,
                                     uint32_t* values_out, size_t n, evosort_dtype dt,
                                     const evosort_params* p) {
    if (n && (!values_in || !values_out)) return finish(EVOSORT_ERR_INVALID, "null value pointer");
    return sort_common(keys_in, keys_out, values_in, values_out, n, dt, p);
}

size_t evosort_segmented_workspace_bytes(size_t total, size_t nseg, evosort_dtype dt) {
    if (!valid_dtype(dt)) return 0;
    return segmented_workspace_bytes(total, nseg, dtype_bytes(dt));
}

evosort_status evosort_segmented_sort(void* keys, size_t total, const uint64_t* offsets, size_t nseg,
                                      evosort_dtype dt, const evosort_params* p) {
    std::string err;
    set_error("");
    if (!valid_dtype(dt)) return finish(EVOSORT_ERR_INVALID, "unknown dtype");
    if (nseg == 0) return total == 0 ? EVOSORT_OK : finish(EVOSORT_ERR_INVALID, "total keys with no segments");
    if (!offsets) return finish(EVOSORT_ERR_INVALID, "null offsets pointer");
    if ((uintptr_t)offsets % 8) return finish(EVOSORT_ERR_INVALID, "misaligned offsets pointer");
    const int w = dtype_bytes(dt);
    if (total && !keys) return finish(EVOSORT_ERR_INVALID, "null key pointer");
    if ((uintptr_t)keys % w) return finish(EVOSORT_ERR_INVALID, "misaligned key pointer");
    if (nseg >= 0xFFFFFFFFull) return finish(EVOSORT_ERR_UNSUPPORTED, "nseg >= 2^32");
    if (total >= (1ull << 40)) return finish(EVOSORT_ERR_UNSUPPORTED, "total >= 2^40");
    // tuned tier cut-overs for batches of this size when the caller leaves
    // the choice open
    evosort_params planned;
    if ((!p || p->algo == EVOSORT_ALGO_AUTO) && table_nonempty()) {
        evosort_default_params(&planned);
        planned.algo = EVOSORT_ALGO_AUTO;
        if (table_lookup(dt, total, EVOSORT_CLASS_SEGMENTED, &planned)) {
            if (p) {
                planned.stream = p->stream;
                planned.workspace = p->workspace;
                planned.workspace_bytes = p->workspace_bytes;
                planned.descending = p->descending;
            } else {
                planned.stream = nullptr;
                planned.workspace = nullptr;
                planned.workspace_bytes = 0;
            }
            p = &planned;
        }
    }
    Plan pl;
    int rc = resolve(p, dt, false, &pl, &err);
    if (rc) return finish(rc, err);
    cudaStream_t s = p ? (cudaStream_t)p->stream : nullptr;
    const size_t need = segmented_workspace_bytes(total, nseg, w);
    void* ws = p ? p->workspace : nullptr;
    size_t ws_bytes = p ? p->workspace_bytes : 0;
    bool owned = false;
    if (!ws) {
        const DevInfo* di = device_info(&err);
        if (!di) return finish(EVOSORT_ERR_CUDA, err);
        cudaError_t e = cudaMallocAsync(&ws, need, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return finish(EVOSORT_ERR_NOMEM, std::string("scratch allocation: ") + cudaGetErrorString(e));
        }
        ws_bytes = need;
        owned = true;
    } else if ((uintptr_t)ws % 256) {
        return finish(EVOSORT_ERR_INVALID, "workspace must be 256-byte aligned");
    }
    rc = segmented_sort(keys, total, offsets, nseg, dt, pl, ws, ws_bytes, !owned, s, &err);
    if (owned) cudaFreeAsync(ws, s);
    return finish(rc, err);
}

evosort_status evosort_sync(void* stream) {
    std::string err;
    set_error("");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return finish(EVOSORT_ERR_CUDA, std::string("synchronize: ") + cudaGetErrorString(e));
    uint32_t* sw = status_word(&err);
    if (!sw) return finish(EVOSORT_ERR_CUDA, err);
    uint32_t v = 0;
    e = cudaMemcpy(&v, sw, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return finish(EVOSORT_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    if (v) {
        uint32_t zero = 0;
        cudaMemcpy(sw, &zero, sizeof(zero), cudaMemcpyHostToDevice);
        if (v & ST_TIMEOUT) return finish(EVOSORT_ERR_TIMEOUT, "a bounded device wait ran out");
        if (v & ST_RANGE)
            return finish(EVOSORT_ERR_CUDA, "internal error: a radix scatter offset fell outside the array "
                                            "(stores skipped, output invalid)");
        return finish(EVOSORT_ERR_INVALID, "device-side argument check failed (segment offsets)");
    }
    return EVOSORT_OK;
}

evosort_status evosort_release(void) {
    set_error("");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();   // every stream-ordered free has run
    cudaMemPool_t pool;
    if (e == cudaSuccess) e = cudaDeviceGetDefaultMemPool(&pool, dev);
    if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
    if (e != cudaSuccess) return finish(EVOSORT_ERR_CUDA, std::string("release: ") + cudaGetErrorString(e));
    return EVOSORT_OK;
}

const char* evosort_last_error(void) { return t_err.c_str(); }

void evosort_set_wait_limit(uint32_t polls) { g_wait_limit.store(polls, std::memory_order_relaxed); }

evosort_status evosort_profile(int enable) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (enable && !g_arena) {
        cudaError_t e = cudaMallocHost((void**)&g_arena, sizeof(PassDesc) * kArenaDescs);
        if (e != cudaSuccess) {
            g_arena = nullptr;
            set_error(std::string("pinned arena: ") + cudaGetErrorString(e));
            return EVOSORT_ERR_CUDA;
        }
    }
    g_prof_on = enable != 0;
    return EVOSORT_OK;
}

size_t evosort_profile_read(evosort_kernel_record* out, size_t cap) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    size_t k = 0;
    for (size_t i = 0; i < g_prof.size(); ++i) {
        ProfRecord& r = g_prof[i];
        cudaEventSynchronize(r.e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.e0, r.e1);
        int active = 1;
        const ProfCall& c = g_prof_calls[r.call];
        if (c.copied) cudaEventSynchronize(c.copied);
        if (c.host_desc) {
            if (r.kind == EVOSORT_K_RADIX_ONESWEEP && r.pass >= 0 && r.pass < c.ndesc)
                active = c.host_desc[r.pass].active && (r.rank == 0 || c.host_desc[r.pass].rank == r.rank);
            if (r.kind == EVOSORT_K_RADIX_FIXUP && r.pass >= 0 && r.pass < c.ndesc)
                active = c.host_desc[r.pass].fixup != FIX_NONE;
        }
        if (out && k < cap) {
            out[k].kind = r.kind;
            out[k].pass = r.pass;
            out[k].active = active;
            out[k].ms = ms;
            out[k].bytes = active ? r.bytes : 0.0;
            out[k].items = r.items;
            out[k].rank = r.rank;
        }
        ++k;
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    for (ProfCall& c : g_prof_calls)
        if (c.copied) cudaEventDestroy(c.copied);
    g_arena_used = 0;
    g_prof.clear();
    g_prof_calls.clear();
    return k;
}

uint64_t evosort_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
