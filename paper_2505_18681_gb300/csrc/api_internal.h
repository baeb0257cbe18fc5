// Host-side declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "evosort.h"

namespace evosort {

// Resolved parameters of one sort call.
struct Plan {
    int algo;                 // 0 radix, 1 merge
    int digit_bits;           // radix digit width d
    int block_size;           // threads per CTA
    int keys_per_thread;      // keys each thread holds in a tile
    int insertion_threshold;  // mergesort base-run length
    int rank_mode;            // radix tile ranking variant
    int seg_block_cap;        // segmented sort: longest segment sorted in shared memory
    bool descending;          // non-increasing order
    int pass_kernel;          // radix pass kernel: 0 not chosen yet, 1 staged tile, 2 register tile
    int adapt_later;          // adaptive ranking thresholds, as -log2 of the concentration
    int adapt_first;
    int seg_warp_cap;         // segmented sort: warp tier below this length
    int small_cap;            // single-CTA path for lone arrays up to this size (1 = off)
    long long seg_giant;      // segmented sort: device-wide path above this length (-1 = off)
};

// Single-CTA path for lone small arrays (Algorithm 5's small-array branch):
// default and largest cut-over, in keys.
constexpr int kSmallDefault = 4096;
constexpr int kSmallMax = 8192;
int small_sort(const void* in, void* out, const uint32_t* vin, uint32_t* vout, size_t n, int dt, const Plan& pl,
               cudaStream_t s, std::string* err);

// Poll limit of the bounded device-side waits (look-back slots); set by
// evosort_set_wait_limit, 0 = the built-in default.
uint32_t wait_limit();

void set_error(const std::string& msg);
void default_radix_plan(int dt, Plan* pl, size_t n = 0);
bool table_nonempty();
// Largest distinct-value count of the dictionary path, and the smallest
// array it and the ordered path are tried on (below that the radix sort's
// fixed cost is small).
constexpr int kDictMax = 64;
constexpr size_t kDictMinKeys = (size_t)1 << 16;
// What a sample shows beyond its class: its distinct keys in the key map's
// order (ascending) when there are at most kDictMax, and whether every
// neighbour pair is non-decreasing (order 1), non-increasing (-1) or neither.
struct SampleInfo {
    std::vector<uint64_t> dict;
    int order = 0;
};
int classify_sample(const unsigned char* buf, size_t m, int dt, bool descending = false,
                    SampleInfo* info = nullptr);
int classify_host(const void* keys, size_t n, int dt, bool descending = false);
// evosort_plan for a sort in the given direction (the class is read in the
// order the sort will produce)
evosort_status plan_for(const void* keys, size_t n, int dt, void* stream, bool descending, evosort_params* out,
                        int* cls_out, SampleInfo* info = nullptr);
// Counting sort over the sample's distinct keys (keys only): *done is false
// when a key is not among them (the input is then untouched).
int dict_sort(const void* in, void* out, size_t n, int dt, bool descending, const std::vector<uint64_t>& dict,
              cudaStream_t s, bool* done, std::string* err);
// Copy (or reversed copy, keys only) of an input the sample shows in order
// (hint 1) or in reverse order (hint -1), checked on the way: *done is false
// when some key is out of order (the output is then to be rewritten; the
// input is untouched).
int ordered_sort(const void* in, void* out, const uint32_t* vin, uint32_t* vout, size_t n, int dt, bool descending,
                 int hint, cudaStream_t s, bool* done, std::string* err);
// Counting sort of a narrow key range inside the radix path (keys only,
// 8-bit digits): launched after K2, it decides on the device and, when it
// applies, sorts and turns the passes off.  bins: counting_bins_bytes() of
// zeroed scratch.
struct RadixArgs;
size_t counting_bins_bytes();
cudaError_t launch_radix_counting(int w, const RadixArgs& a, unsigned long long* bins, cudaStream_t s);
bool table_lookup(int dt, size_t n, int cls, evosort_params* out);

void count_launches(uint64_t k);
int sm_count();
uint32_t* status_word(std::string* err);

struct PassDesc;
bool prof_enabled();
int prof_call_begin(const PassDesc* dev_desc, int ndesc, cudaStream_t s);
void prof_call_end(int call, cudaStream_t s, const PassDesc* dev_desc);
// Records a CUDA event pair around one launch while instrumentation is on.
class ProfScope {
  public:
    ProfScope(int call, int kind, int pass, double bytes, uint64_t items, cudaStream_t s, int rank = 0);
    ~ProfScope();
  private:
    int call_, idx_;
    cudaStream_t s_;
};

// Smallest sort that uses adaptive ranking (rank mode 4); smaller ones rank
// with match masks only.
constexpr size_t kAdaptMinKeys = (size_t)1 << 21;
size_t radix_workspace_bytes(size_t n, int w, bool pairs, const Plan& pl);
int radix_sort(const void* in, void* out, const uint32_t* vin, uint32_t* vout, size_t n, int dt,
               const Plan& pl, void* ws, size_t ws_bytes, cudaStream_t s, std::string* err);

size_t segmented_workspace_bytes(size_t total, size_t nseg, int w);
int segmented_sort(void* keys, size_t total, const uint64_t* off, size_t nseg, int dt, const Plan& pl, void* ws,
                   size_t ws_bytes, bool caller_ws, cudaStream_t s, std::string* err);

size_t merge_workspace_bytes(size_t n, int w, bool pairs, const Plan& pl);
int merge_sort(const void* in, void* out, const uint32_t* vin, uint32_t* vout, size_t n, int dt,
               const Plan& pl, void* ws, size_t ws_bytes, cudaStream_t s, std::string* err);

}  // namespace evosort
