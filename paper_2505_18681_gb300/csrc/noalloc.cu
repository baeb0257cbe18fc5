// Keys-only radix sort that allocates nothing (evosort_sort_noalloc).
//
// Some callers may not allocate device memory on the path where they sort:
// code that runs inside another framework's execute callback (an inference
// server plugin, a custom operator) where that framework owns all device
// memory and forbids allocation calls, or a latency-critical loop that must
// not block in the allocator or fail with out-of-memory half way through.
// This entry point serves them: its scratch space is a buffer of fixed size
// in the library's own device image.  The CUDA runtime loads that image
// lazily by default, so the buffer is reserved on each device the first time
// this entry point runs there (or when the library's module is loaded, if
// lazy loading is turned off), and it stays reserved until the process exits.
#include <mutex>

#include "evosort.h"
#include "api_internal.h"
#include "common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;   // 64 MiB per device

// The scratch buffer.  Every device where it has been reserved holds one until
// the process exits.  In host code this name only stands for the buffer; its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64];   // device address of the buffer, per device

}  // namespace

extern "C" evosort_status evosort_sort_noalloc(const void* keys_in, void* keys_out, size_t n, evosort_dtype dt,
                                               void* stream) {
    using namespace evosort;
    set_error("");
    if (dt < EVOSORT_I32 || dt > EVOSORT_F64) {
        set_error("unknown dtype");
        return EVOSORT_ERR_INVALID;
    }
    if (n == 0) return EVOSORT_OK;
    const int w = dtype_bytes(dt);
    if (!keys_in || !keys_out) {
        set_error("null key pointer");
        return EVOSORT_ERR_INVALID;
    }
    if (((uintptr_t)keys_in % w) || ((uintptr_t)keys_out % w)) {
        set_error("misaligned key pointer");
        return EVOSORT_ERR_INVALID;
    }
    const char* a = (const char*)keys_in;
    const char* b = (const char*)keys_out;
    if (a != b && a < b + n * w && b < a + n * w) {
        set_error("keys_in and keys_out overlap");
        return EVOSORT_ERR_INVALID;
    }
    Plan pl;
    default_radix_plan(dt, &pl, n);   // the tile shape the allocating sort would pick for n keys
    const size_t need = radix_workspace_bytes(n, w, false, pl);
    if (need > kNoAllocScratchBytes) {
        set_error("evosort_sort_noalloc: " + std::to_string(n) + " keys need " + std::to_string(need) +
                  " bytes of scratch; its fixed buffer holds " + std::to_string(kNoAllocScratchBytes) +
                  " bytes (64 MiB)");
        return EVOSORT_ERR_INVALID;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return EVOSORT_ERR_CUDA;
    }
    void* scratch = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                set_error(std::string("cudaGetSymbolAddress of the scratch buffer: ") + cudaGetErrorString(e));
                return EVOSORT_ERR_CUDA;
            }
            g_noalloc_addr[dev] = p;
        }
        scratch = g_noalloc_addr[dev];
    }
    std::string err;
    const int rc = radix_sort(keys_in, keys_out, nullptr, nullptr, n, dt, pl, scratch, kNoAllocScratchBytes,
                              (cudaStream_t)stream, &err);
    if (rc != EVOSORT_OK) set_error(err);
    return (evosort_status)rc;
}
