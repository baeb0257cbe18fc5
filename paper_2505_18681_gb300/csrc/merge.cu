// Bottom-up mergesort (Algorithm 3 of the paper).
#include "evosort.h"
#include "api_internal.h"
#include "common.cuh"

namespace evosort {

size_t merge_workspace_bytes(size_t n, int w, bool pairs, const Plan&) {
    return ((n * w + 255) / 256 + (pairs ? (n * 4 + 255) / 256 : 0)) * 256 + 256;
}

int merge_sort(const void*, void*, const uint32_t*, uint32_t*, size_t, int, const Plan&, void*, size_t,
               cudaStream_t, std::string* err) {
    *err = "mergesort not built yet";
    return EVOSORT_ERR_UNSUPPORTED;
}

}  // namespace evosort
