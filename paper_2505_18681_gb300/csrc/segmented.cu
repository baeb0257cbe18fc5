// Batched segmented sort.
#include "evosort.h"
#include "api_internal.h"

extern "C" evosort_status evosort_segmented_sort(void* keys, const uint64_t* offsets, size_t nseg,
                                                 evosort_dtype dt, const evosort_params* p) {
    (void)keys; (void)offsets; (void)nseg; (void)dt; (void)p;
    evosort::set_error("segmented sort not built yet");
    return EVOSORT_ERR_UNSUPPORTED;
}
