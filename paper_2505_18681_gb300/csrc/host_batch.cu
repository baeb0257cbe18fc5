// Sort of arrays held in host memory: three device slots, an upload stream
// and a download stream around the caller's stream, so that the upload of the
// next array and the download of the previous one overlap the sort of the
// current one on the GPU.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "evosort.h"
#include "api_internal.h"
#include "common.cuh"

using namespace evosort;

namespace {

constexpr int kSlots = 3;

struct BatchRes {
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t ev_start = nullptr, ev_alloc = nullptr, ev_up_done = nullptr, ev_down_done = nullptr;
    cudaEvent_t loaded[kSlots] = {}, sorted[kSlots] = {}, drained[kSlots] = {};
    bool ok = false;

    std::string create() {
        cudaError_t e = cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking);
        cudaEvent_t* all[] = {&ev_start, &ev_alloc, &ev_up_done, &ev_down_done};
        for (cudaEvent_t* ev : all)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        for (int k = 0; k < kSlots && e == cudaSuccess; ++k) {
            e = cudaEventCreateWithFlags(&loaded[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sorted[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&drained[k], cudaEventDisableTiming);
        }
        ok = e == cudaSuccess;
        return ok ? std::string() : std::string(cudaGetErrorString(e));
    }
    // Streams and events are released once the work enqueued on them is done.
    ~BatchRes() {
        cudaEvent_t evs[] = {ev_start, ev_alloc, ev_up_done, ev_down_done};
        for (cudaEvent_t ev : evs)
            if (ev) cudaEventDestroy(ev);
        for (int k = 0; k < kSlots; ++k) {
            if (loaded[k]) cudaEventDestroy(loaded[k]);
            if (sorted[k]) cudaEventDestroy(sorted[k]);
            if (drained[k]) cudaEventDestroy(drained[k]);
        }
        if (up) cudaStreamDestroy(up);
        if (down) cudaStreamDestroy(down);
    }
};

bool ranges_overlap(const void* a, const void* b, size_t bytes) {
    const char* x = (const char*)a;
    const char* y = (const char*)b;
    return x != y && x < y + bytes && y < x + bytes;
}

evosort_status fail(evosort_status st, const std::string& msg) {
    set_error("evosort_sort_host_batch: " + msg);
    return st;
}

}  // namespace

extern "C" evosort_status evosort_sort_host_batch(const void* const* keys_in, void* const* keys_out,
                                                  const size_t* n, size_t count, evosort_dtype dt,
                                                  const evosort_params* p) {
    set_error("");
    if (dt < EVOSORT_I32 || dt > EVOSORT_F64) return fail(EVOSORT_ERR_INVALID, "unknown dtype");
    if (count == 0) return EVOSORT_OK;
    if (!keys_in || !keys_out || !n) return fail(EVOSORT_ERR_INVALID, "null array list");
    const int w = dtype_bytes(dt);
    size_t max_n = 0;
    for (size_t i = 0; i < count; ++i) {
        if (n[i] == 0) continue;
        if (!keys_in[i] || !keys_out[i]) return fail(EVOSORT_ERR_INVALID, "null key pointer");
        if (((uintptr_t)keys_in[i] % w) || ((uintptr_t)keys_out[i] % w))
            return fail(EVOSORT_ERR_INVALID, "misaligned key pointer");
        if (ranges_overlap(keys_in[i], keys_out[i], n[i] * w))
            return fail(EVOSORT_ERR_INVALID, "keys_in and keys_out overlap");
        if (n[i] >= (1ull << 40)) return fail(EVOSORT_ERR_UNSUPPORTED, "n >= 2^40");
        max_n = std::max(max_n, n[i]);
    }
    if (max_n == 0) return EVOSORT_OK;

    // per-array parameters: the caller's, or the dispatcher's from a host sample
    evosort_params base;
    evosort_default_params(&base);
    if (p) base = *p;
    if (evosort_workspace_bytes(max_n, dt, 0, &base) == 0) return fail(EVOSORT_ERR_INVALID, "bad parameters");
    const bool plan_each = base.algo == EVOSORT_ALGO_AUTO && table_nonempty();
    cudaStream_t s = (cudaStream_t)base.stream;

    std::string err;
    if (!status_word(&err)) return fail(EVOSORT_ERR_CUDA, err);
    BatchRes r;
    err = r.create();
    if (!r.ok) return fail(EVOSORT_ERR_CUDA, "stream/event creation: " + err);

    // slots come from the stream-ordered pool on the caller's stream; the copy
    // streams start after the allocation and after the caller's earlier work
    void* slot[kSlots] = {};
    const size_t slot_bytes = max_n * w;
    const int nslots = (int)std::min<size_t>(kSlots, count);
    for (int k = 0; k < nslots; ++k) {
        cudaError_t e = cudaMallocAsync(&slot[k], slot_bytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j < k; ++j) cudaFreeAsync(slot[j], s);
            return fail(EVOSORT_ERR_NOMEM, std::string("device slots: ") + cudaGetErrorString(e));
        }
    }
    cudaEventRecord(r.ev_alloc, s);
    cudaStreamWaitEvent(r.up, r.ev_alloc, 0);
    cudaStreamWaitEvent(r.down, r.ev_alloc, 0);

    evosort_status st = EVOSORT_OK;
    size_t k = 0;   // slot of the next non-empty array
    size_t used = 0;
    for (size_t i = 0; i < count && st == EVOSORT_OK; ++i) {
        if (n[i] == 0) continue;
        const size_t bytes = n[i] * w;
        // upload into the slot once the download of its previous array is done
        if (used >= (size_t)nslots) cudaStreamWaitEvent(r.up, r.drained[k], 0);
        cudaError_t e = cudaMemcpyAsync(slot[k], keys_in[i], bytes, cudaMemcpyHostToDevice, r.up);
        cudaEventRecord(r.loaded[k], r.up);
        // sort on the caller's stream
        evosort_params pi = base;
        if (plan_each) {
            const int cls = classify_host(keys_in[i], n[i], dt, base.descending != 0);
            evosort_params tp;
            if (table_lookup(dt, n[i], cls, &tp)) {
                pi = tp;
                pi.workspace = base.workspace;
                pi.workspace_bytes = base.workspace_bytes;
                pi.descending = base.descending;
            } else {
                pi.algo = EVOSORT_ALGO_RADIX;
            }
            pi.stream = base.stream;
        }
        cudaStreamWaitEvent(s, r.loaded[k], 0);
        if (e == cudaSuccess) {
            st = evosort_sort(slot[k], n[i], dt, &pi);
        } else {
            cudaGetLastError();
            st = fail(EVOSORT_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
        }
        cudaEventRecord(r.sorted[k], s);
        // download after the sort
        cudaStreamWaitEvent(r.down, r.sorted[k], 0);
        if (st == EVOSORT_OK) {
            e = cudaMemcpyAsync(keys_out[i], slot[k], bytes, cudaMemcpyDeviceToHost, r.down);
            if (e != cudaSuccess) {
                cudaGetLastError();
                st = fail(EVOSORT_ERR_CUDA, std::string("download: ") + cudaGetErrorString(e));
            }
        }
        cudaEventRecord(r.drained[k], r.down);
        k = (k + 1) % nslots;
        ++used;
    }
    // the caller's stream waits for both copy streams, then returns the slots
    cudaEventRecord(r.ev_up_done, r.up);
    cudaEventRecord(r.ev_down_done, r.down);
    cudaStreamWaitEvent(s, r.ev_up_done, 0);
    cudaStreamWaitEvent(s, r.ev_down_done, 0);
    for (int j = 0; j < nslots; ++j) cudaFreeAsync(slot[j], s);
    return st;
}
