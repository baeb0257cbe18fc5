// Sort of arrays held in host memory: two device slots and one copy stream
// beside the caller's stream.  The copies run one at a time, in the order
// upload(0), upload(1), download(0), upload(2), download(1), ..., so the sort
// of array i (on the caller's stream) overlaps the upload of array i+1 and the
// download of array i-1.  One copy at a time because on the host link of this
// machine an upload and a download running together each fell to about a
// fifth of their speed alone (40 GB/s each way against 211 / 193 GB/s), and
// uploads split over several streams were slower than one.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "evosort.h"
#include "api_internal.h"
#include "common.cuh"

using namespace evosort;

namespace {

constexpr int kSlots = 2;

struct BatchRes {
    cudaStream_t xfer = nullptr;
    cudaEvent_t ev_alloc = nullptr, ev_xfer_done = nullptr;
    cudaEvent_t loaded[kSlots] = {}, sorted[kSlots] = {};
    bool ok = false;

    std::string create() {
        cudaError_t e = cudaStreamCreateWithFlags(&xfer, cudaStreamNonBlocking);
        cudaEvent_t* all[] = {&ev_alloc, &ev_xfer_done, &loaded[0], &loaded[1], &sorted[0], &sorted[1]};
        for (cudaEvent_t* ev : all)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        ok = e == cudaSuccess;
        return ok ? std::string() : std::string(cudaGetErrorString(e));
    }
    // Streams and events are released once the work enqueued on them is done.
    ~BatchRes() {
        cudaEvent_t evs[] = {ev_alloc, ev_xfer_done, loaded[0], loaded[1], sorted[0], sorted[1]};
        for (cudaEvent_t ev : evs)
            if (ev) cudaEventDestroy(ev);
        if (xfer) cudaStreamDestroy(xfer);
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
    // stream starts after the allocation and after the caller's earlier work
    void* slot[kSlots] = {};
    const size_t slot_bytes = max_n * w;
    std::vector<size_t> order;   // the non-empty arrays
    for (size_t i = 0; i < count; ++i)
        if (n[i]) order.push_back(i);
    const int nslots = (int)std::min<size_t>(kSlots, order.size());
    for (int k = 0; k < nslots; ++k) {
        cudaError_t e = cudaMallocAsync(&slot[k], slot_bytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j < k; ++j) cudaFreeAsync(slot[j], s);
            return fail(EVOSORT_ERR_NOMEM, std::string("device slots: ") + cudaGetErrorString(e));
        }
    }
    cudaEventRecord(r.ev_alloc, s);
    cudaStreamWaitEvent(r.xfer, r.ev_alloc, 0);

    evosort_status st = EVOSORT_OK;
    auto upload = [&](size_t j) {
        const size_t i = order[j];
        const int k = (int)(j % kSlots);
        cudaError_t e = cudaMemcpyAsync(slot[k], keys_in[i], n[i] * w, cudaMemcpyHostToDevice, r.xfer);
        cudaEventRecord(r.loaded[k], r.xfer);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = fail(EVOSORT_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
        }
    };
    upload(0);
    for (size_t j = 0; j < order.size() && st == EVOSORT_OK; ++j) {
        const size_t i = order[j];
        const int k = (int)(j % kSlots);
        // sort array j on the caller's stream once it is on the device
        evosort_params pi = base;
        if (plan_each) {
            const int cls = classify_host(keys_in[i], n[i], dt);
            evosort_params tp;
            if (table_lookup(dt, n[i], cls, &tp)) {
                pi = tp;
                pi.workspace = base.workspace;
                pi.workspace_bytes = base.workspace_bytes;
            } else {
                pi.algo = EVOSORT_ALGO_RADIX;
            }
            pi.stream = base.stream;
        }
        cudaStreamWaitEvent(s, r.loaded[k], 0);
        st = evosort_sort(slot[k], n[i], dt, &pi);
        cudaEventRecord(r.sorted[k], s);
        if (st != EVOSORT_OK) break;
        // the next upload goes first (its slot's previous download is
        // already on the copy stream), then this array's download
        if (j + 1 < order.size()) upload(j + 1);
        cudaStreamWaitEvent(r.xfer, r.sorted[k], 0);
        cudaError_t e = cudaMemcpyAsync(keys_out[i], slot[k], n[i] * w, cudaMemcpyDeviceToHost, r.xfer);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = fail(EVOSORT_ERR_CUDA, std::string("download: ") + cudaGetErrorString(e));
        }
    }
    // the caller's stream waits for the copy stream, then returns the slots
    cudaEventRecord(r.ev_xfer_done, r.xfer);
    cudaStreamWaitEvent(s, r.ev_xfer_done, 0);
    for (int j = 0; j < nslots; ++j) cudaFreeAsync(slot[j], s);
    return st;
}
