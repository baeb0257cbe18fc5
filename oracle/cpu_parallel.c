/*
 * Paper-shaped multithreaded CPU LSD radix sort — CPU BASELINE, test and
 * benchmark infrastructure only (never loaded by the GPU library).
 *
 * This is the shape of the paper's CPU radix sort (Algorithms 4a/4b,
 * RefinedParallelRadixSort): the keys are split into one contiguous chunk per
 * thread; every pass of 8 bits has each thread count the digits of its chunk
 * (per-thread histograms), then one exclusive prefix over (digit, thread) in
 * that order gives every thread its write offset per digit (the "thread-wise
 * offsets"), then each thread places its chunk, in order, into the other
 * buffer (stable), and the buffers swap.  Signed keys have their sign bit
 * flipped first and back at the end, as in the paper; float keys use the same
 * total order as the oracle (sign-magnitude flip, then a rotation by
 * 2^m - 1 that puts NaNs last).  No pass is skipped: 4 passes for 32-bit keys,
 * 8 for 64-bit keys.
 *
 * It exists to time the paper's method on the host cores of the GPU machine;
 * its output is checked against the oracle in the tests.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* dtype codes: 0 int32, 1 int64, 2 uint32, 3 uint64, 4 float32, 5 float64 */

static uint64_t to_key(uint64_t u, int dt) {
    switch (dt) {
        case 0: return (u ^ 0x80000000u) & 0xFFFFFFFFu;
        case 1: return u ^ 0x8000000000000000ull;
        case 2: return u & 0xFFFFFFFFu;
        case 3: return u;
        case 4: {
            uint32_t x = (uint32_t)u;
            uint32_t t = (x >> 31) ? ~x : (x ^ 0x80000000u);
            return (uint32_t)(t - 0x7FFFFFu);
        }
        default: {
            uint64_t t = (u >> 63) ? ~u : (u ^ 0x8000000000000000ull);
            return t - 0xFFFFFFFFFFFFFull;
        }
    }
}

static uint64_t from_key(uint64_t t, int dt) {
    switch (dt) {
        case 0: return (t ^ 0x80000000u) & 0xFFFFFFFFu;
        case 1: return t ^ 0x8000000000000000ull;
        case 2: return t & 0xFFFFFFFFu;
        case 3: return t;
        case 4: {
            uint32_t x = (uint32_t)t + 0x7FFFFFu;
            return (x >> 31) ? (x ^ 0x80000000u) : (uint32_t)~x;
        }
        default: {
            uint64_t x = t + 0xFFFFFFFFFFFFFull;
            return (x >> 63) ? (x ^ 0x8000000000000000ull) : ~x;
        }
    }
}

typedef struct {
    const unsigned char* in;
    unsigned char* out;
    uint64_t* a;
    uint64_t* b;
    size_t n;
    int dt, w, nthreads;
    size_t (*count)[256];   /* [thread][digit] */
    pthread_barrier_t bar;
    pthread_mutex_t mu;     /* start gate: workers wait until the thread */
    pthread_cond_t cv;      /* count is final */
    int go;
} job_t;

typedef struct {
    job_t* job;
    int t;
} arg_t;

static void* worker(void* p) {
    arg_t* arg = (arg_t*)p;
    job_t* j = arg->job;
    const int t = arg->t;
    pthread_mutex_lock(&j->mu);
    while (!j->go) pthread_cond_wait(&j->cv, &j->mu);
    pthread_mutex_unlock(&j->mu);
    if (t >= j->nthreads) return NULL;
    const size_t lo = j->n * (size_t)t / (size_t)j->nthreads;
    const size_t hi = j->n * (size_t)(t + 1) / (size_t)j->nthreads;
    for (size_t i = lo; i < hi; ++i) {
        uint64_t u = 0;
        memcpy(&u, j->in + i * j->w, (size_t)j->w);
        j->a[i] = to_key(u, j->dt);
    }
    uint64_t* src = j->a;
    uint64_t* dst = j->b;
    for (int pass = 0; pass < j->w; ++pass) {
        const int shift = 8 * pass;
        size_t* c = j->count[t];
        memset(c, 0, 256 * sizeof(size_t));
        for (size_t i = lo; i < hi; ++i) c[(src[i] >> shift) & 0xFF] += 1;
        pthread_barrier_wait(&j->bar);
        if (t == 0) {
            /* exclusive prefix over (digit, thread): thread t's keys of digit
               d go after every key of a smaller digit and after the keys of
               digit d of threads before t */
            size_t run = 0;
            for (int d = 0; d < 256; ++d)
                for (int q = 0; q < j->nthreads; ++q) {
                    const size_t k = j->count[q][d];
                    j->count[q][d] = run;
                    run += k;
                }
        }
        pthread_barrier_wait(&j->bar);
        for (size_t i = lo; i < hi; ++i) {
            const uint64_t k = src[i];
            dst[c[(k >> shift) & 0xFF]++] = k;
        }
        pthread_barrier_wait(&j->bar);
        uint64_t* tmp = src;
        src = dst;
        dst = tmp;
    }
    for (size_t i = lo; i < hi; ++i) {
        const uint64_t u = from_key(src[i], j->dt);
        memcpy(j->out + i * j->w, &u, (size_t)j->w);
    }
    return NULL;
}

/* Sorts n keys of dtype dt from keys_in into keys_out (they may be equal)
 * with `threads` threads (<= 0: every online CPU).  Returns the number of
 * threads used, or -1 on a bad argument or allocation failure. */
int cpu_parallel_radix_sort(const void* keys_in, void* keys_out, size_t n, int dt, int threads) {
    if (dt < 0 || dt > 5 || (n && (!keys_in || !keys_out))) return -1;
    if (threads <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        threads = c > 0 ? (int)c : 1;
    }
    if (threads > 1024) threads = 1024;
    if ((size_t)threads > n) threads = n > 0 ? (int)n : 1;
    job_t j;
    j.in = (const unsigned char*)keys_in;
    j.out = (unsigned char*)keys_out;
    j.n = n;
    j.dt = dt;
    j.w = (dt == 1 || dt == 3 || dt == 5) ? 8 : 4;
    j.nthreads = threads;
    j.a = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    j.b = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    j.count = (size_t(*)[256])malloc((size_t)threads * sizeof(*j.count));
    pthread_t* tid = (pthread_t*)malloc((size_t)threads * sizeof(pthread_t));
    arg_t* args = (arg_t*)malloc((size_t)threads * sizeof(arg_t));
    if (!j.a || !j.b || !j.count || !tid || !args) {
        free(j.a);
        free(j.b);
        free(j.count);
        free(tid);
        free(args);
        return -1;
    }
    pthread_mutex_init(&j.mu, NULL);
    pthread_cond_init(&j.cv, NULL);
    j.go = 0;
    for (int t = 0; t < threads; ++t) {
        args[t].job = &j;
        args[t].t = t;
    }
    /* threads that start wait at the gate; the sort runs with the calling
       thread plus however many started */
    int started = 1;
    while (started < threads && pthread_create(&tid[started], NULL, worker, &args[started]) == 0) ++started;
    j.nthreads = started;
    pthread_barrier_init(&j.bar, NULL, (unsigned)started);
    pthread_mutex_lock(&j.mu);
    j.go = 1;
    pthread_cond_broadcast(&j.cv);
    pthread_mutex_unlock(&j.mu);
    worker(&args[0]);
    for (int t = 1; t < started; ++t) pthread_join(tid[t], NULL);
    const int rc = started;
    pthread_barrier_destroy(&j.bar);
    pthread_cond_destroy(&j.cv);
    pthread_mutex_destroy(&j.mu);
    free(j.a);
    free(j.b);
    free(j.count);
    free(tid);
    free(args);
    return rc;
}
