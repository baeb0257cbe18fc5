/*
 * evosort.h — C ABI of the GB300 (sm_103a) sort library.
 *
 * The library sorts fixed-width keys on one GPU.  Its computation is the one
 * EvoSort (arXiv 2505.18681) tunes: a block-based LSD radix sort (Section 3.1;
 * Algorithms 4a/4b: sign flip, per-block digit histograms, prefix sums over the
 * digit counts, stable scatter, one pass per digit) and a bottom-up mergesort
 * whose base runs are insertion-sorted below a threshold and then merged
 * pairwise (Algorithm 3), chosen per call by the dispatcher of Algorithm 5
 * (AdaptivePartitionSort) with parameters found by the genetic algorithm of
 * Algorithm 2 (RunGATuning).
 *
 * Conventions for every entry point:
 *  - Key and value pointers are DEVICE pointers owned by the caller.  Inputs
 *    are read, outputs written; nothing is freed or retained after return.
 *  - Work is enqueued asynchronously on params->stream (a cudaStream_t; NULL
 *    means the legacy default stream).  A call returns once its kernels are
 *    enqueued; results are ready when the stream reaches that point.
 *  - params == NULL means: tuned table entry for (dtype, size, sampled
 *    distribution class) if a table is loaded, else the built-in defaults.
 *  - Scratch memory: params->workspace / workspace_bytes if given (at least
 *    evosort_workspace_bytes() bytes, 256-byte aligned), else the library
 *    takes it from the device's stream-ordered memory pool and returns it to
 *    the pool on the same stream.
 *  - Errors are returned as evosort_status; a message for the calling thread
 *    is available from evosort_last_error().  Nothing is thrown across the ABI.
 *    Errors found on the device (a bounded wait that ran out) are recorded in
 *    a device status word and returned by the next evosort_sync().
 *  - n == 0 returns EVOSORT_OK without touching the device.
 *  - Devices: a call works on the device current in the calling thread.  The
 *    kernels' shared-memory limits and occupancy are set up once per process,
 *    on the first device a kernel runs on; a process that drives several GPUs
 *    may get EVOSORT_ERR_CUDA from the launches of kernels with large shared
 *    tiles on the others.  Use one process per GPU (as the multi-GPU sorts do).
 *
 * Total order of keys (the paper sorts signed integers and flips the sign bit
 * before the passes and back after, Algorithms 4a/4b):
 *  - signed integers: two's-complement numeric order;
 *  - unsigned integers: numeric order;
 *  - floats (the paper has none; this library's reading): -inf < negatives <
 *    -0.0 < +0.0 < positives < +inf < positive NaNs (ascending payload) <
 *    negative NaNs (descending payload).  Every bit pattern is kept, so NaN
 *    payloads and the sign of zero survive the sort.
 * Every sort is stable: keys that compare equal keep their input order, which
 * for key/value sorts makes the value order unique.
 */
#ifndef EVOSORT_H
#define EVOSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EVOSORT_I32 = 0,
    EVOSORT_I64 = 1,
    EVOSORT_U32 = 2,
    EVOSORT_U64 = 3,
    EVOSORT_F32 = 4,
    EVOSORT_F64 = 5
} evosort_dtype;

typedef enum {
    EVOSORT_OK = 0,
    EVOSORT_ERR_INVALID = 1,     /* bad argument (null pointer, dtype, params, offsets) */
    EVOSORT_ERR_NOMEM = 2,       /* device memory or caller workspace too small */
    EVOSORT_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    EVOSORT_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out */
    EVOSORT_ERR_UNSUPPORTED = 5  /* valid request the library cannot serve */
} evosort_status;

/* Algorithm choice, the A_code gene of Section 4.2 (3 = mergesort, 4 = radix). */
typedef enum {
    EVOSORT_ALGO_AUTO = -1,      /* tuned table, else radix */
    EVOSORT_ALGO_RADIX = 0,      /* LSD radix sort, Algorithms 4a/4b */
    EVOSORT_ALGO_MERGE = 1       /* bottom-up mergesort, Algorithm 3 */
} evosort_algo;

/* Tunable parameters.  Zero means "default" for every integer field. */
typedef struct {
    int algo;                 /* evosort_algo */
    int digit_bits;           /* radix digit width d, 4..11 (default 8); the
                                 paper fixes d = 8 (one byte per pass) */
    int keys_per_thread;      /* keys each thread holds in a tile (8, 16 or 32) */
    int block_size;           /* threads per CTA: 256, 512 or 1024; the default
                                 radix tile is the largest of a preference list
                                 that fits shared memory and gives at least
                                 half of the SMs a tile */
    int insertion_threshold;  /* mergesort base-run length T_insertion, 2..2048
                                 (default 32; Section 4.2 bounds); the one-CTA
                                 small-array path caps its runs at 16 keys */
    int rank_mode;            /* radix tile ranking (how a warp finds lanes with
                                 equal digits): 1 = match.any (d = 8 only),
                                 2 = one ballot per digit bit (any d),
                                 3 = shared-memory match masks (d <= 8),
                                 4 = adaptive (d = 8; default): per pass,
                                     match.any when the pass's digit is
                                     concentrated (sum of squared digit
                                     shares above 1/32, or above 1/4 for the
                                     first pass to run), else match masks;
                                     sorts below 2^21 keys use match masks
                                     only */
    int seg_block_cap;        /* segmented sort: segments up to this many keys are
                                 sorted by one CTA in shared memory, longer ones by
                                 a CTA-local radix sort; 256..8192 (32-bit keys),
                                 256..4096 (64-bit keys); default the maximum */
    void* stream;             /* cudaStream_t */
    void* workspace;          /* optional caller scratch, device, 256-B aligned */
    size_t workspace_bytes;
    int descending;           /* nonzero: non-increasing order (stable: equal keys,
                                 and the values moving with them, keep their input
                                 order); default 0, ascending */
    int pass_kernel;          /* radix pass kernel: 0 = default (the register tile
                                 where it is compiled for the request, else the
                                 staged tile), 1 = staged tile (the tile is copied
                                 into shared memory by the TMA engine and ranked
                                 there), 2 = register tile (keys loaded into
                                 registers and ranked one column of 32 at a time;
                                 8-bit digits, rank modes 1, 3 and 4) */
    int adapt_later;          /* adaptive ranking (rank mode 4): a pass after the
                                 first one that runs uses match.any when the sum
                                 of its squared digit shares exceeds
                                 2^-adapt_later; 1..10, default 5 (1/32) */
    int adapt_first;          /* the same threshold for the first pass that
                                 runs, which sees the input order; 1..10,
                                 default 2 (1/4) */
    int seg_warp_cap;         /* segmented sort: segments shorter than this are
                                 sorted by one warp in registers; 32, 64, 128 or
                                 256 (default 256) */
    int small_cap;            /* lone arrays of at most this many keys are sorted
                                 by one CTA in shared memory in a single launch
                                 with no scratch memory (the GPU form of the
                                 paper's small-array fallback, Algorithm 5);
                                 0 = default: 4096 when algo is AUTO, else off;
                                 1 = off; 2..8192 = that cut-over, whatever the
                                 algo */
    long long seg_giant;      /* segmented sort: segments longer than this many
                                 keys are sorted one by one by the device-wide
                                 radix path; finding them costs one small
                                 synchronous read of the length histogram, so it
                                 is skipped while the stream is being captured
                                 into a CUDA graph; 0 = default (2^24), -1 =
                                 never */
} evosort_params;

/* Fills *p with the built-in defaults (radix, d = 8, no workspace, NULL stream).
 * d = 8 is the paper's fixed digit (one byte per pass, Algorithms 4a/4b); the
 * other defaults are the GA's winners on this GPU (Algorithm 2). */
void evosort_default_params(evosort_params* p);

/* Bytes of scratch one call needs for n keys of dtype dt (with_values != 0 for
 * key/value sorts) under params p (NULL = defaults): the temporary array the
 * passes of Algorithms 4a/4b (or the merge rounds of Algorithm 3) write into,
 * plus the digit counts and look-back slots.  The paper allocates these inside
 * the sort; here a caller may supply them.  Host only; 0 for bad params. */
size_t evosort_workspace_bytes(size_t n, evosort_dtype dt, int with_values,
                               const evosort_params* p);

/* The parameters a sort of n keys of dtype dt (with values if with_values)
 * would run with under params p (NULL = defaults), every default resolved:
 * algorithm, pass kernel, tile shape (with n known the default tile follows
 * the closed form fitted to the tuned tables over log10 n, guarded so that
 * small inputs still give half of the SMs a tile), ranking, thresholds.  The
 * dispatcher's table is not consulted (that needs the keys: evosort_plan), and
 * neither are the decisions taken from the data (the few-values and ordered
 * paths, range reduction).  Host only.  The paper has no counterpart: its
 * parameters are the GA genome of Section 4.2, fixed per run. */
evosort_status evosort_resolve(size_t n, evosort_dtype dt, int with_values, const evosort_params* p,
                               evosort_params* out);

/* Sorts keys[0..n) in place (AdaptivePartitionSort, Algorithm 5).
 * keys: device array of n elements of dtype dt.
 * With p == NULL or p->algo AUTO: arrays of at most small_cap keys take the
 * one-CTA path; otherwise, when a tuned table is loaded, the dispatcher reads
 * a 4096-key strided sample back to the host (synchronising p->stream) and
 * takes the table's entry for the sample's class, and two data-dependent
 * paths come first (keys of at least 2^16 elements): a sample with at most
 * 64 distinct keys is sorted by counting over those values (keys only), and
 * a sample in order (or in reverse order, keys only) by one checked copy;
 * each reads one small result back and falls back to the radix sort when a
 * key proves the sample wrong.  Such AUTO calls cannot be captured into a
 * CUDA graph; calls with explicit parameters (or no table) stay
 * asynchronous.  In every radix sort the passes rank key - min when the
 * keys' span needs fewer 8-bit digits than their raw digits that vary (a
 * decision taken on the device).  Whatever the path, the result is the one
 * sorted array. */
evosort_status evosort_sort(void* keys, size_t n, evosort_dtype dt, const evosort_params* p);

/* Out-of-place variant of evosort_sort (Algorithm 5 with the same paths):
 * reads keys_in, writes the sorted keys to keys_out.  keys_in is left unchanged.  keys_in == keys_out is the in-place sort; any
 * other overlap is an error. */
evosort_status evosort_sort_to(const void* keys_in, void* keys_out, size_t n, evosort_dtype dt,
                               const evosort_params* p);

/* Stable key/value sort in place: values[i] travels with keys[i]; among equal
 * keys the input order of the values is kept (argsort when values are
 * 0..n-1).  values: device array of n uint32.  The paper sorts keys alone; the
 * stable placement of Algorithms 4a/4b (and the left-first merge of
 * Algorithm 3) carries the value with its key. */
evosort_status evosort_sort_pairs(void* keys, uint32_t* values, size_t n, evosort_dtype dt,
                                  const evosort_params* p);

/* Out-of-place key/value sort (as evosort_sort_pairs: the stable placement of
 * Algorithms 4a/4b, or Algorithm 3, carrying each value with its key); the
 * inputs are left unchanged.  keys_in == keys_out with values_in == values_out is the in-place
 * sort; keys and values must be both in place or both out of place, and an
 * input that partly overlaps its own output is an error. */
evosort_status evosort_sort_pairs_to(const void* keys_in, const uint32_t* values_in, void* keys_out,
                                     uint32_t* values_out, size_t n, evosort_dtype dt,
                                     const evosort_params* p);

/* Sorts `count` arrays that live in HOST memory (the paper's sort of an
 * array handed over by the caller, Algorithm 5, with the transfers to and
 * from the GPU included).  Array i has n[i] keys of dtype dt at keys_in[i];
 * its sorted keys go to keys_out[i] (== keys_in[i] for in place; any other
 * overlap between an input and an output is an error).  Each array is copied
 * to the device, sorted there by the device path with params p (AUTO and a
 * non-empty table: the dispatcher's parameters for that array, classified
 * from a strided sample read on the host when the call is made, so the input
 * must already hold its keys then), and copied back.  The copies of
 * array i+1 to the device and of array i-1 back to the host run on two
 * internal streams while array i is sorted on p->stream, through three
 * device slots of max(n[i]) keys allocated from the stream-ordered pool for
 * the call.  The whole batch is ordered after earlier work on p->stream, and
 * later work on p->stream waits for all of it: evosort_sync(p->stream) or a
 * stream synchronisation makes the host outputs ready.  Host buffers should
 * be page-locked (cudaHostAlloc / cudaHostRegister): pageable buffers are
 * still sorted correctly, but the CUDA driver then stages each copy and the
 * overlap is lost.  n[i] == 0 arrays are skipped.  Errors before anything is
 * enqueued (bad arguments, no device memory) return a status; a failure of a
 * later array's sort returns its status with the earlier arrays' work left
 * enqueued. */
evosort_status evosort_sort_host_batch(const void* const* keys_in, void* const* keys_out, const size_t* n,
                                       size_t count, evosort_dtype dt, const evosort_params* p);

/* Batched segmented sort: sorts each segment keys[offsets[i] .. offsets[i+1])
 * independently, in place, for i in [0, nseg), in one persistent launch
 * (after three small list-building kernels).  Short segments are sorted by
 * one warp in registers, medium ones by one CTA in shared memory, long ones
 * by a CTA-local LSD radix sort (Algorithms 4a/4b) over global memory.
 *   keys    DEVICE array of total keys of dtype dt
 *   total   number of keys, which must equal offsets[nseg]
 *   offsets DEVICE array of nseg + 1 uint64: offsets[0] == 0, non-decreasing,
 *           offsets[nseg] == total; empty segments are allowed.
 * Keys never cross a segment boundary.  Equal keys are identical bit patterns,
 * so the result is unique although the warp tier is not a stable network.
 * The offsets are checked on the device; a violation is reported by the next
 * evosort_sync() as EVOSORT_ERR_INVALID (keys in segments that were processed
 * may then have been sorted).  Segments longer than 2^32 keys are not
 * supported. */
evosort_status evosort_segmented_sort(void* keys, size_t total, const uint64_t* offsets, size_t nseg,
                                      evosort_dtype dt, const evosort_params* p);

/* Scratch bytes evosort_segmented_sort needs for total keys in nseg segments
 * (its work list and one key buffer of total keys; not in the paper). */
size_t evosort_segmented_workspace_bytes(size_t total, size_t nseg, evosort_dtype dt);

/* ---- Per-rank steps of a multi-GPU sort of one array ---------------------
 * Not in the paper (it names an MPI extension as future work).  Each rank
 * holds a slice of the keys; the ranks agree on the part of the key range
 * each owns from the slices' key ranges and range histograms (reduced over
 * the ranks by the caller), exchange keys, and sort what they receive.
 * Keys are compared in the order-preserving key space of dt (descending:
 * that order reversed); "mapped" values below are keys in that space,
 * zero-extended to 64 bits.  Asynchronous on stream (NULL: legacy default).
 *
 * evosort_key_range: range[0] = the smallest, range[1] = the largest mapped
 * key of keys[0..n) (DEVICE array of 2 words, overwritten; n = 0 leaves
 * range[0] = 2^64 - 1 and range[1] = 0). */
evosort_status evosort_key_range(const void* keys, size_t n, evosort_dtype dt, int descending,
                                 unsigned long long* range, void* stream);

/* evosort_range_histogram: adds to counts[b] (DEVICE array of nbins words,
 * not cleared) the number of keys with (mapped key - base) >> shift == b,
 * a value at or above nbins counting in bin nbins - 1.  nbins 1..8192,
 * 0 <= shift < key bits.  With base the smallest key over all ranks and
 * shift making (largest - base) >> shift < nbins, the bins split the whole
 * range into nbins ordered parts. */
evosort_status evosort_range_histogram(const void* keys, size_t n, evosort_dtype dt, int descending,
                                       unsigned long long base, int shift, int nbins, unsigned long long* counts,
                                       void* stream);

/* ---- Dispatcher and tuned table (Algorithm 5, AdaptivePartitionSort) ----
 * With params == NULL or params->algo == EVOSORT_ALGO_AUTO and a non-empty
 * table, a sort call classifies its input from a strided sample of 4096 keys
 * (one small synchronous device-to-host copy on the call's stream) and uses
 * the table entry for (dtype, size bucket = floor(log2 n), class): the nearest
 * bucket of the same class, else of the RANDOM class, else the defaults.  The
 * caller's stream and workspace are kept.  With an empty table nothing is
 * sampled and the defaults are used. */
typedef enum {
    EVOSORT_CLASS_RANDOM = 0,    /* no structure found */
    EVOSORT_CLASS_SKEWED = 1,    /* over a quarter of the keys share the top byte */
    EVOSORT_CLASS_NARROW = 2,    /* at most half of the key bits vary (more than 16) */
    EVOSORT_CLASS_FEW = 3,       /* at most 64 distinct values in the sample */
    EVOSORT_CLASS_SORTED = 4,    /* >= 90% of the unequal sampled neighbours rise */
    EVOSORT_CLASS_REVERSE = 5,   /* >= 90% of the unequal sampled neighbours fall */
    EVOSORT_CLASS_CONSTANT = 6,  /* one value */
    EVOSORT_CLASS_NARROW16 = 7,  /* at most 16 key bits vary */
    EVOSORT_CLASS_SEGMENTED = 8  /* table entries for batched segmented sorts,
                                    keyed by the batch's total key count; used
                                    by evosort_segmented_sort when params is
                                    NULL or params->algo is AUTO (no sample is
                                    read) */
} evosort_dist_class;

/* Class of keys[0..n) from a strided sample (synchronises the stream). */
evosort_status evosort_classify(const void* keys, size_t n, evosort_dtype dt, void* stream, int* cls);

/* Parameters the dispatcher would use for these keys; *cls receives the class
 * (may be NULL).  Synchronises the stream when the table is not empty. */
evosort_status evosort_plan(const void* keys, size_t n, evosort_dtype dt, void* stream, evosort_params* out,
                            int* cls);

/* The same plan for keys in HOST memory: the strided sample is read directly
 * on the host (no CUDA call, no synchronisation), so a caller that holds a
 * host copy (a serving loop, a host batch) can plan a sort before its upload.
 * descending != 0 reads the class in the order of a descending sort.  The
 * returned stream and workspace are NULL. */
evosort_status evosort_plan_host(const void* keys, size_t n, evosort_dtype dt, int descending,
                                 evosort_params* out, int* cls);

/* Table of tuned parameters: set one entry (ms = its measured time, kept for
 * reference), clear, count, save to / load from a text file (one entry per
 * line: dtype size_bucket class algo digit_bits block_size keys_per_thread
 * rank_mode insertion_threshold seg_block_cap ms; '#' starts a comment). */
evosort_status evosort_table_set(evosort_dtype dt, int size_bucket, int cls, const evosort_params* p, float ms);
void evosort_table_clear(void);
size_t evosort_table_size(void);
evosort_status evosort_table_save(const char* path);
evosort_status evosort_table_load(const char* path);

/* ---- Genetic-algorithm tuner (Algorithm 2, RunGATuning) ------------------
 * Evolves the parameters of one sort of `sample` (a DEVICE array of n keys of
 * dtype dt): algorithm (radix / merge, the paper's A_code), digit width,
 * radix tile shape, ranking variant and insertion threshold.  Fitness is the
 * median CUDA-event time of `reps` sorts; every genome's output is checked
 * first, against `expected` bit for bit when given (a DEVICE array holding the
 * sorted sample), else for sortedness and an order-free multiset fingerprint
 * of the input; a failing genome gets +infinity.  The defaults genome is in
 * the first generation, so the result is never slower than the defaults on
 * the sample.  Writes the best genome's parameters to *best (stream set to
 * `stream`), its time to *best_ms, and per generation best / mean / worst
 * times to log[0 .. min(generations, log_cap)).  Allocates an output buffer
 * of n keys from the stream-ordered pool; synchronises the stream. */
typedef struct {
    int population;          /* 30 (Section 4.2) */
    int generations;         /* 10 */
    double crossover_p;      /* 0.7: uniform crossover per parent pair */
    double mutation_p;       /* 0.3: uniform mutation per individual */
    double gene_mutation_p;  /* 0.2: each gene redrawn when mutating */
    int elite;               /* 2: best genomes copied unchanged */
    int tournament;          /* 3: tournament size of parent selection */
    int reps;                /* 3: timings per genome (median) */
    int tins_init_max;       /* 256: first-generation insertion threshold bound */
    int allow_merge;         /* 1: the algorithm gene may pick mergesort */
    uint64_t seed;           /* 42 */
    int mode;                /* 0: genomes for the sort of one array (algorithm,
                                digit width, pass kernel, tile shape, ranking,
                                adaptive-ranking thresholds, insertion threshold,
                                small-array cut-over); 1: genomes for a batched
                                segmented sort (warp-tier, block-tier and giant
                                cut-overs, insertion threshold).  evosort_tune
                                sets 0. */
    uint64_t sample_keys;    /* keys of the array being tuned (mode 0; 0 =
                                unknown): genomes whose small-array cut-over is
                                at or above it all take the one-CTA path and
                                share one evaluation */
} evosort_ga_config;

typedef struct {
    int generation;
    float best_ms, mean_ms, worst_ms;  /* over the genomes with a finite time */
    int evaluations;                   /* distinct genomes timed so far */
    evosort_params best;               /* best genome of the generation */
} evosort_ga_log;

void evosort_default_ga_config(evosort_ga_config* c);

/* The GA loop alone, with the fitness supplied by the caller: fitness(p,
 * best_so_far_ms (or -1 if none yet), ctx) returns the genome's time in ms,
 * or a negative value for a failed genome.  evosort_tune runs it with a
 * fitness that times the sort on the device; key_bytes (4 or 8) selects the
 * default genome seeded into the first generation.  Deterministic for a given
 * seed and fitness function. */
typedef float (*evosort_fitness_fn)(const evosort_params* p, float best_so_far_ms, void* ctx);
evosort_status evosort_ga_search(const evosort_ga_config* cfg, int key_bytes, evosort_fitness_fn fitness,
                                 void* ctx, evosort_params* best, float* best_ms, evosort_ga_log* log,
                                 int log_cap);
evosort_status evosort_tune(const void* sample, size_t n, evosort_dtype dt, const void* expected,
                            const evosort_ga_config* cfg, void* stream, evosort_params* best, float* best_ms,
                            evosort_ga_log* log, int log_cap);

/* Keys-only sort that allocates no memory (the paper has no counterpart).
 * For callers that may not allocate device memory where they sort: code
 * running inside another framework's execute callback (a server plugin or a
 * custom operator) whose host framework owns all device memory and forbids
 * allocation calls, or latency-critical loops that must not block in the
 * allocator.  The result is the one evosort_sort_to gives with default
 * parameters, and the kernels and tile shape are the ones it picks for n
 * keys.  keys_in/keys_out: DEVICE arrays of n keys of dtype dt; they may be
 * equal (in place) but must not otherwise overlap.  stream: cudaStream_t
 * (NULL = legacy default stream).
 * Scratch: a fixed 64 MiB buffer inside the library's device image, reserved
 * on each device the first time this entry point runs there (or when the
 * library's module is loaded, if the CUDA runtime's lazy loading is off) and
 * held until the process exits.  Sizes whose scratch exceeds it (above about
 * 7.7 million 64-bit or 14.9 million 32-bit keys) are rejected with
 * EVOSORT_ERR_INVALID before anything is launched.
 * The first call on each device looks up the buffer's device address (once,
 * with that device current); make that first call before any stream capture.
 * Every call on a device shares the one buffer: calls whose work overlaps on
 * the GPU (different streams, or another thread) race and corrupt each other;
 * order them on one stream.  The buffer keeps the last call's contents; the
 * sort clears what it needs cleared itself. */
evosort_status evosort_sort_noalloc(const void* keys_in, void* keys_out, size_t n, evosort_dtype dt,
                                    void* stream);

/* Waits for params-stream work (stream = NULL: the legacy default stream) and
 * returns the first error recorded on the device since the last call
 * (EVOSORT_ERR_TIMEOUT for a bounded wait that ran out; EVOSORT_ERR_CUDA when a
 * radix scatter offset fell outside the array, whose stores the kernel skips;
 * EVOSORT_ERR_INVALID for bad segment offsets), then clears it. */
evosort_status evosort_sync(void* stream);

/* Returns the scratch memory the library holds on the current device to the
 * CUDA driver.  Sorts that allocate their own scratch take it from the
 * device's stream-ordered pool (cudaMallocAsync), which the library sets to
 * keep freed memory reserved so that repeated sorts do not pay for driver
 * allocations; after one sort of 1e9 64-bit keys about 8.7 GB stays reserved.
 * This call waits for all work on the device (cudaDeviceSynchronize), then
 * trims that pool to zero bytes; memory still backing an allocation in use by
 * another stream-ordered user of the same pool is kept.  Later sorts reserve
 * again.  The fixed buffer of evosort_sort_noalloc is not affected.  Not in
 * the paper (host memory needs no such call there). */
evosort_status evosort_release(void);

/* Poll limit of the bounded device-side waits on look-back slots, for tests
 * of the failure path and for debugging (the paper has no counterpart).
 * polls == 0 restores the built-in limit (2^22 polls, about a second).  A
 * wait that runs out records EVOSORT_ERR_TIMEOUT for the next evosort_sync
 * and its kernel returns; that sort's output is then invalid.  Applies to
 * sorts enqueued after the call, process-wide. */
void evosort_set_wait_limit(uint32_t polls);

/* Message describing the calling thread's last error ("" if none). */
const char* evosort_last_error(void);

/* ---- Instrumentation --------------------------------------------------
 * While enabled, the library records a CUDA event pair on the call's stream
 * around every kernel it launches.  evosort_profile_read() waits for the
 * recorded events, fills up to cap records (oldest first), clears the list and
 * returns how many records there were.  "bytes" is the launch's algorithmic
 * traffic (keys and values read plus written); it is 0 for a radix pass whose
 * digit was constant (skipped on the device) and for a copy that was not
 * needed.  Events add a few microseconds per launch; leave this off outside
 * measurements.  Not in the paper (it times whole sorts, Section 5): this is
 * how the roofline of each kernel is measured. */
typedef enum {
    EVOSORT_K_RADIX_HISTOGRAM = 0,   /* all-digit histogram (one key read) */
    EVOSORT_K_RADIX_SCAN = 1,        /* digit-count prefix sums + pass plan */
    EVOSORT_K_RADIX_ONESWEEP = 2,    /* one stable scatter pass */
    EVOSORT_K_RADIX_FIXUP = 3,       /* copy into the output buffer */
    EVOSORT_K_MERGE_BLOCK = 4,       /* insertion-sorted runs merged in a tile */
    EVOSORT_K_MERGE_PARTITION = 5,   /* merge-path split points */
    EVOSORT_K_MERGE_PASS = 6,        /* one pairwise merge round */
    EVOSORT_K_SEGMENTED = 7,         /* batched segmented sort kernels */
    EVOSORT_K_SMALL = 8,             /* one-CTA shared-memory sort of a small array */
    EVOSORT_K_DICT = 9,              /* few distinct keys: count (pass 0) and fill (pass 1) */
    EVOSORT_K_ORDERED = 10,          /* input in order: checked copy (pass 0), check (1), reversed copy (2) */
    EVOSORT_K_RADIX_COUNT = 11       /* narrow key range: value count and fill (both launches in one record) */
} evosort_kernel_kind;

typedef struct {
    int kind;        /* evosort_kernel_kind */
    int pass;        /* radix pass or merge round, -1 if none */
    int active;      /* 0 if the kernel found nothing to do */
    float ms;        /* device time between the events around the launch */
    double bytes;    /* algorithmic bytes moved by the launch */
    uint64_t items;  /* keys the launch covers */
    int rank;        /* radix pass under adaptive ranking: the ranking variant
                        of this launch (1 or 3); 0 otherwise */
} evosort_kernel_record;

evosort_status evosort_profile(int enable);
size_t evosort_profile_read(evosort_kernel_record* out, size_t cap);

/* Number of kernels this library has launched in this process (all threads). */
uint64_t evosort_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* EVOSORT_H */
