/*
 * EvoSort CPU oracle — TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded C that computes what the GPU sort path
 * computes.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load this library; the product path never does, and this
 * file shares no code, header, table or constant with the CUDA sources.
 *
 * What is computed (the result has a plain definition, so every algorithm
 * here must reach exactly the same bits):
 *   - keys only:  the non-decreasing rearrangement of the input under the
 *                 total order "prec" defined by ordered_bits() below;
 *   - key/value:  the stable sort of the pairs (key[j], value[j]) by key, ties
 *                 kept in input order (the paper asks for output identical to
 *                 np.sort and for stability where it applies, Section
 *                 "Experimental Setup", validation methodology);
 *   - segmented:  the keys-only sort applied to each [off[i], off[i+1]).
 *
 * Two independent algorithms reach it:
 *   O1  oracle_radix_sort  — LSD radix sort with 8-bit digits, as in
 *       Algorithms 4a/4b (RefinedParallelRadixSort_int32 / _int64): flip to
 *       the unsigned domain, one counting pass per byte (histogram, exclusive
 *       prefix sum, stable placement into a temporary array, swap), flip back.
 *       The paper's per-thread histograms collapse to one histogram because
 *       this oracle runs on one thread.
 *   O2  oracle_merge_sort  — bottom-up mergesort as in Algorithm 3
 *       (RefinedParallelMergeSort): insertion sort of chunks of chunkSize,
 *       then pairwise merges of runs of currSize, doubling until currSize >= n.
 *       A run without a partner is carried to the next round unchanged.
 *
 * Total order (the paper sorts integers only; Section 3.1 and Algorithms
 * 4a/4b flip the sign bit of signed integers).  For floats this oracle uses
 * the reading: -inf < negatives < -0.0 < +0.0 < positives < +inf < positive
 * NaNs (ascending payload) < negative NaNs (descending payload).  It is reached
 * by mapping the IEEE bits u to t = sign ? ~u : u ^ signbit and then rotating
 * t down by (2^m - 1) modulo 2^w, where m is the mantissa width (23 or 52),
 * which moves the NaN blocks above +inf.  The map is a bijection, so NaN
 * payloads survive the sort.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* dtype codes of this oracle (its own numbering, set by its Python loader) */
enum { OR_I32 = 0, OR_I64 = 1, OR_U32 = 2, OR_U64 = 3, OR_F32 = 4, OR_F64 = 5 };

/* Fault switch used only by the self-tests that show the pins catch a wrong
 * oracle: 0 = correct; 1 = no sign flip; 2 = unstable (reverse) placement in
 * one pass; 3 = last digit pass dropped; 4 = merge takes the right run on ties;
 * 5 = float NaN rotation dropped. */
static int g_fault = 0;
void oracle_set_fault(int f) { g_fault = f; }

static int key_bytes(int dt) {
    return (dt == OR_I32 || dt == OR_U32 || dt == OR_F32) ? 4 : 8;
}

/* Map the raw bits of one key to an unsigned integer whose numeric order is
 * the total order "prec" on keys of dtype dt. */
static uint64_t ordered_bits(uint64_t u, int dt) {
    switch (dt) {
    case OR_I32:
        return g_fault == 1 ? u : (u ^ 0x80000000u);          /* Alg. 4a, XOR */
    case OR_I64:
        return g_fault == 1 ? u : (u ^ 0x8000000000000000ull); /* Alg. 4b, XOR */
    case OR_U32:
    case OR_U64:
        return u;
    case OR_F32: {
        uint32_t x = (uint32_t)u;
        uint32_t t = (x >> 31) ? ~x : (x ^ 0x80000000u);
        if (g_fault != 5) t = t - 0x007FFFFFu;                 /* NaNs after +inf */
        return t;
    }
    case OR_F64: {
        uint64_t t = (u >> 63) ? ~u : (u ^ 0x8000000000000000ull);
        if (g_fault != 5) t = t - 0x000FFFFFFFFFFFFFull;
        return t;
    }
    }
    return u;
}

/* Inverse of ordered_bits. */
static uint64_t raw_bits(uint64_t t, int dt) {
    switch (dt) {
    case OR_I32:
        return g_fault == 1 ? t : (t ^ 0x80000000u);
    case OR_I64:
        return g_fault == 1 ? t : (t ^ 0x8000000000000000ull);
    case OR_U32:
    case OR_U64:
        return t;
    case OR_F32: {
        uint32_t x = (uint32_t)t;
        if (g_fault != 5) x = x + 0x007FFFFFu;
        return (x >> 31) ? (x ^ 0x80000000u) : ~x;
    }
    case OR_F64: {
        uint64_t x = t;
        if (g_fault != 5) x = x + 0x000FFFFFFFFFFFFFull;
        return (x >> 63) ? (x ^ 0x8000000000000000ull) : ~x;
    }
    }
    return t;
}

static uint64_t load_bits(const void* p, size_t i, int w) {
    if (w == 4) return ((const uint32_t*)p)[i];
    return ((const uint64_t*)p)[i];
}

static void store_bits(void* p, size_t i, int w, uint64_t v) {
    if (w == 4) ((uint32_t*)p)[i] = (uint32_t)v;
    else ((uint64_t*)p)[i] = v;
}

/* Exposed so the tests can check the map itself against the float order. */
uint64_t oracle_ordered_bits(uint64_t raw, int dt) { return ordered_bits(raw, dt); }

/* ---------------------------------------------------------------------------
 * O1: LSD radix sort, 8-bit digits (Algorithms 4a and 4b).
 * keys_in/vals_in are read, keys_out/vals_out receive the sorted result
 * (vals may be NULL).  In and out may alias.  Returns 0, or -1 on allocation
 * failure.
 * ------------------------------------------------------------------------- */
int oracle_radix_sort(const void* keys_in, const uint32_t* vals_in, size_t n, int dt,
                      void* keys_out, uint32_t* vals_out) {
    const int w = key_bytes(dt);
    if (n == 0) return 0;
    uint64_t* a = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint64_t* tmp = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint32_t* va = NULL;
    uint32_t* vtmp = NULL;
    if (vals_in) {
        va = (uint32_t*)malloc(n * sizeof(uint32_t));
        vtmp = (uint32_t*)malloc(n * sizeof(uint32_t));
    }
    if (!a || !tmp || (vals_in && (!va || !vtmp))) {
        free(a); free(tmp); free(va); free(vtmp);
        return -1;
    }
    /* step 1: flip every key into the unsigned domain */
    for (size_t i = 0; i < n; ++i) a[i] = ordered_bits(load_bits(keys_in, i, w), dt);
    if (vals_in) memcpy(va, vals_in, n * sizeof(uint32_t));

    int passes = w;                       /* 4 passes for 32-bit, 8 for 64-bit */
    if (g_fault == 3) passes -= 1;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        size_t count[256];
        memset(count, 0, sizeof(count));
        /* histogram of this byte */
        for (size_t i = 0; i < n; ++i) count[(a[i] >> shift) & 0xFF] += 1;
        /* exclusive prefix sum: first output slot of each digit */
        size_t offset[256];
        size_t run = 0;
        for (int b = 0; b < 256; ++b) { offset[b] = run; run += count[b]; }
        /* stable placement into the temporary array, in input order */
        if (g_fault == 2 && pass == 1) {
            for (int b = 0; b < 256; ++b) offset[b] += count[b];
            for (size_t i = 0; i < n; ++i) {
                size_t b = (a[i] >> shift) & 0xFF;
                size_t dst = --offset[b];   /* reverses equal digits: unstable */
                tmp[dst] = a[i];
                if (va) vtmp[dst] = va[i];
            }
        } else {
            for (size_t i = 0; i < n; ++i) {
                size_t b = (a[i] >> shift) & 0xFF;
                size_t dst = offset[b]++;
                tmp[dst] = a[i];
                if (va) vtmp[dst] = va[i];
            }
        }
        /* swap input and temporary array */
        uint64_t* s = a; a = tmp; tmp = s;
        if (va) { uint32_t* t = va; va = vtmp; vtmp = t; }
    }
    /* last step: flip back */
    for (size_t i = 0; i < n; ++i) store_bits(keys_out, i, w, raw_bits(a[i], dt));
    if (vals_out) memcpy(vals_out, va, n * sizeof(uint32_t));
    free(a); free(tmp); free(va); free(vtmp);
    return 0;
}

/* ---------------------------------------------------------------------------
 * O2: bottom-up mergesort with insertion-sorted base chunks (Algorithm 3).
 * chunk_size is chunkSize (the insertion threshold), >= 1.
 * ------------------------------------------------------------------------- */
static int takes_right(uint64_t left, uint64_t right) {
    /* stable merge: the right run wins only when strictly smaller */
    if (g_fault == 4) return right <= left;
    return right < left;
}

int oracle_merge_sort(const void* keys_in, const uint32_t* vals_in, size_t n, int dt,
                      size_t chunk_size, void* keys_out, uint32_t* vals_out) {
    const int w = key_bytes(dt);
    if (n == 0) return 0;
    if (chunk_size < 1) chunk_size = 1;
    uint64_t* a = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint64_t* b = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint32_t* va = NULL;
    uint32_t* vb = NULL;
    if (vals_in) {
        va = (uint32_t*)malloc(n * sizeof(uint32_t));
        vb = (uint32_t*)malloc(n * sizeof(uint32_t));
    }
    if (!a || !b || (vals_in && (!va || !vb))) {
        free(a); free(b); free(va); free(vb);
        return -1;
    }
    for (size_t i = 0; i < n; ++i) a[i] = ordered_bits(load_bits(keys_in, i, w), dt);
    if (vals_in) memcpy(va, vals_in, n * sizeof(uint32_t));

    /* insertion sort of each chunk of chunk_size elements */
    for (size_t lo = 0; lo < n; lo += chunk_size) {
        size_t hi = lo + chunk_size < n ? lo + chunk_size : n;
        for (size_t i = lo + 1; i < hi; ++i) {
            uint64_t k = a[i];
            uint32_t v = va ? va[i] : 0;
            size_t j = i;
            while (j > lo && a[j - 1] > k) {      /* strictly greater: stable */
                a[j] = a[j - 1];
                if (va) va[j] = va[j - 1];
                --j;
            }
            a[j] = k;
            if (va) va[j] = v;
        }
    }
    /* pairwise merges, currSize doubling */
    for (size_t curr = chunk_size; curr < n; curr *= 2) {
        for (size_t lo = 0; lo < n; lo += 2 * curr) {
            size_t mid = lo + curr < n ? lo + curr : n;
            size_t hi = lo + 2 * curr < n ? lo + 2 * curr : n;
            size_t i = lo, j = mid, o = lo;
            while (i < mid && j < hi) {
                if (takes_right(a[i], a[j])) {
                    b[o] = a[j];
                    if (va) vb[o] = va[j];
                    ++j;
                } else {
                    b[o] = a[i];
                    if (va) vb[o] = va[i];
                    ++i;
                }
                ++o;
            }
            while (i < mid) { b[o] = a[i]; if (va) vb[o] = va[i]; ++i; ++o; }
            while (j < hi) { b[o] = a[j]; if (va) vb[o] = va[j]; ++j; ++o; }
        }
        uint64_t* s = a; a = b; b = s;
        if (va) { uint32_t* t = va; va = vb; vb = t; }
    }
    for (size_t i = 0; i < n; ++i) store_bits(keys_out, i, w, raw_bits(a[i], dt));
    if (vals_out) memcpy(vals_out, va, n * sizeof(uint32_t));
    free(a); free(b); free(va); free(vb);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Segmented keys-only sort: O1 applied to each segment [off[i], off[i+1]).
 * offsets holds nseg + 1 non-decreasing entries.  Returns 0, -1 on allocation
 * failure, -2 on bad offsets.
 * ------------------------------------------------------------------------- */
int oracle_segmented_sort(const void* keys_in, const uint64_t* offsets, size_t nseg, int dt,
                          void* keys_out) {
    const int w = key_bytes(dt);
    for (size_t s = 0; s < nseg; ++s)
        if (offsets[s + 1] < offsets[s]) return -2;
    const size_t total = nseg ? (size_t)offsets[nseg] : 0;
    if (keys_out != keys_in && total)
        memcpy((char*)keys_out + (size_t)offsets[0] * w, (const char*)keys_in + (size_t)offsets[0] * w,
               (total - (size_t)offsets[0]) * w);
    for (size_t s = 0; s < nseg; ++s) {
        size_t lo = (size_t)offsets[s], len = (size_t)(offsets[s + 1] - offsets[s]);
        char* p = (char*)keys_out + lo * w;
        int rc = oracle_radix_sort(p, NULL, len, dt, p, NULL);
        if (rc) return rc;
    }
    return 0;
}
