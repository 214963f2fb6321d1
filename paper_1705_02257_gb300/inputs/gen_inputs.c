/*
 * Seeded synthetic input generators for the samplesort benchmarks and tests.
 *
 * This file holds no sorting-method arithmetic: it only produces the inputs
 * that both the CPU oracle and the GPU path consume.  The distributions are
 * the nine of the paper's experimental setup (Section 5): Uniform,
 * Exponential, AlmostSorted, Sorted, ReverseSorted, Ones, RootDup, TwoDup and
 * EightDup, plus the element types of the same section (64-bit keys,
 * float64 keys, key/payload pairs, 100-byte records with a 10-byte key).
 *
 * Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), used in
 * counter form: output i of the stream with seed s is mix(s + (i+1)*gamma),
 * so every element can be generated independently and in parallel.
 *
 * Readings of definitions the paper leaves open (Section 5 cites PBBS for
 * Uniform/Exponential/AlmostSorted without defining them, and the duplicate
 * formulas are typeset without parentheses):
 *   Exponential   : bucket i uniform in [0, L), L = floor(log2 n) >= 1, then a
 *                   value uniform in [2^i, 2^(i+1)).
 *   AlmostSorted  : Sorted, then floor(sqrt n) transpositions of two
 *                   uniformly drawn positions (stream seed 2).
 *   Sorted        : the Uniform array (same seed) in ascending order.
 *   ReverseSorted : Sorted, reversed.
 *   RootDup       : A[i] = i mod floor(sqrt n), i = 0..n-1.
 *   TwoDup        : A[i] = (i^2 + n/2) mod n.
 *   EightDup      : A[i] = (i^8 + n/2) mod n   (exact 128-bit mulmod).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

enum {
    DIST_UNIFORM = 0, DIST_EXPONENTIAL = 1, DIST_ALMOST_SORTED = 2, DIST_SORTED = 3,
    DIST_REVERSE_SORTED = 4, DIST_ONES = 5, DIST_ROOT_DUP = 6, DIST_TWO_DUP = 7,
    DIST_EIGHT_DUP = 8, DIST_COUNT = 9
};

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output i (0-based) of the SplitMix64 stream started at `seed`. */
uint64_t gen_splitmix64_at(uint64_t seed, uint64_t i) {
    return mix64(seed + (i + 1) * GAMMA);
}

/* Uniform integer in [0, m) from a 64-bit draw (multiply-high). */
static inline uint64_t below(uint64_t r, uint64_t m) {
    return (uint64_t)(((unsigned __int128)r * m) >> 64);
}

static inline uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) {
    return (uint64_t)(((unsigned __int128)a * b) % m);
}

static uint64_t isqrt_floor(uint64_t n) {
    uint64_t r = (uint64_t)sqrt((double)n);
    while (r * r > n) --r;
    while ((r + 1) * (r + 1) <= n) ++r;
    return r;
}

static int floor_log2(uint64_t n) {
    int l = -1;
    while (n) { n >>= 1; ++l; }
    return l;
}

/* LSD radix sort on 64-bit unsigned values (8 passes of 8 bits).  Used only
 * to put the Uniform array in order for the Sorted family of inputs. */
static int radix_sort_u64(uint64_t* a, uint64_t n) {
    if (n < 2) return 0;
    uint64_t* tmp = (uint64_t*)malloc(n * sizeof(uint64_t));
    if (!tmp) return -1;
    uint64_t* src = a; uint64_t* dst = tmp;
    for (int pass = 0; pass < 8; ++pass) {
        uint64_t cnt[256];
        memset(cnt, 0, sizeof cnt);
        int sh = 8 * pass;
        for (uint64_t i = 0; i < n; ++i) cnt[(src[i] >> sh) & 255]++;
        uint64_t sum = 0;
        for (int d = 0; d < 256; ++d) { uint64_t c = cnt[d]; cnt[d] = sum; sum += c; }
        for (uint64_t i = 0; i < n; ++i) dst[cnt[(src[i] >> sh) & 255]++] = src[i];
        uint64_t* t = src; src = dst; dst = t;
    }
    /* 8 passes: result is back in `a`. */
    free(tmp);
    return 0;
}

/* Fill out[0..n) with 64-bit keys of distribution `dist`. Returns 0 on success. */
int gen_u64(uint64_t* out, uint64_t n, int dist, uint64_t seed) {
    if (dist < 0 || dist >= DIST_COUNT) return -1;
    if (n == 0) return 0;
    switch (dist) {
    case DIST_UNIFORM:
    case DIST_SORTED:
    case DIST_REVERSE_SORTED:
    case DIST_ALMOST_SORTED: {
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = gen_splitmix64_at(seed, (uint64_t)i);
        if (dist == DIST_UNIFORM) return 0;
        if (radix_sort_u64(out, n)) return -2;
        if (dist == DIST_REVERSE_SORTED) {
            for (uint64_t i = 0, j = n - 1; i < j; ++i, --j) { uint64_t t = out[i]; out[i] = out[j]; out[j] = t; }
        } else if (dist == DIST_ALMOST_SORTED) {
            uint64_t swaps = isqrt_floor(n);
            for (uint64_t s = 0; s < swaps; ++s) {
                uint64_t i = below(gen_splitmix64_at(2, 2 * s), n);
                uint64_t j = below(gen_splitmix64_at(2, 2 * s + 1), n);
                uint64_t t = out[i]; out[i] = out[j]; out[j] = t;
            }
        }
        return 0;
    }
    case DIST_EXPONENTIAL: {
        int L = floor_log2(n);
        if (L < 1) L = 1;
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < (int64_t)n; ++i) {
            uint64_t b = below(gen_splitmix64_at(seed, 2 * (uint64_t)i), (uint64_t)L);
            uint64_t lo = 1ULL << b;
            uint64_t r = gen_splitmix64_at(seed, 2 * (uint64_t)i + 1);
            out[i] = lo + (b == 63 ? (r & (lo - 1)) : below(r, lo));
        }
        return 0;
    }
    case DIST_ONES:
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = 1;
        return 0;
    case DIST_ROOT_DUP: {
        uint64_t r = isqrt_floor(n);
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = (uint64_t)i % r;
        return 0;
    }
    case DIST_TWO_DUP: {
        uint64_t h = n / 2;
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < (int64_t)n; ++i) {
            uint64_t p = mulmod((uint64_t)i, (uint64_t)i, n);
            out[i] = (p + h) % n;
        }
        return 0;
    }
    case DIST_EIGHT_DUP: {
        uint64_t h = n / 2;
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < (int64_t)n; ++i) {
            uint64_t p = (uint64_t)i % n;
            p = mulmod(p, p, n);   /* i^2 */
            p = mulmod(p, p, n);   /* i^4 */
            p = mulmod(p, p, n);   /* i^8 */
            out[i] = (p + h) % n;
        }
        return 0;
    }
    }
    return -1;
}

/* float64 keys.  The Uniform family maps a 64-bit draw x to (x >> 11) * 2^-53,
 * a value in [0, 1) that is never NaN or -0.0; the Sorted family sorts those
 * values (their order equals the order of x >> 11).  The integer families
 * (Exponential, Ones, *Dup) convert the 64-bit key to the nearest double. */
int gen_f64(double* out, uint64_t n, int dist, uint64_t seed) {
    if (dist < 0 || dist >= DIST_COUNT) return -1;
    if (n == 0) return 0;
    uint64_t* u = (uint64_t*)out;
    int rc = gen_u64(u, n, dist, seed);
    if (rc) return rc;
    const double scale = 1.0 / 9007199254740992.0; /* 2^-53 */
    int unit = (dist == DIST_UNIFORM || dist == DIST_SORTED || dist == DIST_REVERSE_SORTED ||
                dist == DIST_ALMOST_SORTED);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint64_t x = u[i];
        double d = unit ? (double)(x >> 11) * scale : (double)x;
        memcpy(&out[i], &d, 8);
    }
    return 0;
}

/* Key/payload pairs, 16 bytes each: out[2i] = key, out[2i+1] = payload. */
int gen_pair(uint64_t* out, uint64_t n, int dist, uint64_t key_seed, uint64_t payload_seed) {
    if (dist < 0 || dist >= DIST_COUNT) return -1;
    if (n == 0) return 0;
    uint64_t* keys = (uint64_t*)malloc(n * sizeof(uint64_t));
    if (!keys) return -2;
    int rc = gen_u64(keys, n, dist, key_seed);
    if (rc) { free(keys); return rc; }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        out[2 * i] = keys[i];
        out[2 * i + 1] = gen_splitmix64_at(payload_seed, (uint64_t)i);
    }
    free(keys);
    return 0;
}

/* 100-byte records: bytes [0,10) key, bytes [10,100) payload.
 * Key bytes of record r: little-endian bytes of draws 2r (8 bytes) and 2r+1
 * (low 2 bytes) of the key stream.  Payload: draws 12r..12r+11 of the payload
 * stream, first 90 bytes.  `dist` other than Uniform replaces the key by the
 * big-endian bytes of the 64-bit key of that distribution followed by two
 * zero bytes, so the lexicographic key order equals the integer order. */
int gen_rec100(uint8_t* out, uint64_t n, int dist, uint64_t key_seed, uint64_t payload_seed) {
    if (dist < 0 || dist >= DIST_COUNT) return -1;
    if (n == 0) return 0;
    uint64_t* keys = NULL;
    if (dist != DIST_UNIFORM) {
        keys = (uint64_t*)malloc(n * sizeof(uint64_t));
        if (!keys) return -2;
        int rc = gen_u64(keys, n, dist, key_seed);
        if (rc) { free(keys); return rc; }
    }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint8_t* rec = out + 100 * (uint64_t)i;
        if (keys) {
            uint64_t k = keys[i];
            for (int b = 0; b < 8; ++b) rec[b] = (uint8_t)(k >> (56 - 8 * b));
            rec[8] = 0; rec[9] = 0;
        } else {
            uint64_t a = gen_splitmix64_at(key_seed, 2 * (uint64_t)i);
            uint64_t c = gen_splitmix64_at(key_seed, 2 * (uint64_t)i + 1);
            for (int b = 0; b < 8; ++b) rec[b] = (uint8_t)(a >> (8 * b));
            rec[8] = (uint8_t)c; rec[9] = (uint8_t)(c >> 8);
        }
        uint8_t pay[96];
        for (int w = 0; w < 12; ++w) {
            uint64_t p = gen_splitmix64_at(payload_seed, 12 * (uint64_t)i + w);
            for (int b = 0; b < 8; ++b) pay[8 * w + b] = (uint8_t)(p >> (8 * b));
        }
        memcpy(rec + 10, pay, 90);
    }
    free(keys);
    return 0;
}

/* Segment lengths for the batched workload: floor(2^U), U uniform in
 * [lo_log2, hi_log2], from the given stream.  Writes count lengths. */
int gen_log_uniform_lengths(uint64_t* out, uint64_t count, double lo_log2, double hi_log2, uint64_t seed) {
    if (!(hi_log2 >= lo_log2)) return -1;
    for (uint64_t i = 0; i < count; ++i) {
        double u = (double)(gen_splitmix64_at(seed, i) >> 11) * (1.0 / 9007199254740992.0);
        double e = lo_log2 + u * (hi_log2 - lo_log2);
        uint64_t v = (uint64_t)floor(exp2(e));
        uint64_t lo = (uint64_t)ceil(exp2(lo_log2)), hi = (uint64_t)floor(exp2(hi_log2));
        if (v < lo) v = lo;
        if (v > hi) v = hi;
        out[i] = v;
    }
    return 0;
}

/* Keys of a batch of independent arrays stored back to back: array j (the
 * (first + j)-th of the batch, length lengths[j]) is gen_u64(lengths[j],
 * dist, seed + 2^32 * (first + j)), so that every array has its own value
 * stream and the distribution formulas use the array's own length. */
int gen_u64_segments(uint64_t* out, const uint64_t* lengths, uint64_t count, int dist, uint64_t seed,
                     uint64_t first) {
    if (dist < 0 || dist >= DIST_COUNT) return -1;
    uint64_t* starts = (uint64_t*)malloc((count + 1) * sizeof(uint64_t));
    if (!starts) return -2;
    starts[0] = 0;
    for (uint64_t j = 0; j < count; ++j) starts[j + 1] = starts[j] + lengths[j];
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int64_t j = 0; j < (int64_t)count; ++j)
        bad |= gen_u64(out + starts[j], lengths[j], dist, seed + ((first + (uint64_t)j) << 32)) != 0;
    free(starts);
    return bad ? -3 : 0;
}

/* Raw draws of a SplitMix64 stream: out[j] = output (first + j) of the
 * stream with the given seed (used for request types, distributions and
 * arrival times of the served workload). */
int gen_splitmix64_range(uint64_t* out, uint64_t count, uint64_t seed, uint64_t first) {
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (int64_t)count; ++j) out[j] = gen_splitmix64_at(seed, first + (uint64_t)j);
    return 0;
}
