/*
 * Sequential CPU samplesort oracle for the IPS4o distribution path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * GPU library is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg load it; the library never does, and the
 * two share no code.
 *
 * What it computes (Section 1, problem statement): the elements of A[0..n)
 * rearranged so that their keys are non-decreasing under a total order.  That
 * arrangement is unique for the keys, so any correct sort produces the same
 * key sequence; payloads of equal keys may come out in any order.
 *
 * How (Section 3, super scalar samplesort; Sections 4.4 and 4.7):
 *   1. n <= n0: insertion sort (Section 4.7, base case n0 = 16).
 *   2. oversampling factor alpha = max(1, floor(0.2 * log2 n)) (Section 4.7);
 *      draw alpha*k - 1 positions uniformly with replacement and sort the
 *      sample (Section 3).
 *   3. splitters s_j = sample[j*alpha - 1], j = 1..k-1, equally spaced in the
 *      sorted sample (Section 3); remove duplicates, and turn equality
 *      buckets on when any were removed (Section 4.7).
 *   4. element e goes to bucket i where s_i <= e < s_{i+1}, i.e. i = number of
 *      splitters <= e (Section 3).  With equality buckets (Section 4.4) the
 *      buckets interleave: 2i-1 holds the keys equal to s_i, 2i the keys
 *      strictly between s_i and s_{i+1}.
 *   5. distribute stably into a scratch array (a counting sort; the oracle
 *      need not be in place) and copy back.
 *   6. recurse on every bucket except the equality buckets, which are already
 *      sorted (Section 4.4).  On the last two levels k shrinks so that final
 *      buckets are not tiny (Section 4.7): while n < k^2 * n0, k is the largest
 *      power of two <= sqrt(n / n0), at least 2.
 *
 * Classification uses plain comparisons against the sorted splitter array
 * (binary search for the count of splitters <= e), not the implicit search
 * tree, so that it is checkable by eye and independent of the GPU code.
 *
 * Key types and their total orders:
 *   0 u64    8-byte little-endian unsigned integer.
 *   1 f64    IEEE-754 double, ordered by '<'; to make the order total the
 *            bit pattern b is mapped to (b has sign bit) ? ~b : b | 2^63, so
 *            -0.0 < +0.0 and NaNs sort to the ends.  On inputs without NaN and
 *            -0.0 this is exactly IEEE '<'.
 *   2 pair   16 bytes {u64 key; u64 payload}, ordered by key only.
 *   3 rec100 100 bytes, key = bytes [0,10) compared as unsigned bytes
 *            (lexicographically), payload = bytes [10,100).
 *   4 quartet 32 bytes {u64 k0, k1, k2; u64 payload}, key = (k0, k1, k2)
 *            compared lexicographically (Section 5: three key words and one
 *            word of associated information).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

enum { KT_U64 = 0, KT_F64 = 1, KT_PAIR = 2, KT_REC100 = 3, KT_QUARTET = 4 };

typedef struct {
    int k;          /* maximum number of buckets per level (power of two, >= 2) */
    int n0;         /* base-case size: n <= n0 is sorted by insertion sort */
    int alpha;      /* oversampling factor; <= 0 means max(1, floor(0.2 log2 n)) */
    int adaptive;   /* 1: shrink k on the last two levels (Section 4.7) */
    uint64_t seed;  /* sampling seed */
} oracle_params;

/* Comparable key: (hi, lo, lo2) compared lexicographically as unsigned. */
typedef struct { uint64_t hi, lo, lo2; } okey;

static size_t elem_size(int kt) {
    switch (kt) {
    case KT_U64: case KT_F64: return 8;
    case KT_PAIR: return 16;
    case KT_REC100: return 100;
    case KT_QUARTET: return 32;
    }
    return 0;
}

static okey key_of(const uint8_t* e, int kt) {
    okey k = {0, 0, 0};
    uint64_t v;
    switch (kt) {
    case KT_U64:
    case KT_PAIR:
        memcpy(&v, e, 8);
        k.hi = v;
        break;
    case KT_F64:
        memcpy(&v, e, 8);
        k.hi = (v >> 63) ? ~v : (v | 0x8000000000000000ULL);
        break;
    case KT_REC100:
        for (int b = 0; b < 8; ++b) k.hi = (k.hi << 8) | e[b];
        k.lo = ((uint64_t)e[8] << 8) | e[9];
        break;
    case KT_QUARTET:
        memcpy(&k.hi, e, 8);
        memcpy(&k.lo, e + 8, 8);
        memcpy(&k.lo2, e + 16, 8);
        break;
    }
    return k;
}

static int key_less(okey a, okey b) {
    return a.hi < b.hi || (a.hi == b.hi && (a.lo < b.lo || (a.lo == b.lo && a.lo2 < b.lo2)));
}
static int key_eq(okey a, okey b) { return a.hi == b.hi && a.lo == b.lo && a.lo2 == b.lo2; }

static int key_cmp_qsort(const void* pa, const void* pb) {
    const okey* a = (const okey*)pa;
    const okey* b = (const okey*)pb;
    return key_less(*a, *b) ? -1 : (key_less(*b, *a) ? 1 : 0);
}

/* SplitMix64 (Steele, Lea, Flood 2014) as the sampling stream. */
static uint64_t sm64_next(uint64_t* s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static int floor_log2_u64(uint64_t n) { int l = -1; while (n) { n >>= 1; ++l; } return l; }

/* ---- base case: insertion sort (Section 4.7) ---- */
static void insertion_sort(uint8_t* a, size_t n, size_t s, int kt, uint8_t* tmp) {
    for (size_t i = 1; i < n; ++i) {
        memcpy(tmp, a + i * s, s);
        okey ki = key_of(tmp, kt);
        size_t j = i;
        while (j > 0 && key_less(ki, key_of(a + (j - 1) * s, kt))) {
            memcpy(a + j * s, a + (j - 1) * s, s);
            --j;
        }
        memcpy(a + j * s, tmp, s);
    }
}

/* ---- fallback used only when a level makes no progress (k = 2 corner) ---- */
typedef struct { okey k; size_t idx; } keyed;
static int keyed_cmp(const void* pa, const void* pb) {
    const keyed* a = (const keyed*)pa; const keyed* b = (const keyed*)pb;
    if (key_less(a->k, b->k)) return -1;
    if (key_less(b->k, a->k)) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}
static int library_sort(uint8_t* a, size_t n, size_t s, int kt) {
    keyed* ks = (keyed*)malloc(n * sizeof(keyed));
    uint8_t* out = (uint8_t*)malloc(n * s);
    if (!ks || !out) { free(ks); free(out); return -1; }
    for (size_t i = 0; i < n; ++i) { ks[i].k = key_of(a + i * s, kt); ks[i].idx = i; }
    qsort(ks, n, sizeof(keyed), keyed_cmp);
    for (size_t i = 0; i < n; ++i) memcpy(out + i * s, a + ks[i].idx * s, s);
    memcpy(a, out, n * s);
    free(ks); free(out);
    return 0;
}

/* ---- one distribution step (Sections 3, 4.4, 4.7) ----
 * Returns the number of buckets (2m+1 with equality buckets, m+1 without) and
 * fills bounds[0..nb] with bucket boundaries (bounds[0] = 0, bounds[nb] = n).
 * Splitters (as keys) go to spl[0..m), *eq_out says whether equality buckets
 * were used.  Returns -1 on allocation failure. */
typedef struct {
    size_t m;          /* number of distinct splitters */
    int eq;            /* equality buckets on */
    okey* spl;         /* m splitters, ascending */
    size_t nb;         /* number of buckets */
    size_t* bounds;    /* nb + 1 bucket boundaries */
} level_result;

static int level_k(size_t n, const oracle_params* p) {
    int k = p->k;
    if (p->adaptive && (double)n < (double)k * (double)k * (double)p->n0) {
        double r = sqrt((double)n / (double)p->n0);
        int kk = 2;
        while ((double)(kk * 2) <= r && kk * 2 <= k) kk *= 2;
        k = kk;
    }
    return k;
}

static size_t count_le(const okey* spl, size_t m, okey e) {
    /* number of splitters <= e: first index whose splitter is > e */
    size_t lo = 0, hi = m;
    while (lo < hi) {
        size_t mid = lo + (hi - lo) / 2;
        if (key_less(e, spl[mid])) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static size_t bucket_of(const level_result* L, okey e) {
    size_t i = count_le(L->spl, L->m, e);
    if (!L->eq) return i;
    if (i >= 1 && key_eq(e, L->spl[i - 1])) return 2 * i - 1;
    return 2 * i;
}

static int distribute(uint8_t* a, size_t n, size_t s, int kt, const oracle_params* p,
                      int level, size_t offset, level_result* L) {
    memset(L, 0, sizeof *L);
    int k = level_k(n, p);
    int alpha = p->alpha > 0 ? p->alpha : (int)floor(0.2 * (double)floor_log2_u64(n));
    if (alpha < 1) alpha = 1;
    size_t ns = (size_t)alpha * (size_t)k - 1;

    /* sample with replacement */
    okey* sample = (okey*)malloc(ns * sizeof(okey));
    if (!sample) return -1;
    uint64_t st = p->seed ^ (0x632BE59BD9B4E019ULL * (uint64_t)(level + 1)) ^ (0x9E3779B97F4A7C15ULL * (uint64_t)offset);
    for (size_t j = 0; j < ns; ++j) {
        uint64_t r = sm64_next(&st);
        size_t pos = (size_t)(((unsigned __int128)r * n) >> 64);
        sample[j] = key_of(a + pos * s, kt);
    }
    qsort(sample, ns, sizeof(okey), key_cmp_qsort);

    /* equally spaced splitters, then duplicates removed */
    okey* spl = (okey*)malloc((size_t)k * sizeof(okey));
    if (!spl) { free(sample); return -1; }
    size_t m = 0;
    int dup = 0;
    for (int j = 1; j < k; ++j) {
        okey c = sample[(size_t)j * alpha - 1];
        if (m > 0 && key_eq(c, spl[m - 1])) { dup = 1; continue; }
        spl[m++] = c;
    }
    free(sample);
    L->m = m; L->eq = dup; L->spl = spl;
    L->nb = dup ? 2 * m + 1 : m + 1;

    /* classify and count */
    size_t* bid = (size_t*)malloc(n * sizeof(size_t));
    size_t* cnt = (size_t*)calloc(L->nb + 1, sizeof(size_t));
    uint8_t* tmp = (uint8_t*)malloc(n * s);
    if (!bid || !cnt || !tmp) { free(bid); free(cnt); free(tmp); free(spl); L->spl = NULL; return -1; }
    for (size_t i = 0; i < n; ++i) {
        bid[i] = bucket_of(L, key_of(a + i * s, kt));
        cnt[bid[i]]++;
    }
    /* bucket boundaries by prefix sum */
    L->bounds = (size_t*)malloc((L->nb + 1) * sizeof(size_t));
    if (!L->bounds) { free(bid); free(cnt); free(tmp); free(spl); L->spl = NULL; return -1; }
    size_t sum = 0;
    for (size_t b = 0; b < L->nb; ++b) { L->bounds[b] = sum; sum += cnt[b]; }
    L->bounds[L->nb] = sum;
    /* stable counting-sort distribution */
    for (size_t b = 0; b < L->nb; ++b) cnt[b] = L->bounds[b];
    for (size_t i = 0; i < n; ++i) memcpy(tmp + (cnt[bid[i]]++) * s, a + i * s, s);
    memcpy(a, tmp, n * s);
    free(bid); free(cnt); free(tmp);
    return 0;
}

static void free_level(level_result* L) { free(L->spl); free(L->bounds); L->spl = NULL; L->bounds = NULL; }

static int sort_rec(uint8_t* a, size_t n, size_t s, int kt, const oracle_params* p,
                    int level, size_t offset, uint8_t* tmp_elem) {
    if (n <= (size_t)p->n0 || n < 2) {
        insertion_sort(a, n, s, kt, tmp_elem);
        return 0;
    }
    level_result L;
    if (distribute(a, n, s, kt, p, level, offset, &L)) return -1;
    int rc = 0;
    for (size_t b = 0; b < L.nb && rc == 0; ++b) {
        if (L.eq && (b % 2 == 1)) continue;           /* equality bucket: done */
        size_t lo = L.bounds[b], hi = L.bounds[b + 1];
        if (hi - lo < 2) continue;
        if (hi - lo == n) {                            /* no progress (only k = 2) */
            rc = library_sort(a + lo * s, hi - lo, s, kt);
            continue;
        }
        rc = sort_rec(a + lo * s, hi - lo, s, kt, p, level + 1, offset + lo, tmp_elem);
    }
    free_level(&L);
    return rc;
}

static void fill_defaults(oracle_params* q, const oracle_params* p) {
    q->k = 256; q->n0 = 16; q->alpha = 0; q->adaptive = 1; q->seed = 0x1234567ULL;
    if (p) *q = *p;
    if (q->k < 2) q->k = 2;
    if (q->n0 < 1) q->n0 = 1;
}

/* Sort data[0..n) in place.  Returns 0, or -1 on bad arguments / no memory. */
int oracle_sort(void* data, size_t n, int kt, const oracle_params* params) {
    size_t s = elem_size(kt);
    if (!s) return -1;
    if (n < 2) return 0;
    if (!data) return -1;
    oracle_params p;
    fill_defaults(&p, params);
    uint8_t tmp_elem[128];
    return sort_rec((uint8_t*)data, n, s, kt, &p, 0, 0, tmp_elem);
}

/* One distribution step on data[0..n) (rearranged in place into buckets).
 * Outputs: spl_hi/spl_lo[0..m) the splitter keys, *m_out, *eq_out,
 * bounds[0..nb] (caller provides room for 2*k+2 entries), *nb_out. */
int oracle_partition(void* data, size_t n, int kt, const oracle_params* params,
                     uint64_t* spl_hi, uint64_t* spl_lo, size_t* m_out, int* eq_out,
                     size_t* bounds, size_t* nb_out, uint64_t* spl_lo2) {
    size_t s = elem_size(kt);
    if (!s || n < 2 || !data) return -1;
    oracle_params p;
    fill_defaults(&p, params);
    level_result L;
    if (distribute((uint8_t*)data, n, s, kt, &p, 0, 0, &L)) return -1;
    for (size_t j = 0; j < L.m; ++j) {
        spl_hi[j] = L.spl[j].hi;
        spl_lo[j] = L.spl[j].lo;
        if (spl_lo2) spl_lo2[j] = L.spl[j].lo2;
    }
    *m_out = L.m;
    *eq_out = L.eq;
    for (size_t b = 0; b <= L.nb; ++b) bounds[b] = L.bounds[b];
    *nb_out = L.nb;
    free_level(&L);
    return 0;
}

/* The comparable key of one element, as (hi, lo, lo2). */
void oracle_key(const void* elem, int kt, uint64_t* hi, uint64_t* lo, uint64_t* lo2) {
    okey k = key_of((const uint8_t*)elem, kt);
    *hi = k.hi; *lo = k.lo; *lo2 = k.lo2;
}

/* Order-statistic check at any size: counts the elements of data[0..n)
 * whose key is < and <= the key of `elem`.  The element of rank j in the
 * sorted output has key v exactly when less(v) <= j < less_equal(v). */
int oracle_rank_counts(const void* data, size_t n, int kt, const void* elem,
                       uint64_t* less, uint64_t* less_equal) {
    size_t s = elem_size(kt);
    if (!s) return -1;
    okey v = key_of((const uint8_t*)elem, kt);
    uint64_t lt = 0, le = 0;
    const uint8_t* a = (const uint8_t*)data;
    for (size_t i = 0; i < n; ++i) {
        okey e = key_of(a + i * s, kt);
        if (key_less(e, v)) { ++lt; ++le; }
        else if (key_eq(e, v)) ++le;
    }
    *less = lt; *less_equal = le;
    return 0;
}

/* Order-independent multiset hash of whole elements (all bytes, payload
 * included): out[0] = sum, out[1] = xor of a mixed 64-bit digest of each
 * element.  Equal multisets give equal hashes; a single changed element
 * changes both with overwhelming probability. */
static uint64_t mix_fin(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
int oracle_multiset_hash(const void* data, size_t n, int kt, uint64_t* out) {
    size_t s = elem_size(kt);
    if (!s) return -1;
    const uint8_t* a = (const uint8_t*)data;
    uint64_t sum = 0, x = 0;
    for (size_t i = 0; i < n; ++i) {
        uint64_t h = 0x243F6A8885A308D3ULL;
        const uint8_t* e = a + i * s;
        size_t off = 0;
        for (; off + 8 <= s; off += 8) { uint64_t w; memcpy(&w, e + off, 8); h = mix_fin(h ^ w) + off; }
        if (off < s) { uint64_t w = 0; memcpy(&w, e + off, s - off); h = mix_fin(h ^ w ^ 0xA5A5ULL); }
        h = mix_fin(h);
        sum += h; x ^= h;
    }
    out[0] = sum; out[1] = x;
    return 0;
}

/* 1 if the keys of data[0..n) are non-decreasing, else 0. */
int oracle_is_sorted(const void* data, size_t n, int kt) {
    size_t s = elem_size(kt);
    const uint8_t* a = (const uint8_t*)data;
    for (size_t i = 1; i < n; ++i)
        if (key_less(key_of(a + i * s, kt), key_of(a + (i - 1) * s, kt))) return 0;
    return 1;
}
