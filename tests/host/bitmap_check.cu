// Host-side check of first_live_bucket (ips4o_common.cuh), the search of the
// block permutation's exhausted bitmap (Section 4.2: a mover whose primary
// bucket has no unprocessed block left takes the next bucket that has one).
//
// For bitmaps with every bucket marked, none marked, one bucket free, runs of
// free buckets across word boundaries and random densities, and for every
// start 0..511 (callers pass start = bucket + 1 <= 256), the result must be
// the first unmarked bucket c in start, start + 1, ... (mod 256), found by
// testing the bits one at a time, or 0xffffffff when there is none.  Prints
// "ok <cases checked>" and exits 0, or prints the first mismatch and exits 1.
#include <cstdio>
#include <random>

#include "ips4o_common.cuh"

using namespace ips4o;

static u32 brute(const u32 (&w)[8], u32 start) {
    for (u32 s = 0; s < 256; ++s) {
        const u32 c = (start + s) & 255u;
        if (!((w[c >> 5] >> (c & 31)) & 1u)) return c;
    }
    return 0xffffffffu;
}

static long checked = 0;

static bool check(const u32 (&w)[8]) {
    for (u32 start = 0; start < 512; ++start) {
        const u32 got = first_live_bucket(w, start), exp = brute(w, start);
        ++checked;
        if (got != exp) {
            std::printf("mismatch: start %u got %u expected %u; bitmap", start, got, exp);
            for (int i = 0; i < 8; ++i) std::printf(" %08x", w[i]);
            std::printf("\n");
            return false;
        }
    }
    return true;
}

int main() {
    u32 w[8];
    for (int i = 0; i < 8; ++i) w[i] = 0xffffffffu;
    if (!check(w)) return 1;                                // every bucket marked
    for (int i = 0; i < 8; ++i) w[i] = 0;
    if (!check(w)) return 1;                                // none marked
    for (u32 b = 0; b < 256; ++b) {                         // exactly one bucket free
        for (int i = 0; i < 8; ++i) w[i] = 0xffffffffu;
        w[b >> 5] &= ~(1u << (b & 31));
        if (!check(w)) return 1;
    }
    for (u32 lo = 0; lo < 256; lo += 7) {                   // a run of free buckets, wrapping around
        for (u32 len = 1; len <= 70; len += 3) {
            for (int i = 0; i < 8; ++i) w[i] = 0xffffffffu;
            for (u32 k = 0; k < len; ++k) {
                const u32 b = (lo + k) & 255u;
                w[b >> 5] &= ~(1u << (b & 31));
            }
            if (!check(w)) return 1;
        }
    }
    std::mt19937_64 rng(20261204);
    for (int t = 0; t < 2000; ++t) {                        // random densities
        const double p = (double)(t % 100) / 100.0;         // probability that a bucket is marked
        std::bernoulli_distribution bit(p);
        for (int i = 0; i < 8; ++i) {
            w[i] = 0;
            for (int k = 0; k < 32; ++k) w[i] |= (bit(rng) ? 1u : 0u) << k;
        }
        if (!check(w)) return 1;
    }
    std::printf("ok %ld\n", checked);
    return 0;
}
