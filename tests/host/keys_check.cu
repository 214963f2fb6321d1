// Host-side check of the order-preserving key maps of ips4o_common.cuh
// against the plain definitions of each element type's total order:
//   f64:     IEEE '<' on values, with -0.0 < +0.0 and NaNs at the ends
//            (negative-signed NaNs below -inf, positive ones above +inf);
//            unkey(key(x)) gives back x bit for bit;
//   rec100:  bytes [0, 10) compared as unsigned bytes (memcmp);
//   quartet: (k0, k1, k2) compared lexicographically.
// Inputs: the special doubles, doubles of every magnitude, neighbours of
// each other, and random bit patterns; records and quartets drawn from small
// alphabets so that most pairs tie on a prefix.  Prints "ok <pairs checked>"
// and exits 0, or prints the first mismatch and exits 1.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <random>
#include <vector>

#include "ips4o_common.cuh"

using namespace ips4o;

static long checked = 0;

static u64 bits_of(double d) { u64 b; std::memcpy(&b, &d, 8); return b; }

// -1, 0, 1 by the definition of the f64 total order
static int f64_order(u64 a, u64 b) {
    double x, y;
    std::memcpy(&x, &a, 8);
    std::memcpy(&y, &b, 8);
    const bool nx = std::isnan(x), ny = std::isnan(y);
    const bool sx = (a >> 63) != 0, sy = (b >> 63) != 0;
    auto rank_nan = [](bool nan, bool sign) { return nan ? (sign ? -1 : 1) : 0; };   // -1: below all, 1: above all
    const int rx = rank_nan(nx, sx), ry = rank_nan(ny, sy);
    if (rx != ry) return rx < ry ? -1 : 1;
    if (nx && ny) {                                    // same side: by the bit pattern's magnitude
        const u64 mx = a & 0x7fffffffffffffffull, my = b & 0x7fffffffffffffffull;
        if (mx == my) return 0;
        return (sx ? mx > my : mx < my) ? -1 : 1;
    }
    if (x == 0.0 && y == 0.0) return sx == sy ? 0 : (sx ? -1 : 1);
    return x < y ? -1 : (y < x ? 1 : 0);
}

static bool check_f64(const std::vector<u64>& v) {
    for (u64 a : v) {
        if (TF64::unkey(TF64::key(a)) != a) {
            std::printf("f64 unkey(key(%016llx)) != itself\n", (unsigned long long)a);
            return false;
        }
        for (u64 b : v) {
            const u64 ka = TF64::key(a), kb = TF64::key(b);
            const int got = ka < kb ? -1 : (kb < ka ? 1 : 0), exp = f64_order(a, b);
            ++checked;
            if (got != exp) {
                std::printf("f64 order %016llx vs %016llx: key gives %d, definition %d\n", (unsigned long long)a,
                            (unsigned long long)b, got, exp);
                return false;
            }
        }
    }
    return true;
}

int main() {
    std::mt19937_64 rng(20261204);
    // ---- f64
    const double inf = std::numeric_limits<double>::infinity(), dmin = std::numeric_limits<double>::denorm_min();
    std::vector<double> special = {0.0, -0.0, 1.0, -1.0, inf, -inf, dmin, -dmin, std::numeric_limits<double>::min(),
                                   -std::numeric_limits<double>::min(), std::numeric_limits<double>::max(),
                                   -std::numeric_limits<double>::max(), 0.5, -0.5, 1e-300, -1e-300, 1e300, -1e300};
    std::vector<u64> v;
    for (double d : special) v.push_back(bits_of(d));
    v.push_back(0x7ff8000000000000ull);                  // quiet NaN
    v.push_back(0xfff8000000000000ull);                  // negative quiet NaN
    v.push_back(0x7ff0000000000001ull);                  // signalling NaN
    v.push_back(0xfff0000000000001ull);
    v.push_back(0x7fffffffffffffffull);
    v.push_back(0xffffffffffffffffull);
    for (int e = -1074; e <= 1023; e += 37) {            // every magnitude, both signs, and neighbours
        const double d = std::ldexp(1.0, e);
        v.push_back(bits_of(d));
        v.push_back(bits_of(-d));
        v.push_back(bits_of(std::nextafter(d, inf)));
        v.push_back(bits_of(std::nextafter(-d, -inf)));
    }
    for (int i = 0; i < 200; ++i) v.push_back(rng());    // random bit patterns (some NaN)
    if (!check_f64(v)) return 1;

    // ---- rec100: key bytes from a 3-letter alphabet, so that prefixes tie
    std::uniform_int_distribution<int> letter(0, 2);
    std::vector<RecElem> recs(300);
    for (auto& r : recs) {
        unsigned char* p = (unsigned char*)r.w;
        for (int i = 0; i < 100; ++i) p[i] = (unsigned char)(i < 10 ? 0x7f + 0x40 * letter(rng) : rng());
    }
    for (const auto& x : recs) {
        for (const auto& y : recs) {
            const int c = std::memcmp(x.w, y.w, 10);
            const RKey kx = TRec::key(x), ky = TRec::key(y);
            const int got = kx < ky ? -1 : (ky < kx ? 1 : 0), exp = c < 0 ? -1 : (c > 0 ? 1 : 0);
            ++checked;
            if (got != exp || (kx == ky) != (c == 0)) {
                std::printf("rec100 order: key gives %d, memcmp %d\n", got, exp);
                return 1;
            }
        }
    }

    // ---- quartet: words from {0, 1, 2^63, 2^64 - 1}
    const u64 words[4] = {0ull, 1ull, 1ull << 63, ~0ull};
    std::uniform_int_distribution<int> pick(0, 3);
    std::vector<QuartetElem> qs(200);
    for (auto& q : qs) q = QuartetElem{words[pick(rng)], words[pick(rng)], words[pick(rng)], rng()};
    for (const auto& x : qs) {
        for (const auto& y : qs) {
            const int exp = x.k0 != y.k0 ? (x.k0 < y.k0 ? -1 : 1)
                          : x.k1 != y.k1 ? (x.k1 < y.k1 ? -1 : 1)
                          : x.k2 != y.k2 ? (x.k2 < y.k2 ? -1 : 1) : 0;
            const QKey kx = TQuartet::key(x), ky = TQuartet::key(y);
            const int got = kx < ky ? -1 : (kx > ky ? 1 : 0);
            ++checked;
            if (got != exp || (kx == ky) != (exp == 0) || (kx <= ky) != (exp <= 0) || (kx >= ky) != (exp >= 0)) {
                std::printf("quartet order: key gives %d, definition %d\n", got, exp);
                return 1;
            }
        }
    }
    std::printf("ok %ld\n", checked);
    return 0;
}
