// Host-side check of the splitter lookup table of the local classification
// (lut_* in ips4o_common.cuh) against brute-force counting.
//
// For random and adversarial sorted splitter sets (full 64-bit range, a
// small range, keys just below 2^64, magnitudes spread over many octaves,
// clusters), padded to L - 1 entries by repeating the largest as the
// sampling step does, both cell maps (linear and logarithmic) must give
// i(e) = #{t in [1, L-1] : s_t <= e} for every splitter, every splitter +- 1,
// the first key of sampled cells +- 1, the ends of the key domain and random
// keys.  The table is built exactly as the kernel builds it: lo_c from the
// first key of cell c, hi_c = lo_{c+1} (L - 1 for the last cell), the extra
// entry (0, 0) for keys below s_1 (relative maps).  The absolute linear map
// (cells aligned to multiples of 2^shift, cell 0 starting at key 0) is
// checked in both its 64-bit and its 32-bit high-word form.  Prints "ok <keys checked>" and exits 0,
// or prints the first mismatch and exits 1.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "ips4o_common.cuh"

using namespace ips4o;

static int count_le(const std::vector<u64>& spl, int L, u64 e) {
    int c = 0;
    for (int t = 1; t < L; ++t) c += spl[t] <= e ? 1 : 0;
    return c;
}

int main(int argc, char** argv) {
    const int trials = argc > 1 ? std::atoi(argv[1]) : 600;
    std::mt19937_64 rng(7);
    long long checked = 0;
    for (int trial = 0; trial < trials; ++trial) {
        const int kind = trial % 6;
        int m = 1 + (int)(rng() % 255);
        std::vector<u64> c;
        for (int i = 0; i < m; ++i) {
            u64 v;
            switch (kind) {
            case 0: v = rng(); break;
            case 1: v = rng() % 1000; break;
            case 2: v = ~0ull - rng() % 100000; break;
            case 3: v = (u64)std::exp((double)(rng() % 4000) / 100.0); break;
            case 4: v = rng() >> (rng() % 64); break;
            default: v = (1ull << 63) + (rng() % 5000) * (1ull << 40); break;
            }
            c.push_back(v);
        }
        std::sort(c.begin(), c.end());
        c.erase(std::unique(c.begin(), c.end()), c.end());
        m = (int)c.size();
        int L = 2;
        while (L < m + 1) L <<= 1;
        std::vector<u64> spl(kMaxLeaves, 0);
        for (int i = 0; i < kMaxLeaves; ++i) spl[i] = c[(i >= 1 ? (i <= m ? i : m) : 1) - 1];
        const u64 base = spl[1], top = spl[L - 1];
        const u32 sh = lut_shift(base, top);
        if (((top - base) >> sh) >= (u64)kLutCells) {
            std::printf("shift %u leaves the range wider than the table\n", sh);
            return 1;
        }
        // map 3: linear cells aligned in the key domain (absolute), with the
        // 32-bit high-word form wherever the shift allows it
        const u32 ash = lut_abs_shift(base, top);
        const u64 ac0 = base >> ash;
        if ((top >> ash) - ac0 >= (u64)kLutCells) {
            std::printf("absolute shift %u leaves the range wider than the table\n", ash);
            return 1;
        }
        for (int mode = 1; mode <= 3; ++mode) {
            auto start = [&](u32 cc, u64* st) {
                if (mode == 3) return lut_cell_start_abs(cc, ac0, ash, st);
                return mode == 1 ? lut_cell_start(cc, base, sh, st) : lut_cell_start_log(cc, base, st);
            };
            auto cell = [&](u64 e) -> u32 {
                if (mode == 3) {
                    const u32 c = lut_cell_abs(e, ac0, ash);
                    if (ash >= 32 && lut_cell_abs_hi((u32)(e >> 32), (u32)ac0, ash - 32) != c) return kLutCells + 7;
                    return c;
                }
                return mode == 1 ? lut_cell(e, base, sh) : lut_cell_log(e, base);
            };
            std::vector<unsigned char> lo(kLutCells);
            for (u32 cc = 0; cc < (u32)kLutCells; ++cc) {
                u64 st;
                lo[cc] = start(cc, &st) ? (unsigned char)count_le(spl, L, st) : (unsigned char)(L - 1);
            }
            std::vector<unsigned short> lut(kLutCells + 1);
            for (int cc = 0; cc <= kLutCells; ++cc) {
                u32 ent = 0;
                if (cc < kLutCells) ent = (u32)lo[cc] | ((cc + 1 < kLutCells ? (u32)lo[cc + 1] : (u32)(L - 1)) << 8);
                lut[cc] = (unsigned short)ent;
            }
            if (mode == 3 && lo[0] != (unsigned char)count_le(spl, L, 0)) {
                std::printf("absolute map: cell 0 does not start at key 0\n");
                return 1;
            }
            std::vector<u64> keys = {0ull, ~0ull, base, top, base - 1, top + 1};
            for (int t = 1; t < L; ++t) {
                keys.push_back(spl[t]);
                keys.push_back(spl[t] - 1);
                keys.push_back(spl[t] + 1);
            }
            for (u32 cc = 0; cc < (u32)kLutCells; cc += 1 + (u32)(rng() % 64)) {
                u64 st;
                if (start(cc, &st)) {
                    keys.push_back(st);
                    keys.push_back(st - 1);
                    keys.push_back(st + 1);
                }
            }
            for (int r = 0; r < 500; ++r) {
                keys.push_back(rng());
                keys.push_back(top > base ? base + rng() % (top - base) : base);
            }
            if (mode == 3)
                for (int r = 0; r < 200; ++r) keys.push_back(base > 0 ? rng() % base : 0);   // below s_1
            for (u64 e : keys) {
                const u32 ce = cell(e);
                if (ce > (u32)kLutCells || (mode == 3 && ce >= (u32)kLutCells)) {
                    std::printf("cell %u out of range (map %d, key %llu)\n", ce, mode, e);
                    return 1;
                }
                const int got = lut_refine(e, lut[ce], spl.data());
                const int exp = count_le(spl, L, e);
                ++checked;
                if (got != exp) {
                    std::printf("mismatch: trial %d kind %d map %d key %llu: table %d, count %d\n", trial, kind, mode,
                                e, got, exp);
                    return 1;
                }
            }
        }
    }
    std::printf("ok %lld\n", checked);
    return 0;
}
