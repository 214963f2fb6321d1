// Host-side check that ips4o_sort_noalloc's fixed scratch holds the
// workspace of every sort it accepts.
//
// The workspace of a sort of n elements follows from the same sizing rules
// the driver uses (caps_for, carve, host_stage_bytes in ips4o_driver.cuh,
// with the library's default parameters).  For every element type, every n
// from 2 to the entry point's limit (powers of two, their neighbours and
// seeded random sizes) and SM counts 1..kMaxSms, the device part must fit
// the __device__ scratch and the host part the static staging buffer.
// Prints "ok <cases> <largest device bytes> <largest host bytes>" and exits
// 0, or the first case that does not fit and exits 1.
#include <cstdio>
#include <random>
#include <vector>

#include "ips4o_driver.cuh"

using namespace ips4o;

constexpr int kMaxSms = 160;

template <class T>
static bool check(u64 n, int sms, size_t* dmax, size_t* hmax, const char* name) {
    const ips4o_params& p = kDefaultParams;
    const Caps<T> c = caps_for<T>(n, sms, p.stripes_per_sm, recursion_cap<T>(p));
    const size_t d = carve<T>(c, nullptr, nullptr), h = host_stage_bytes<T>(c);
    if (d > *dmax) *dmax = d;
    if (h > *hmax) *hmax = h;
    if (d > kNoAllocScratchBytes || h > kNoAllocHostBytes) {
        std::printf("does not fit: %s n=%llu sms=%d device=%zu host=%zu\n", name, n, sms, d, h);
        return false;
    }
    return true;
}

int main() {
    std::vector<u64> ns;
    for (u64 p = 2; p <= kNoAllocMaxN; p <<= 1) {
        ns.push_back(p - 1);
        ns.push_back(p);
        ns.push_back(p + 1);
    }
    std::mt19937_64 rng(7);
    for (int i = 0; i < 200; ++i) ns.push_back(2 + rng() % (kNoAllocMaxN - 1));
    size_t dmax = 0, hmax = 0, cases = 0;
    for (u64 n : ns) {
        if (n < 2 || n > kNoAllocMaxN) continue;
        for (int sms = 1; sms <= kMaxSms; ++sms) {
            if (!check<TU64>(n, sms, &dmax, &hmax, "u64") || !check<TF64>(n, sms, &dmax, &hmax, "f64") ||
                !check<TPair>(n, sms, &dmax, &hmax, "pair"))
                return 1;
            cases += 3;
        }
    }
    std::printf("ok %zu %zu %zu\n", cases, dmax, hmax);
    return 0;
}
