"""The seeded generators reproduce the paper's input definitions (Section 5).

Each distribution is recomputed here independently (Python integers or numpy)
and compared element by element, and the duplicate counts are pinned to
closed forms: the number of squares modulo 2^m (m >= 3) is (2^m + 8)/6 for
even m and (2^m + 10)/6 for odd m, and adding n/2 modulo n is a bijection,
so TwoDup at n = 2^20 has exactly 174,764 distinct keys.
"""
import math

import numpy as np
import pytest

from paper_1705_02257_gb300 import inputs

M64 = (1 << 64) - 1


def _sm64(seed, i):
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_splitmix64_reference_values():
    # SplitMix64 from state 0: first outputs of the published generator.
    assert inputs.splitmix64_at(0, 0) == 0xE220A8397B1DCDAF
    assert inputs.splitmix64_at(0, 1) == 0x6E789E6AA1B965F4
    for i in range(50):
        assert inputs.splitmix64_at(1, i) == _sm64(1, i)


def test_uniform_is_the_stream():
    a = inputs.u64(1000)
    assert [int(x) for x in a] == [_sm64(1, i) for i in range(1000)]


@pytest.mark.parametrize("n", [1 << 16, 100003])
def test_dup_families_exact(n):
    i = np.arange(n, dtype=object)
    r = math.isqrt(n)
    assert np.array_equal(inputs.u64(n, "root_dup"), np.array([x % r for x in range(n)], np.uint64))
    two = np.array([(x * x + n // 2) % n for x in range(n)], dtype=np.uint64)
    assert np.array_equal(inputs.u64(n, "two_dup"), two)
    eight = np.array([(pow(x, 8, n) + n // 2) % n for x in range(n)], dtype=np.uint64)
    assert np.array_equal(inputs.u64(n, "eight_dup"), eight)


@pytest.mark.parametrize("m", [10, 13, 20])
def test_two_dup_distinct_count_closed_form(m):
    n = 1 << m
    expected = (n + 8) // 6 if m % 2 == 0 else (n + 10) // 6
    assert len(np.unique(inputs.u64(n, "two_dup"))) == expected


def test_root_dup_and_ones_counts():
    n = 1 << 20
    a = inputs.u64(n, "root_dup")
    vals, cnt = np.unique(a, return_counts=True)
    assert len(vals) == 1024 and cnt.max() == 1024
    assert np.all(inputs.u64(1000, "ones") == 1)


def test_sorted_family():
    n = 50001
    u = inputs.u64(n)
    s = inputs.u64(n, "sorted")
    assert np.array_equal(s, np.sort(u))
    assert np.array_equal(inputs.u64(n, "reverse_sorted"), np.sort(u)[::-1])
    al = inputs.u64(n, "almost_sorted")
    assert np.array_equal(np.sort(al), s)
    # floor(sqrt n) transpositions move at most 2*floor(sqrt n) positions
    assert np.count_nonzero(al != s) <= 2 * math.isqrt(n)


def test_exponential_ranges():
    n = 1 << 16
    a = inputs.u64(n, "exponential")
    L = 16
    assert a.min() >= 1 and a.max() < (1 << L)
    # bucket index floor(log2 v) is roughly uniform over [0, L)
    b = np.floor(np.log2(a.astype(np.float64))).astype(int)
    cnt = np.bincount(b, minlength=L)
    assert len(cnt) == L and cnt.min() > 0.8 * n / L and cnt.max() < 1.2 * n / L


def test_f64_uniform_unit_interval():
    a = inputs.f64(100000)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert not np.any(np.isnan(a)) and not np.any(np.signbit(a))
    u = inputs.u64(100000)
    assert np.array_equal(a, (u >> np.uint64(11)).astype(np.float64) * 2.0 ** -53)


def test_pair_and_rec100_layout():
    p = inputs.pair(100, "root_dup")
    assert np.array_equal(p["key"], inputs.u64(100, "root_dup"))
    assert [int(x) for x in p["payload"]] == [_sm64(3, i) for i in range(100)]
    r = inputs.rec100(10)
    for i in range(10):
        a, c = _sm64(1, 2 * i), _sm64(1, 2 * i + 1)
        assert bytes(r[i, :8]) == a.to_bytes(8, "little")
        assert bytes(r[i, 8:10]) == (c & 0xFFFF).to_bytes(2, "little")
        pay = b"".join(_sm64(3, 12 * i + w).to_bytes(8, "little") for w in range(12))
        assert bytes(r[i, 10:]) == pay[:90]


def test_log_uniform_lengths():
    L = inputs.log_uniform_lengths(100000, 4, 20)
    assert L.min() >= 16 and L.max() <= 1 << 20
    e = np.log2(L.astype(np.float64))
    assert abs(np.median(e) - 12) < 0.1


def test_u64_segments_are_independent_arrays():
    """Array j of a batch equals the generator run alone on its own length
    with value seed 1 + 2^32 * j (so TwoDup etc. use the array's length)."""
    lengths = np.array([5, 0, 17, 1, 64], dtype=np.uint64)
    for dist in ("uniform", "two_dup", "almost_sorted"):
        a = inputs.u64_segments(lengths, dist)
        off = np.concatenate([[0], np.cumsum(lengths)]).astype(int)
        for j in range(len(lengths)):
            alone = inputs.u64(int(lengths[j]), dist, seed=1 + (j << 32))
            assert np.array_equal(a[off[j]:off[j + 1]], alone)
    b = inputs.u64_segments(lengths[2:], "uniform", first=2)
    assert np.array_equal(b[:17], inputs.u64(17, "uniform", seed=1 + (2 << 32)))


def test_splitmix64_range_matches_single_draws():
    r = inputs.splitmix64_range(5, 5, first=3)
    assert [int(x) for x in r] == [inputs.splitmix64_at(5, 3 + j) for j in range(5)]
    u = inputs.unit_uniform(1000, 5)
    assert u.min() >= 0.0 and u.max() < 1.0


def test_request_stream_mix_and_rate():
    sizes, types, dists, arr = inputs.request_stream(20000, 10, 26, rate=100.0)
    assert sizes.min() >= 1024 and sizes.max() <= 1 << 26
    frac = {t: types.count(t) / len(types) for t in ("u64", "f64", "pair")}
    assert abs(frac["u64"] - 0.5) < 0.02 and abs(frac["f64"] - 0.25) < 0.02 and abs(frac["pair"] - 0.25) < 0.02
    assert set(dists) == set(inputs.DISTRIBUTIONS)
    assert arr[0] == 0.0 and np.all(np.diff(arr) >= 0)
    # Poisson process: mean gap 1 / rate
    assert abs(np.diff(arr).mean() - 0.01) < 0.0005
