"""Pins for the CPU oracle (no GPU).

The oracle is a sequential samplesort (Sections 3, 4.4, 4.7).  It is pinned
here to things other than itself:
  * library routines that compute the same unique result (numpy.sort, Python
    sorted on the raw key bytes),
  * brute force over every permutation of small inputs,
  * the bucket rule of one distribution step (Section 3: s_i <= e < s_{i+1})
    and the equality-bucket property (Section 4.4), checked with
    numpy.searchsorted,
  * order-statistic and multiset invariants.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1705_02257_gb300 import inputs

DISTS = inputs.DISTRIBUTIONS


# ---------------------------------------------------------------- full sorts
@pytest.mark.parametrize("dist", DISTS)
@pytest.mark.parametrize("n", [0, 1, 2, 17, 1000, 65536 + 7])
def test_u64_matches_numpy(dist, n):
    a = inputs.u64(n, dist)
    assert np.array_equal(oracle.sort(a, "u64"), np.sort(a, kind="stable"))


@pytest.mark.parametrize("dist", DISTS)
def test_u64_small_k_and_base_case(dist):
    # k = 4, n0 = 1: forces many levels of sampling/classification/recursion.
    a = inputs.u64(5000, dist)
    out = oracle.sort(a, "u64", k=4, n0=1)
    assert np.array_equal(out, np.sort(a))


def test_u64_k2_quicksort_like_terminates():
    a = inputs.u64(3000, "two_dup")
    assert np.array_equal(oracle.sort(a, "u64", k=2, n0=1), np.sort(a))


def test_f64_matches_numpy_including_negatives_and_specials():
    rng = np.random.default_rng(7)
    a = np.concatenate([
        inputs.f64(20000),
        rng.standard_normal(20000) * 1e6,
        np.array([np.inf, -np.inf, 5e-324, -5e-324, 1e308, -1e308, 0.0, 1.0, -1.0]),
    ])
    rng.shuffle(a)
    out = oracle.sort(a, "f64")
    assert np.array_equal(out, np.sort(a))


def test_f64_total_order_on_signed_zero_and_nan():
    # IEEE '<' does not order -0.0/+0.0 or NaN; the oracle's map makes the
    # order total: -NaN < -inf < ... < -0.0 < +0.0 < ... < +inf < +NaN.
    neg_nan = np.frombuffer(np.uint64(0xFFF8000000000000).tobytes(), np.float64)[0]
    vals = np.array([np.nan, 0.0, -0.0, np.inf, -np.inf, 1.5, -1.5, neg_nan] * 5)
    out = oracle.sort(vals, "f64", n0=1, k=4)
    bits = out.view(np.uint64)
    mapped = np.where(bits >> np.uint64(63) == 1, ~bits, bits | np.uint64(1 << 63))
    assert np.all(mapped[1:] >= mapped[:-1])
    assert np.signbit(out[np.where(out == 0)[0][0]])  # first zero is -0.0
    assert np.isnan(out[0]) and np.isnan(out[-1])


@pytest.mark.parametrize("dist", ["uniform", "root_dup", "ones"])
def test_pair_keys_sorted_and_pairs_preserved(dist):
    p = inputs.pair(30001, dist)
    out = oracle.sort(p, "pair")
    assert np.array_equal(out["key"], np.sort(p["key"]))
    # same multiset of (key, payload): compare after a full lexicographic sort
    a = np.sort(p, order=["key", "payload"])
    b = np.sort(out, order=["key", "payload"])
    assert np.array_equal(a, b)


@pytest.mark.parametrize("dist", ["uniform", "two_dup"])
def test_rec100_lexicographic_keys(dist):
    r = inputs.rec100(20000, dist)
    out = oracle.sort(r, "rec100")
    assert [bytes(x[:10]) for x in out] == sorted(bytes(x[:10]) for x in r)
    assert sorted(bytes(x) for x in out) == sorted(bytes(x) for x in r)


# ------------------------------------------------------------- brute force
def _perm_inputs(n):
    yield "distinct", list(range(n))
    yield "equal", [7] * n
    yield "two", [i % 2 for i in range(n)]


@pytest.mark.parametrize("params", [dict(), dict(k=4, n0=1), dict(k=2, n0=1, alpha=1)])
@pytest.mark.parametrize("n", range(0, 9))
def test_brute_force_all_permutations(n, params):
    lib = oracle.load()
    for _, base in _perm_inputs(n):
        expected = np.array(sorted(base), dtype=np.uint64)
        seen = set()
        for perm in itertools.permutations(base):
            if perm in seen:
                continue
            seen.add(perm)
            a = np.array(perm, dtype=np.uint64)
            assert np.array_equal(oracle.sort(a, "u64", lib=lib, **params), expected), perm


# ------------------------------------------------ one distribution step
def _check_partition(a, key_type="u64", **params):
    out, spl, eq, bounds = oracle.partition(a, key_type, **params)
    n = len(a)
    assert bounds[0] == 0 and bounds[-1] == n
    assert np.all(np.diff(bounds) >= 0)
    keys = oracle.keys(out, key_type) if key_type != "u64" else np.stack(
        [out, np.zeros_like(out), np.zeros_like(out)], axis=1)
    s_hi = spl[:, 0]
    assert np.all(np.diff(s_hi.astype(np.float64)) >= 0)
    nb = len(bounds) - 1
    assert nb == (2 * len(spl) + 1 if eq else len(spl) + 1)
    # splitters strictly increasing (duplicates removed)
    sk = [tuple(x) for x in spl]
    assert all(sk[i] < sk[i + 1] for i in range(len(sk) - 1))
    for b in range(nb):
        seg = [tuple(x) for x in keys[bounds[b]:bounds[b + 1]]]
        if not seg:
            continue
        if eq:
            i, is_eq = (b + 1) // 2, b % 2 == 1
            if is_eq:
                assert set(seg) == {sk[i - 1]}, "equality bucket must hold one key"
                continue
        else:
            i = b
        lo = sk[i - 1] if i >= 1 else None
        hi = sk[i] if i < len(sk) else None
        for e in seg:
            if lo is not None:
                assert (e > lo) if eq else (e >= lo)
            if hi is not None:
                assert e < hi
    return out, spl, eq, bounds


@pytest.mark.parametrize("dist", DISTS)
def test_partition_bucket_rule(dist):
    a = inputs.u64(20000, dist)
    out, spl, eq, bounds = _check_partition(a)
    # the arrangement is a permutation of the input
    assert np.array_equal(np.sort(out), np.sort(a))
    # bucket sizes equal the counts given by numpy.searchsorted on the splitters
    s = spl[:, 0]
    if not eq:
        idx = np.searchsorted(s, a, side="right")
        counts = np.bincount(idx, minlength=len(s) + 1)
        assert np.array_equal(np.diff(bounds), counts)


def test_partition_ones_single_equality_bucket():
    a = inputs.u64(10000, "ones")
    out, spl, eq, bounds = _check_partition(a)
    assert eq and len(spl) == 1
    sizes = np.diff(bounds)
    assert sizes[1] == len(a) and sizes.sum() == len(a)


def test_partition_duplicates_turn_on_equality_buckets():
    a = inputs.u64(20000, "root_dup")   # 141 distinct keys, each ~141 times
    _, spl, eq, _ = _check_partition(a)
    assert eq
    b = inputs.u64(20000, "uniform")
    _, _, eq2, _ = _check_partition(b)
    assert not eq2


@pytest.mark.parametrize("key_type", ["f64", "pair", "rec100", "quartet"])
def test_partition_other_types(key_type):
    a = inputs.make(key_type, 3000, "uniform")
    _check_partition(a, key_type)


def test_adaptive_k_shrinks_small_levels():
    # Section 4.7: for n < k^2 n0 the number of buckets drops to the largest
    # power of two <= sqrt(n / n0); n = 2^17, n0 = 16 gives 64 buckets.
    a = inputs.u64(1 << 17)
    _, spl, eq, bounds = oracle.partition(a, "u64")
    assert not eq and len(spl) == 63
    _, spl2, _, _ = oracle.partition(a, "u64", adaptive=False)
    assert len(spl2) == 255


# ------------------------------------------------------------ invariants
def test_rank_counts_match_sorted_positions():
    a = inputs.u64(5000, "root_dup")
    s = np.sort(a)
    for j in [0, 1, 77, 2500, 4999]:
        lt, le = oracle.rank_counts(a, "u64", s[j:j + 1])
        assert lt <= j < le


def test_multiset_hash_permutation_invariant_and_sensitive():
    p = inputs.pair(4096, "root_dup")
    h = oracle.multiset_hash(p, "pair")
    q = p[np.random.default_rng(3).permutation(len(p))]
    assert oracle.multiset_hash(q, "pair") == h
    q["payload"][5] ^= np.uint64(1)
    assert oracle.multiset_hash(q, "pair") != h


def test_is_sorted():
    a = np.sort(inputs.u64(1000))
    assert oracle.is_sorted(a, "u64")
    a[[3, 4]] = a[[4, 3]]
    assert not oracle.is_sorted(a, "u64")


def test_rec100_key_is_big_endian_bytes():
    r = np.zeros((1, 100), dtype=np.uint8)
    r[0, :10] = np.arange(1, 11)
    k = oracle.keys(r, "rec100")[0]
    assert int(k[0]) == int.from_bytes(bytes(range(1, 9)), "big")
    assert int(k[1]) == (9 << 8) | 10


def test_splitters_are_equally_spaced_order_statistics():
    # Section 3: the k-1 splitters are picked equidistantly from the sorted
    # sample of alpha*k - 1 keys, s_j = sample[j*alpha - 1], i.e. s_j is the
    # (j*alpha)-th smallest of the sample.  For a sample drawn uniformly from
    # the keys 0..n-1, the r-th smallest of m draws has mean about
    # r / (m + 1) * n (order statistics of the uniform distribution), so with
    # k = 8, alpha = 3 (m = 23) the mean of s_j / n is j / 8.  Taking the
    # neighbouring sample entry instead (j*alpha or j*alpha - 2) shifts every
    # mean by 1/24, far outside the tolerance over 400 seeded samples.
    n = 1 << 16
    a = np.random.default_rng(5).permutation(n).astype(np.uint64)
    k, alpha = 8, 3
    rows = []
    for seed in range(1, 401):
        _, spl, eq, _ = oracle.partition(a, "u64", k=k, alpha=alpha, adaptive=False, seed=seed)
        if eq or len(spl) != k - 1:
            continue                      # the sample repeated a key (rare with distinct keys)
        rows.append(spl[:, 0].astype(np.float64) / n)
    assert len(rows) >= 390
    means = np.mean(np.array(rows), axis=0)
    expected = np.arange(1, k) / k
    assert np.all(np.abs(means - expected) < 0.025), means
    assert abs(float(np.mean(means - expected))) < 0.012, means


# ---------------------------------------------------------------- quartets
@pytest.mark.parametrize("dist", DISTS)
def test_quartet_matches_numpy_lexsort(dist):
    # Section 5: Quartet elements are compared lexicographically on their
    # three key words; numpy's lexsort (last key primary) gives the unique
    # key sequence, and the payloads form the same multiset
    a = inputs.quartet(20_011, dist)
    out = oracle.sort(a, "quartet")
    exp = a[np.lexsort((a["k2"], a["k1"], a["k0"]))]
    for f in ("k0", "k1", "k2"):
        assert np.array_equal(out[f], exp[f])
    assert np.array_equal(np.sort(out, order=["k0", "k1", "k2", "payload"]),
                          np.sort(a, order=["k0", "k1", "k2", "payload"]))


def test_quartet_ties_decided_by_later_words():
    # equal first words (Ones): the order comes from k1, then k2 alone
    a = inputs.quartet(5000, "ones")
    out = oracle.sort(a, "quartet", k=8, n0=4)
    assert np.all(out["k0"] == 1)
    pairs = list(zip(out["k1"].tolist(), out["k2"].tolist()))
    assert pairs == sorted(pairs)
