"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Keys are compared bit for bit with the oracle's output (the sorted key
sequence is unique).  For pairs the keys are compared bit for bit and the
(key, payload) multiset is compared exactly, since the method is not stable.
Sizes cover the shared-memory base case alone, one and two distribution
levels, n not a multiple of the block size (overflow block), and tiny n.
"""
import numpy as np
import pytest

import oracle
from paper_1705_02257_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ips4o():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_02257_gb300 import build
    build.build()
    from paper_1705_02257_gb300 import ips4o as m
    m.reset_params()
    return m


def gpu_sort(ips4o, a, kt):
    raw = np.ascontiguousarray(a).view(np.uint8).reshape(-1)
    t = torch.from_numpy(raw.copy()).cuda()
    ips4o.sort(t, kt)
    torch.cuda.synchronize()
    return t.cpu().numpy().view(a.dtype).reshape(a.shape)


def check_u64(ips4o, a):
    got = gpu_sort(ips4o, a, "u64")
    exp = oracle.sort(a, "u64")
    if not np.array_equal(got, exp):
        bad = np.nonzero(got != exp)[0]
        raise AssertionError(f"{len(bad)} mismatches, first at {bad[:5]} (n={len(a)})")


EDGE_SIZES = [0, 1, 2, 3, 31, 63, 64, 65, 1000, 8191, 8192, 8193, 8256, 16385, 100003]


@pytest.mark.parametrize("n", EDGE_SIZES)
@pytest.mark.parametrize("dist", ["uniform", "ones", "two_dup", "sorted"])
def test_u64_edge_sizes(ips4o, n, dist):
    check_u64(ips4o, inputs.u64(n, dist))


@pytest.mark.parametrize("dist", inputs.DISTRIBUTIONS)
def test_u64_all_distributions_2pow20(ips4o, dist):
    check_u64(ips4o, inputs.u64(1 << 20, dist))


@pytest.mark.parametrize("dist", inputs.DISTRIBUTIONS)
def test_u64_all_distributions_ragged_two_levels(ips4o, dist):
    # 3,000,017 keys: several stripes, two distribution levels, n % b != 0
    check_u64(ips4o, inputs.u64(3_000_017, dist))


def _key_range_case(kind, n):
    u = inputs.u64(n, "uniform", seed=11)
    v = inputs.u64(n, "uniform", seed=12)
    if kind == "near_top":          # keys just below 2^64: cell starts past the top of the key domain
        return (np.uint64(0xFFFFFFFFFFFFFFFF) - (u % np.uint64(100_000))).astype(np.uint64)
    if kind == "mixed_scales":      # every magnitude: cells holding many splitters
        return (u >> (v % np.uint64(64))).astype(np.uint64)
    if kind == "clusters":          # 8 narrow clusters far apart
        return (((v % np.uint64(8)) << np.uint64(60)) | (u % np.uint64(1000))).astype(np.uint64)
    raise ValueError(kind)


@pytest.mark.parametrize("n", [200_003, 3_000_017])
@pytest.mark.parametrize("kind", ["near_top", "mixed_scales", "clusters"])
def test_u64_key_range_corners(ips4o, kind, n):
    # the splitter lookup table of the local classification: cells past the
    # top of the domain, cells with many splitters, single-key cells
    check_u64(ips4o, _key_range_case(kind, n))


def test_u64_repeated_calls_same_result(ips4o):
    a = inputs.u64(500_001, "exponential")
    r1 = gpu_sort(ips4o, a, "u64")
    r2 = gpu_sort(ips4o, a, "u64")
    assert np.array_equal(r1, r2)
    assert np.array_equal(r1, oracle.sort(a, "u64"))


@pytest.mark.parametrize("n", [5, 8193, 1 << 20, 1_234_567])
def test_f64(ips4o, n):
    a = inputs.f64(n)
    got = gpu_sort(ips4o, a, "f64")
    assert np.array_equal(got.view(np.uint64), oracle.sort(a, "f64").view(np.uint64))


def test_f64_negative_and_special_values(ips4o):
    rng = np.random.default_rng(11)
    a = np.concatenate([rng.standard_normal(300_000) * 1e3,
                        np.array([0.0, -0.0, np.inf, -np.inf, 5e-324, -5e-324] * 1000)])
    rng.shuffle(a)
    got = gpu_sort(ips4o, a, "f64")
    assert np.array_equal(got.view(np.uint64), oracle.sort(a, "f64").view(np.uint64))


@pytest.mark.parametrize("dist", ["uniform", "root_dup", "ones", "eight_dup"])
@pytest.mark.parametrize("n", [4097, 700_001])
def test_pair(ips4o, dist, n):
    p = inputs.pair(n, dist)
    got = gpu_sort(ips4o, p, "pair")
    exp = oracle.sort(p, "pair")
    assert np.array_equal(got["key"], exp["key"])
    assert np.array_equal(np.sort(got, order=["key", "payload"]), np.sort(p, order=["key", "payload"]))


def _mapped_keys(a, kt):
    if kt == "u64":
        return a.view(np.uint64)
    if kt == "f64":
        b = a.view(np.uint64)
        return np.where(b >> np.uint64(63) == 1, ~b, b | np.uint64(1 << 63))
    if kt == "pair":
        return a["key"]
    raise ValueError(kt)


@pytest.mark.parametrize("kt,dist,n", [
    ("u64", "uniform", 1 << 20), ("u64", "root_dup", 1 << 20), ("u64", "ones", 300_000),
    ("u64", "exponential", 2_000_003), ("u64", "two_dup", 1 << 20), ("f64", "uniform", 777_777),
    ("pair", "root_dup", 500_000), ("u64", "uniform", 100), ("u64", "uniform", 7),
])
def test_partition_bucket_rule(ips4o, kt, dist, n):
    """One distribution step: every bucket holds exactly the keys the
    splitters assign to it (Section 3, s_i <= e < s_{i+1}; Section 4.4,
    equality buckets hold one key), and the step permutes the input."""
    _check_partition(ips4o, inputs.make(kt, n, dist), kt)


@pytest.mark.parametrize("n", [200_003, 3_000_017])
@pytest.mark.parametrize("kind", ["near_top", "mixed_scales", "clusters"])
def test_partition_bucket_rule_key_range_corners(ips4o, kind, n):
    _check_partition(ips4o, _key_range_case(kind, n), "u64")


def _check_partition(ips4o, a, kt):
    n = len(a)
    raw = np.ascontiguousarray(a).view(np.uint8).reshape(-1)
    t = torch.from_numpy(raw.copy()).cuda()
    bounds, spl, eq = ips4o.partition(t, kt)
    torch.cuda.synchronize()
    out = t.cpu().numpy().view(a.dtype).reshape(a.shape)
    assert bounds[0] == 0 and bounds[-1] == n and np.all(np.diff(bounds) >= 0)
    assert np.all(spl[1:] >= spl[:-1])
    keys = _mapped_keys(out, kt)
    nb = len(bounds) - 1
    assert nb == (2 * (len(spl) + 1) - 1 if eq else len(spl) + 1)
    for b in range(nb):
        seg = keys[bounds[b]:bounds[b + 1]]
        if len(seg) == 0:
            continue
        if eq:
            i = b // 2
            if b % 2 == 1:
                assert np.all(seg == spl[i]), f"equality bucket {b}"
                continue
            if i >= 1:
                assert np.all(seg > spl[i - 1]), f"bucket {b} lower bound"
            if i < len(spl):
                assert np.all(seg < spl[i]), f"bucket {b} upper bound"
        else:
            if b >= 1:
                assert np.all(seg >= spl[b - 1]), f"bucket {b} lower bound"
            if b < len(spl):
                assert np.all(seg < spl[b]), f"bucket {b} upper bound"
    # a permutation of the input
    assert oracle.multiset_hash(out, kt) == oracle.multiset_hash(a, kt)


def test_ones_single_equality_bucket(ips4o):
    a = inputs.u64(200_000, "ones")
    t = torch.from_numpy(a.view(np.int64).copy()).cuda()
    bounds, spl, eq = ips4o.partition(t, "u64")
    sizes = np.diff(bounds)
    assert eq
    assert sizes.max() == len(a)
    big = int(np.argmax(sizes))
    assert big % 2 == 1 and spl[big // 2] == 1


def test_stats_counters(ips4o):
    ips4o.ips4o_release_workspace()     # the workspace is then sized for this call alone
    a = inputs.u64(1 << 22)
    t = torch.from_numpy(a.view(np.int64).copy()).cuda()
    ips4o.sort(t, "u64")
    torch.cuda.synchronize()
    st = ips4o.stats()
    assert st["n"] == 1 << 22
    assert st["levels"] >= 1
    assert st["blocks_moved"] > 0
    assert st["base_case_buckets"] > 0
    assert st["workspace_bytes"] == ips4o.ips4o_workspace_bytes(1 << 22, ips4o.U64)


def test_sort_host_roundtrip(ips4o):
    a = inputs.u64(1_000_003, "two_dup")
    b = a.copy()
    ips4o.sort_host(b, "u64")
    assert np.array_equal(b, oracle.sort(a, "u64"))


@pytest.mark.parametrize("kt,dist,n", [
    ("u64", "uniform", 3_000_017), ("u64", "exponential", 2_000_003), ("u64", "ones", 300_001),
    ("u64", "ones", 3_000_001), ("u64", "two_dup", 3_000_017), ("u64", "eight_dup", 2_000_003),
    ("u64", "sorted", 2_000_003), ("u64", "exponential", 6_000_011), ("u64", "root_dup", 1_000_003),
    ("u64", "uniform", 1), ("u64", "uniform", 2), ("u64", "uniform", 1000), ("u64", "ones", 1000),
    ("u64", "two_dup", 16_384), ("u64", "two_dup", 16_385), ("f64", "uniform", 1_000_003),
    ("pair", "root_dup", 1_500_001), ("pair", "ones", 700_001), ("pair", "uniform", 777),
    ("quartet", "two_dup", 1_000_003), ("rec100", "uniform", 100_003),
])
def test_sort_host_pinned(ips4o, kt, dist, n):
    """Pinned host buffers: the first distribution level reads the host
    buffer through its device address (no separate copy pass), and the base
    case writes each sorted bucket straight back into it; equality buckets,
    single elements and subproblems of the segment scheduler are copied back
    by a kernel.  Inputs no larger than the base case are copied first.  The
    host buffer must end up sorted and the input must not be needed
    afterwards."""
    a = inputs.make(kt, n, dist)
    h = torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1).copy()).pin_memory()
    rc = ips4o.ips4o_sort_host(h.data_ptr(), n, ips4o.KEY_TYPES[kt], 0)
    assert rc == 0, ips4o.ips4o_status_string(rc)
    got = h.numpy().view(a.dtype).reshape(a.shape)
    exp = oracle.sort(a, kt)
    if kt == "pair":
        assert np.array_equal(got["key"], exp["key"])
        assert np.array_equal(np.sort(got, order=["key", "payload"]), np.sort(a, order=["key", "payload"]))
    elif kt == "quartet":
        for f in ("k0", "k1", "k2"):
            assert np.array_equal(got[f], exp[f]), f
        assert oracle.multiset_hash(got, "quartet") == oracle.multiset_hash(a, "quartet")
    elif kt == "rec100":
        assert np.array_equal(got, exp)
    else:
        assert np.array_equal(got.view(np.uint64), exp.view(np.uint64))


@pytest.mark.parametrize("dist", ["uniform", "two_dup", "exponential", "ones"])
def test_sort_host_pinned_deep(ips4o, dist):
    # a small base case and 4 buckets per step: many rounds, subproblems left
    # to the segment scheduler, and many equality buckets copied back
    a = inputs.u64(400_009, dist)
    ips4o.set_params(base_case_max=64, k_max=4)
    try:
        h = torch.from_numpy(a.view(np.uint8).copy()).pin_memory()
        rc = ips4o.ips4o_sort_host(h.data_ptr(), len(a), ips4o.U64, 0)
    finally:
        ips4o.reset_params()
    assert rc == 0, ips4o.ips4o_status_string(rc)
    assert np.array_equal(h.numpy().view(np.uint64), oracle.sort(a, "u64"))


@pytest.mark.parametrize("dist", ["uniform", "two_dup", "exponential", "ones"])
@pytest.mark.parametrize("k_max,bcm", [(256, 64), (4, 256), (16, 100)])
def test_deep_recursion(ips4o, dist, k_max, bcm):
    """A small base case and few buckets force several distribution levels
    (Section 4: the step recurses on every non-equality bucket)."""
    ips4o.set_params(base_case_max=bcm, k_max=k_max)
    try:
        a = inputs.u64(200_003, dist)
        check_u64(ips4o, a)
        if dist in ("uniform", "exponential"):
            assert ips4o.stats()["levels"] >= 2
    finally:
        ips4o.reset_params()


@pytest.mark.parametrize("kt,n", [("u64", 45_312_840), ("pair", 19_488_133)])
def test_heavy_duplicates_repeated(ips4o, kt, n):
    """RootDup keys (the first n of a 2^26-element RootDup array: 8192 keys,
    each about n / 8192 times) make equality buckets (Section 4.4), with
    empty buckets between non-empty ones, so the last block of a bucket can
    overshoot across empty buckets into the head of the next non-empty one
    (Section 4.3).  The head may only be written after the overshoot has
    been read; a wrong hand-off is a race, so the sort is repeated and every
    result compared with the oracle's."""
    a = inputs.make(kt, 1 << 26, "root_dup")[:n].copy()
    exp = oracle.sort(a, kt)
    exp_keys = exp["key"] if kt == "pair" else exp
    d_exp = torch.from_numpy(exp_keys.view(np.int64).copy()).cuda()
    src = torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1).copy()).cuda()
    work = torch.empty_like(src)
    for it in range(30):
        work.copy_(src)
        ips4o.sort(work, kt)
        keys = work.view(torch.int64)
        if kt == "pair":
            keys = keys.view(-1, 2)[:, 0]
        assert torch.equal(keys, d_exp), f"iteration {it}"
    if kt == "pair":
        got = work.cpu().numpy().view(inputs.PAIR_DTYPE)
        assert oracle.multiset_hash(got, kt) == oracle.multiset_hash(a, kt)


def _rec_keys(r):
    """The 10-byte keys of (n, 100) uint8 records as (big-endian 8 bytes, 2 bytes) columns."""
    b = np.ascontiguousarray(r[:, :10])
    hi = b[:, :8].copy().view(">u8").reshape(-1).astype(np.uint64)
    lo = (b[:, 8].astype(np.uint64) << np.uint64(8)) | b[:, 9].astype(np.uint64)
    return hi, lo


@pytest.mark.parametrize("dist", ["uniform", "ones", "two_dup", "root_dup", "sorted"])
@pytest.mark.parametrize("n", [1, 2, 7, 1000, 100_003, 1 << 20])
def test_rec100(ips4o, dist, n):
    """100-byte records (Section 5): the key order equals the oracle's bit
    for bit, and the records are a permutation of the input."""
    a = inputs.rec100(n, dist)
    t = torch.from_numpy(a.reshape(-1).copy()).cuda()
    ips4o.sort(t, "rec100")
    torch.cuda.synchronize()
    got = t.cpu().numpy().reshape(n, 100)
    exp = oracle.sort(a, "rec100")
    gh, gl = _rec_keys(got)
    eh, el = _rec_keys(exp)
    assert np.array_equal(gh, eh) and np.array_equal(gl, el)
    assert oracle.multiset_hash(got, "rec100") == oracle.multiset_hash(a, "rec100")


def test_rec100_equal_prefix_tie_break(ips4o):
    """Keys that agree in their first 8 bytes and differ only in bytes 8..9,
    and fully equal keys: ordered by all 10 bytes, equal keys in input order."""
    rng = np.random.default_rng(9)
    n = 50_000
    a = rng.integers(0, 256, size=(n, 100), dtype=np.uint8)
    a[:, :8] = rng.integers(0, 3, size=(n, 1), dtype=np.uint8)        # three 8-byte prefixes
    a[:, 8:10] = rng.integers(0, 4, size=(n, 2), dtype=np.uint8)      # 16 suffixes
    t = torch.from_numpy(a.reshape(-1).copy()).cuda()
    ips4o.sort(t, "rec100")
    got = t.cpu().numpy().reshape(n, 100)
    exp = oracle.sort(a, "rec100")
    assert np.array_equal(got[:, :10], exp[:, :10])
    # equal keys keep the input order: compare with a stable sort by key
    hi, lo = _rec_keys(a)
    order = np.lexsort((lo, hi))        # numpy's lexsort is stable
    assert np.array_equal(got, a[order])


def test_sort_only_enqueues_and_reports_through_the_stream(ips4o):
    """ips4o_sort plans the recursion on the device: the call returns while
    the sort is still running, and the stream status reports its outcome."""
    a = inputs.u64(1 << 27, "uniform")
    t = torch.from_numpy(a.view(np.int64).copy()).cuda()
    s = torch.cuda.current_stream()
    ips4o.sort(t, "u64")                     # warm-up: the workspace is allocated here
    torch.cuda.synchronize()
    t.copy_(torch.from_numpy(a.view(np.int64)))
    torch.cuda.synchronize()
    rc = ips4o.ips4o_sort(t.data_ptr(), t.numel(), ips4o.U64, s.cuda_stream)
    still_running = not s.query()
    assert rc == 0
    assert ips4o.ips4o_stream_status(s.cuda_stream) == 0
    assert still_running
    out = t.cpu().numpy().view(np.uint64)
    assert oracle.is_sorted(out, "u64") and oracle.multiset_hash(out, "u64") == oracle.multiset_hash(a, "u64")


@pytest.mark.parametrize("kt,n", [("u64", 3_000_017), ("pair", 1_000_003), ("f64", 20_000)])
def test_sort_captured_in_a_cuda_graph(ips4o, kt, n):
    """With its workspace reserved, ips4o_sort is capturable: the captured
    graph, replayed on new contents of the same buffer, sorts them."""
    kid = ips4o.KEY_TYPES[kt]
    s = torch.cuda.Stream()
    a0 = inputs.make(kt, n, "two_dup", seed=3)
    buf = torch.from_numpy(np.ascontiguousarray(a0).view(np.uint8).reshape(-1).copy()).cuda()
    with torch.cuda.stream(s):
        assert ips4o.ips4o_reserve_workspace(n, 1, kid, s.cuda_stream) == 0
        ips4o.sort(buf, kt, stream=s.cuda_stream)          # first call on the stream: kernel attributes
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = ips4o.ips4o_sort(buf.data_ptr(), n, kid, s.cuda_stream)
    assert rc == 0
    for seed in (5, 6):
        a = inputs.make(kt, n, "uniform" if seed == 5 else "root_dup", seed=seed)
        buf.copy_(torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1)))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert ips4o.ips4o_stream_status(s.cuda_stream) == 0
        got = buf.cpu().numpy().view(a.dtype).reshape(a.shape)
        exp = oracle.sort(a, kt)
        if kt == "pair":
            assert np.array_equal(got["key"], exp["key"])
            assert oracle.multiset_hash(got, kt) == oracle.multiset_hash(a, kt)
        else:
            assert np.array_equal(got.view(np.uint64), exp.view(np.uint64))


def test_capture_without_reserved_workspace_is_refused(ips4o):
    """Under capture nothing may be allocated: a sort larger than the
    stream's workspace returns IPS4O_ERR_TOO_LARGE and queues nothing."""
    s = torch.cuda.Stream()
    n = 1 << 22
    t = torch.zeros(n, dtype=torch.int64, device="cuda")
    x = torch.zeros(16, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        x.add_(1)
        rc = ips4o.ips4o_sort(t.data_ptr(), n, ips4o.U64, s.cuda_stream)
    assert rc == 8
    g.replay()
    torch.cuda.synchronize()
    assert int(x.sum().item()) == 16


def _check_quartet(got, a):
    """Quartets: the (k0, k1, k2) sequence equals the oracle's bit for bit;
    the elements are the input's multiset (payload order among equal keys is
    free, the method not being stable)."""
    exp = oracle.sort(a, "quartet")
    for f in ("k0", "k1", "k2"):
        assert np.array_equal(got[f], exp[f]), f
    assert oracle.multiset_hash(got, "quartet") == oracle.multiset_hash(a, "quartet")


@pytest.mark.parametrize("dist", inputs.DISTRIBUTIONS)
@pytest.mark.parametrize("n", [1 << 20, 1_500_007])
def test_quartet(ips4o, dist, n):
    """Section 5's Quartet: three key words compared lexicographically (the
    generator repeats first words and draws the second from four values, so
    later words decide many comparisons), one payload word, sorted in place."""
    a = inputs.quartet(n, dist)
    _check_quartet(gpu_sort(ips4o, a, "quartet"), a)


@pytest.mark.parametrize("n", [0, 1, 2, 15, 16, 17, 1023, 1024, 1025, 4096, 4097, 100_003])
def test_quartet_edge_sizes(ips4o, n):
    a = inputs.quartet(n, "two_dup")
    _check_quartet(gpu_sort(ips4o, a, "quartet"), a)


def test_quartet_segmented(ips4o):
    lengths = inputs.log_uniform_lengths(300, 4, 17)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.uint64)
    a = inputs.quartet(int(off[-1]), "root_dup")
    t = torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1).copy()).cuda()
    ips4o.sort_segmented(t, off, "quartet")
    torch.cuda.synchronize()
    got = t.cpu().numpy().view(inputs.QUARTET_DTYPE)
    for i in range(0, len(lengths), 7):
        lo, hi = int(off[i]), int(off[i + 1])
        _check_quartet(got[lo:hi], a[lo:hi])


@pytest.mark.parametrize("dist", ["uniform", "ones", "two_dup", "root_dup", "sorted", "exponential"])
@pytest.mark.parametrize("n", [1, 2, 5, 1023, 1025, 100_003, 1 << 20])
def test_rec100_block_path(ips4o, dist, n):
    """100-byte records moved in place through the distribution steps
    (params.record_path = 1): the key sequence equals the oracle's bit for
    bit and the records are the input's multiset (the block path is not
    stable, unlike the indirection)."""
    a = inputs.rec100(n, dist)
    ips4o.set_params(record_path=1)
    try:
        t = torch.from_numpy(a.reshape(-1).copy()).cuda()
        ips4o.sort(t, "rec100")
        torch.cuda.synchronize()
    finally:
        ips4o.reset_params()
    got = t.cpu().numpy().reshape(n, 100)
    exp = oracle.sort(a, "rec100")
    gh, gl = _rec_keys(got)
    eh, el = _rec_keys(exp)
    assert np.array_equal(gh, eh) and np.array_equal(gl, el)
    assert oracle.multiset_hash(got, "rec100") == oracle.multiset_hash(a, "rec100")
