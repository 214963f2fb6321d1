"""GPU parity of the strictly in-place sort (Section 4.6, ips4o_sort_strict)
against the CPU oracle, through the C ABI.

The strict recursion finds its remaining work by scanning the array for
bucket heads (keys larger than every key before them) and for descents, a
window at a time, so the cases below vary what the scan meets:
  * windows smaller than one bucket (a piece carried across many windows),
    several windows per distribution level, and the default window;
  * deep recursion (small base case, few buckets per step), so that most
    batches mark buckets and the scan goes back to the batch's start;
  * inputs already sorted, all equal, with long runs of equal keys, skewed;
  * every element type, including 100-byte records moved in place.
Keys are compared bit for bit with the oracle's output and payloads as a
multiset, as for ips4o_sort.
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


def strict_sort(ips4o, a, kt, **params):
    """Sort a copy of a with ips4o_sort_strict under params; returns the
    result (host) and the call's statistics."""
    if params:
        ips4o.set_params(**params)
    try:
        t = torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1).copy()).cuda()
        ips4o.sort_strict(t, kt)
        torch.cuda.synchronize()
        st = ips4o.stats()
    finally:
        ips4o.reset_params()
    return t.cpu().numpy().view(a.dtype).reshape(a.shape), st


def check_u64(ips4o, a, **params):
    got, st = strict_sort(ips4o, a, "u64", **params)
    exp = oracle.sort(a, "u64")
    if not np.array_equal(got, exp):
        bad = np.nonzero(got != exp)[0]
        raise AssertionError(f"{len(bad)} mismatches, first at {bad[:5]} (n={len(a)}, {params})")
    return st


def _rec_keys(r):
    b = np.ascontiguousarray(r[:, :10])
    hi = b[:, :8].copy().view(">u8").reshape(-1).astype(np.uint64)
    lo = (b[:, 8].astype(np.uint64) << np.uint64(8)) | b[:, 9].astype(np.uint64)
    return hi, lo


@pytest.mark.parametrize("n", [0, 1, 2, 3, 100, 16384, 16385, 20_000, 100_003])
def test_edge_sizes(ips4o, n):
    # at most one base case (n <= 16384) and one distribution step just above it
    check_u64(ips4o, inputs.u64(n, "uniform"))
    check_u64(ips4o, inputs.u64(n, "two_dup"))


@pytest.mark.parametrize("dist", inputs.DISTRIBUTIONS)
def test_default_window(ips4o, dist):
    check_u64(ips4o, inputs.u64(3_000_017, dist))


@pytest.mark.parametrize("dist", inputs.DISTRIBUTIONS)
@pytest.mark.parametrize("window", [2048, 3 * 2048, 1 << 18])
def test_small_windows(ips4o, dist, window):
    # pieces reach across many windows (window 2048: every bucket of the first
    # step spans tens of windows), and the scan's tile summaries are linked
    # across tiles and windows
    check_u64(ips4o, inputs.u64(1_000_003, dist), strict_window=window)


@pytest.mark.parametrize("dist", ["uniform", "two_dup", "eight_dup", "sorted", "reverse_sorted", "exponential",
                                  "ones", "root_dup"])
@pytest.mark.parametrize("window", [4096, 1 << 16, 0])
def test_deep_recursion(ips4o, dist, window):
    # base case of 64 elements and 4 buckets per step: about 8 levels, so
    # most batches mark buckets and the scan goes back to their start
    st = check_u64(ips4o, inputs.u64(300_007, dist), base_case_max=64, k_max=4, strict_window=window)
    if dist in ("uniform", "exponential"):
        assert st["levels"] >= 4, st


def test_many_batches_per_window(ips4o):
    # 2^22 keys, base case 1024, 16 buckets per step, windows of 2^20: each
    # window holds many marked buckets of several levels
    check_u64(ips4o, inputs.u64((1 << 22) + 123, "uniform"), base_case_max=1024, k_max=16,
              strict_window=1 << 20)


@pytest.mark.parametrize("n", [700_001, 4_000_037])
def test_f64(ips4o, n):
    a = inputs.f64(n)
    got, _ = strict_sort(ips4o, a, "f64", strict_window=1 << 19)
    assert np.array_equal(got.view(np.uint64), oracle.sort(a, "f64").view(np.uint64))


@pytest.mark.parametrize("dist", ["uniform", "root_dup", "ones", "eight_dup"])
def test_pair(ips4o, dist):
    p = inputs.pair(1_500_007, dist)
    got, _ = strict_sort(ips4o, p, "pair", strict_window=1 << 18, base_case_max=512, k_max=32)
    exp = oracle.sort(p, "pair")
    assert np.array_equal(got["key"], exp["key"])
    assert np.array_equal(np.sort(got, order=["key", "payload"]), np.sort(p, order=["key", "payload"]))


@pytest.mark.parametrize("dist", ["uniform", "two_dup", "sorted", "ones"])
def test_quartet(ips4o, dist):
    a = inputs.quartet(1_000_003, dist)
    got, _ = strict_sort(ips4o, a, "quartet", strict_window=1 << 17)
    exp = oracle.sort(a, "quartet")
    for f in ("k0", "k1", "k2"):
        assert np.array_equal(got[f], exp[f]), f
    assert oracle.multiset_hash(got, "quartet") == oracle.multiset_hash(a, "quartet")


@pytest.mark.parametrize("dist", ["uniform", "ones", "two_dup", "sorted"])
@pytest.mark.parametrize("n", [1000, 300_007])
def test_rec100(ips4o, dist, n):
    # 100-byte records moved in place (blocks of 5 records) by the strict
    # recursion: keys equal to the oracle's bit for bit, records the input's
    # multiset
    a = inputs.rec100(n, dist)
    got, _ = strict_sort(ips4o, a, "rec100", strict_window=1 << 16)
    exp = oracle.sort(a, "rec100")
    gh, gl = _rec_keys(got)
    eh, el = _rec_keys(exp)
    assert np.array_equal(gh, eh) and np.array_equal(gl, el)
    assert oracle.multiset_hash(got, "rec100") == oracle.multiset_hash(a, "rec100")


def test_full_size_2pow28(ips4o):
    # the benchmark's 2^28 uint64 Uniform keys with the default window (8
    # windows): non-decreasing, the input's multiset, and the oracle's rank
    # rule at seeded positions (the checks of the full-size ips4o_sort tests)
    n = 1 << 28
    a = inputs.u64(n, "uniform")
    t = torch.from_numpy(a.view(np.uint8)).cuda()
    ips4o.sort_strict(t, "u64")
    torch.cuda.synchronize()
    out = t.cpu().numpy().view(np.uint64)
    del t
    assert oracle.is_sorted(out, "u64")
    assert oracle.multiset_hash(out, "u64") == oracle.multiset_hash(a, "u64")
    for r in np.concatenate([np.random.default_rng(20261).integers(0, n, 8), [0, n - 1]]):
        v = out[r]
        lt = int(np.count_nonzero(a < v))
        le = int(np.count_nonzero(a <= v))
        assert lt <= r < le, (int(r), lt, le)


def test_workspace_reported(ips4o):
    # the workspace the call holds is what ips4o_workspace_bytes_strict says
    # (the stream's buffer grows to the largest call made on it)
    a = inputs.u64(1 << 22, "uniform")
    _, st = strict_sort(ips4o, a, "u64")
    assert st["workspace_bytes"] >= ips4o.workspace_bytes_strict(1 << 22, "u64")


def test_refused_under_capture(ips4o):
    # the call synchronises between batches, so a stream being captured is
    # refused before anything is queued and the capture stays valid
    x = torch.zeros(1024, dtype=torch.int64, device="cuda")
    t = torch.from_numpy(inputs.u64(100_000).view(np.int64).copy()).cuda()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            x.add_(1)
            rc = ips4o.ips4o_sort_strict(t.data_ptr(), t.numel(), ips4o.U64, s.cuda_stream)
            x.add_(1)
    assert rc == 1                      # IPS4O_ERR_INVALID_ARG
    assert "captured" in ips4o.last_cuda_error()
    g.replay()
    torch.cuda.synchronize()
    assert int(x.sum().item()) == 2 * 1024
