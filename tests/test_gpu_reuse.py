"""GPU parity of consecutive calls on one stream: entry points, element types
and sizes alternate, so each call carves the stream's workspace differently
and finds there whatever the previous call left.

The counters a launch keeps in the workspace between its CTAs (the base
case's next-task counter, the permutation's CTAs per subproblem) must not
depend on that: each result is compared with the CPU oracle, keys bit for bit
and pairs as a multiset, and the first calls are repeated at the end.
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1).copy()).cuda()


def _host(t, a):
    return t.cpu().numpy().view(a.dtype).reshape(a.shape)


def _same_keys(got, a, kt):
    exp = oracle.sort(a, kt)
    if kt == "pair":
        assert np.array_equal(got["key"], exp["key"])
        assert np.array_equal(np.sort(got, order=["key", "payload"]), np.sort(a, order=["key", "payload"]))
    elif kt == "quartet":
        for f in ("k0", "k1", "k2"):
            assert np.array_equal(got[f], exp[f]), f
        assert oracle.multiset_hash(got, "quartet") == oracle.multiset_hash(a, "quartet")
    else:
        assert np.array_equal(got.view(np.uint64), exp.view(np.uint64))


def _sort(ips4o, kt, a):
    t = _dev(a)
    ips4o.sort(t, kt)
    torch.cuda.synchronize()
    _same_keys(_host(t, a), a, kt)


def _strict(ips4o, a):
    t = _dev(a)
    ips4o.sort_strict(t, "u64")
    torch.cuda.synchronize()
    _same_keys(_host(t, a), a, "u64")


def _segmented(ips4o, count, hi_log2, dist):
    lengths = inputs.log_uniform_lengths(count, 1, hi_log2)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.uint64)
    a = inputs.u64_segments(lengths, dist)
    t = _dev(a)
    ips4o.sort_segmented(t, off, "u64")
    torch.cuda.synchronize()
    got = _host(t, a)
    for i in range(count):
        lo, hi = int(off[i]), int(off[i + 1])
        assert np.array_equal(got[lo:hi], oracle.sort(a[lo:hi], "u64")), i


def _batched(ips4o, sizes):
    arrays = [inputs.u64(n, "two_dup", seed=100 + i) for i, n in enumerate(sizes)]
    ts = [_dev(x) for x in arrays]
    ips4o.sort_batched(ts, "u64")
    torch.cuda.synchronize()
    for t, x in zip(ts, arrays):
        assert np.array_equal(_host(t, x), oracle.sort(x, "u64"))


def _host_sort(ips4o, a):
    b = a.copy()
    ips4o.sort_host(b, "u64")
    assert np.array_equal(b, oracle.sort(a, "u64"))


def test_alternating_calls_on_one_stream(ips4o):
    first = [
        lambda: _sort(ips4o, "u64", inputs.u64(3_000_017, "uniform")),
        lambda: _sort(ips4o, "pair", inputs.pair(500_003, "root_dup")),
        lambda: _sort(ips4o, "u64", inputs.u64(5_000, "uniform")),             # one base case
    ]
    rest = [
        lambda: _segmented(ips4o, 300, 16, "exponential"),
        lambda: _sort(ips4o, "f64", inputs.f64(1_000_003)),
        lambda: _strict(ips4o, inputs.u64(700_001, "two_dup")),
        lambda: _host_sort(ips4o, inputs.u64(1_000_003, "exponential")),
        # two levels: the second level's permutation has 256 subproblems, and
        # CTAs that finish join the ones that still have blocks to move
        lambda: _sort(ips4o, "u64", inputs.u64(20_000_003, "uniform")),
        lambda: _sort(ips4o, "quartet", inputs.quartet(300_007, "uniform")),
        lambda: _sort(ips4o, "u64", inputs.u64(1, "uniform")),
        lambda: _sort(ips4o, "u64", inputs.u64(0, "uniform")),
        lambda: _batched(ips4o, [1, 17, 4_096, 4_097, 70_000, 300_001]),
        lambda: _sort(ips4o, "u64", inputs.u64(9_000_011, "eight_dup")),
    ]
    for call in first + rest + first:
        call()
