"""GPU parity at the benchmark's full sizes, in the configuration bench.py
times (default parameters, one ips4o_sort call on a device array).

At 2^28 keys the oracle's full sort would take most of a minute per case, so
the output is checked through properties that fix it at any size, with the
oracle's own checkers:
  * non-decreasing in the key order (oracle.is_sorted);
  * the same multiset as the input (oracle.multiset_hash: order-independent
    sum and xor of mixed (key, payload) words);
  * at 12 seeded ranks r (and both ends), the output's key is the r-th smallest input key,
    counted directly: #{keys < v} <= r < #{keys <= v}.
Non-decreasing and the same multiset together determine the key sequence.
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


def _order_keys(a, kt):
    """Keys as uint64 in the sort order (f64: the order-preserving map of the bits)."""
    if kt == "pair":
        return np.ascontiguousarray(a["key"])
    k = np.ascontiguousarray(a).view(np.uint64)
    if kt == "f64":
        neg = (k >> np.uint64(63)) != 0
        return np.where(neg, ~k, k | np.uint64(1 << 63))
    return k


@pytest.mark.parametrize("kt,dist,log2n", [
    ("u64", "uniform", 28), ("u64", "two_dup", 28), ("f64", "uniform", 27), ("pair", "uniform", 27),
])
def test_full_size(ips4o, kt, dist, log2n):
    n = 1 << log2n
    a = inputs.make(kt, n, dist)
    t = torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1)).cuda()
    ips4o.sort(t, kt)
    torch.cuda.synchronize()
    out = t.cpu().numpy().view(a.dtype).reshape(a.shape)
    del t
    assert oracle.is_sorted(out, kt)
    assert oracle.multiset_hash(out, kt) == oracle.multiset_hash(a, kt)
    keys_in, keys_out = _order_keys(a, kt), _order_keys(out, kt)
    ranks = np.random.default_rng(20260).integers(0, n, 12)
    for r in np.concatenate([ranks, [0, n - 1]]):
        v = keys_out[r]
        lt = int(np.count_nonzero(keys_in < v))
        le = int(np.count_nonzero(keys_in <= v))
        assert lt <= r < le, (int(r), lt, le)
