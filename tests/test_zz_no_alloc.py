"""ips4o_sort_noalloc: the sort for callers that cannot allocate memory.

Such callers (services whose device memory is fixed at start-up, plug-ins
whose host process owns every device allocation) use this entry point, which
works in a fixed scratch area built into the library instead of allocating a
workspace.  Its result must equal the oracle's sort and that of ips4o_sort,
exactly, on consecutive calls (the scratch keeps the previous call's
contents, so the second call checks that nothing stale leaks into it).  This
file is collected last on purpose.
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
    return m


def _both(ips4o, a, kt):
    kid = ips4o.KEY_TYPES[kt]
    raw = np.ascontiguousarray(a).view(np.uint8).reshape(-1)
    n = raw.size // ips4o.ELEM_SIZE[kid]
    t_noalloc = torch.from_numpy(raw.copy()).cuda()
    t_ref = torch.from_numpy(raw.copy()).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    rc = ips4o.ips4o_sort_noalloc(t_noalloc.data_ptr(), n, kid, stream)
    assert rc == 0, ips4o.ips4o_status_string(rc)
    ips4o.sort(t_ref, kt)
    torch.cuda.synchronize()
    return t_noalloc.cpu().numpy(), t_ref.cpu().numpy()


@pytest.mark.parametrize("kt,dist,n", [
    ("u64", "uniform", 1 << 20), ("u64", "two_dup", 777_777),
    ("f64", "uniform", 300_001), ("f64", "uniform", 1 << 20), ("pair", "root_dup", 500_000),
    ("pair", "uniform", 1 << 20), ("pair", "root_dup", 1 << 20),
])
def test_noalloc_equals_sort_on_two_calls_in_a_row(ips4o, kt, dist, n):
    for seed in (1, 7):
        a = inputs.make(kt, n, dist, seed=seed)
        got, ref = _both(ips4o, a, kt)
        exp = oracle.sort(a, kt)
        if kt != "pair":
            assert np.array_equal(got, ref)
            assert np.array_equal(got.view(np.uint64), exp.view(np.uint64))
        else:
            # not stable: the key sequence is unique, the payload order among
            # equal keys is not, so compare keys and the (key, payload) multiset
            g, r = got.view(inputs.PAIR_DTYPE), ref.view(inputs.PAIR_DTYPE)
            assert np.array_equal(g["key"], r["key"])
            assert np.array_equal(g["key"], exp["key"])
            assert np.array_equal(np.sort(g, order=["key", "payload"]), np.sort(r, order=["key", "payload"]))
            assert np.array_equal(np.sort(g, order=["key", "payload"]), np.sort(a, order=["key", "payload"]))


def test_noalloc_small_inputs(ips4o):
    for n in (0, 1, 2, 100, 16384):
        a = inputs.u64(n)
        got, ref = _both(ips4o, a, "u64")
        assert np.array_equal(got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(ips4o):
    t = torch.zeros((1 << 20) + 1, dtype=torch.int64, device="cuda")
    rc = ips4o.ips4o_sort_noalloc(t.data_ptr(), t.numel(), ips4o.U64, 0)
    assert rc == 8                     # IPS4O_ERR_TOO_LARGE, nothing queued
    assert "2^20" in ips4o.last_cuda_error()


def test_noalloc_refuses_a_stream_under_capture(ips4o):
    """The call synchronises its stream once per level, which a stream being
    captured into a CUDA graph does not allow: it must refuse before queuing
    anything, so the caller's capture stays valid."""
    x = torch.zeros(1024, dtype=torch.int64, device="cuda")
    t = torch.from_numpy(inputs.u64(100_000).view(np.int64).copy()).cuda()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            x.add_(1)
            rc = ips4o.ips4o_sort_noalloc(t.data_ptr(), t.numel(), ips4o.U64, s.cuda_stream)
            x.add_(1)
    assert rc == 1                      # IPS4O_ERR_INVALID_ARG
    assert "captured" in ips4o.last_cuda_error()
    g.replay()
    torch.cuda.synchronize()
    assert int(x[0].item()) == 2 and int(x.sum().item()) == 2 * 1024
