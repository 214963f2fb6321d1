"""GPU parity of the segmented and batched entry points.

Every segment must come out exactly as the oracle sorts it alone (keys bit
for bit; for pairs also the (key, payload) multiset), elements outside the
segments must keep their bytes, and the result must equal sorting each
segment by itself with ips4o_sort.  Segment lengths follow the log-uniform
law of the batched workload (lengths 2^U, U uniform), seed 4.
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


@pytest.fixture(params=[1, 2], ids=["levels", "scheduler"])
def mode(request, ips4o):
    """Both processing forms of segmented and batched calls: level by level
    across all segments (1) and the segment scheduler, one CTA per array (2)."""
    ips4o.set_params(segment_scheduler=request.param)
    yield request.param
    ips4o.reset_params()


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1).copy()).cuda()


def to_host(t, like):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(like.dtype).reshape(like.shape)


def offsets_for(lengths, start=0):
    return np.concatenate([[0], np.cumsum(lengths, dtype=np.uint64)]).astype(np.uint64) + np.uint64(start)


def check_segments(got, a, off, kt):
    for i in range(len(off) - 1):
        lo, hi = int(off[i]), int(off[i + 1])
        seg, exp = got[lo:hi], oracle.sort(a[lo:hi], kt)
        if kt == "pair":
            assert np.array_equal(seg["key"], exp["key"]), f"segment {i} [{lo}, {hi})"
            assert np.array_equal(np.sort(seg, order=["key", "payload"]),
                                  np.sort(a[lo:hi], order=["key", "payload"])), f"segment {i} payloads"
        else:
            assert np.array_equal(seg.view(np.uint64), exp.view(np.uint64)), f"segment {i} [{lo}, {hi})"


@pytest.mark.parametrize("kt,dist", [("u64", "uniform"), ("u64", "two_dup"), ("f64", "uniform"),
                                     ("pair", "root_dup"), ("u64", "ones")])
def test_segmented_log_uniform_lengths(ips4o, mode, kt, dist):
    lengths = inputs.log_uniform_lengths(1000, 4, 17)
    off = offsets_for(lengths)
    a = inputs.make(kt, int(off[-1]), dist)
    t = to_dev(a)
    ips4o.sort_segmented(t, off, kt)
    check_segments(to_host(t, a), a, off, kt)


def test_segmented_offsets_on_device_and_untouched_margins(ips4o, mode):
    lengths = np.array([0, 1, 2, 3, 17, 0, 8192, 8193, 16384, 16385, 70_000, 1, 200_003], dtype=np.uint64)
    start = 1000
    off = offsets_for(lengths, start)
    n = int(off[-1]) + 777
    a = inputs.u64(n, "uniform")
    t = to_dev(a)
    d_off = torch.from_numpy(off.view(np.int64).copy()).cuda()
    ips4o.sort_segmented(t, d_off, "u64")
    got = to_host(t, a)
    assert np.array_equal(got[:start], a[:start])
    assert np.array_equal(got[int(off[-1]):], a[int(off[-1]):])
    check_segments(got, a, off, "u64")


def test_segmented_equals_each_segment_sorted_alone(ips4o, mode):
    lengths = inputs.log_uniform_lengths(300, 4, 19)
    off = offsets_for(lengths)
    a = inputs.pair(int(off[-1]), "eight_dup")
    t = to_dev(a)
    ips4o.sort_segmented(t, off, "pair")
    got = to_host(t, a)
    for i in range(len(off) - 1):
        lo, hi = int(off[i]), int(off[i + 1])
        s = to_dev(a[lo:hi])
        ips4o.sort(s, "pair")
        alone = to_host(s, a[lo:hi])
        assert np.array_equal(got[lo:hi]["key"], alone["key"])
        assert np.array_equal(np.sort(got[lo:hi], order=["key", "payload"]),
                              np.sort(alone, order=["key", "payload"]))


def test_segmented_all_large_segments(ips4o, mode):
    lengths = np.array([300_001, 1 << 20, 65_536, 2_000_000, 500_000], dtype=np.uint64)
    off = offsets_for(lengths)
    a = inputs.u64(int(off[-1]), "exponential")
    t = to_dev(a)
    ips4o.sort_segmented(t, off, "u64")
    check_segments(to_host(t, a), a, off, "u64")
    st = ips4o.stats()
    assert st["n"] == int(off[-1])
    assert st["levels"] >= 1


@pytest.mark.parametrize("k_max,bcm", [(16, 64), (256, 100)])
def test_segmented_deep_recursion(ips4o, k_max, bcm):
    ips4o.set_params(k_max=k_max, base_case_max=bcm, segment_scheduler=1)
    try:
        lengths = inputs.log_uniform_lengths(200, 4, 16)
        off = offsets_for(lengths)
        a = inputs.u64(int(off[-1]), "uniform")
        t = to_dev(a)
        ips4o.sort_segmented(t, off, "u64")
        check_segments(to_host(t, a), a, off, "u64")
    finally:
        ips4o.reset_params()


def test_batched_separate_arrays_with_gaps(ips4o, mode):
    """Arrays carved out of one allocation with gaps between them, passed
    in a shuffled order: the gaps keep their bytes."""
    lengths = inputs.log_uniform_lengths(120, 4, 18)
    gap = 37
    starts = np.concatenate([[0], np.cumsum(lengths + gap)])[:-1].astype(np.int64)
    n = int(starts[-1] + lengths[-1] + gap)
    a = inputs.u64(n, "root_dup")
    big = torch.from_numpy(a.view(np.int64).copy()).cuda()
    views = [big[int(s):int(s) + int(L)] for s, L in zip(starts, lengths)]
    order = np.random.default_rng(5).permutation(len(views))
    ips4o.sort_batched([views[i] for i in order], "u64")
    got = big.cpu().numpy().view(np.uint64)
    mask = np.ones(n, dtype=bool)
    for s, L in zip(starts, lengths):
        s, L = int(s), int(L)
        mask[s:s + L] = False
        assert np.array_equal(got[s:s + L], oracle.sort(a[s:s + L], "u64"))
    assert np.array_equal(got[mask], a[mask])


def test_batched_device_tables_and_empty_arrays(ips4o, mode):
    arrs = [to_dev(inputs.f64(L, seed=10 + i)) for i, L in enumerate([0, 5, 100_000, 0, 20_000])]
    ptrs = torch.tensor([x.data_ptr() for x in arrs], dtype=torch.int64).cuda()
    lens = torch.tensor([x.numel() // 8 for x in arrs], dtype=torch.int64).cuda()
    rc = ips4o.ips4o_sort_batched(ptrs.data_ptr(), lens.data_ptr(), len(arrs), ips4o.F64,
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    for i, L in enumerate([0, 5, 100_000, 0, 20_000]):
        a = inputs.f64(L, seed=10 + i)
        got = to_host(arrs[i], a)
        assert np.array_equal(got.view(np.uint64), oracle.sort(a, "f64").view(np.uint64))


def test_segmented_and_batched_argument_errors(ips4o):
    t = torch.zeros(1000, dtype=torch.int64).cuda()
    bad = np.array([0, 500, 400, 1000], dtype=np.uint64)             # decreasing
    assert ips4o.ips4o_sort_segmented(t.data_ptr(), bad.ctypes.data, 3, ips4o.U64, 0) == 1
    assert ips4o.ips4o_sort_segmented(t.data_ptr(), bad.ctypes.data, 3, 17, 0) == 2
    assert ips4o.ips4o_sort_segmented(t.data_ptr() + 4, bad.ctypes.data, 3, ips4o.U64, 0) == 3
    ptrs = np.array([t.data_ptr(), t.data_ptr() + 8 * 100], dtype=np.uint64)
    lens = np.array([200, 100], dtype=np.uint64)                      # overlapping arrays
    assert ips4o.ips4o_sort_batched(ptrs.ctypes.data, lens.ctypes.data, 2, ips4o.U64, 0) == 1
    ptrs = np.array([t.data_ptr() + 4], dtype=np.uint64)
    assert ips4o.ips4o_sort_batched(ptrs.ctypes.data, lens.ctypes.data, 1, ips4o.U64, 0) == 3
    assert ips4o.ips4o_stream_status(0) == 0
    # nothing was touched
    assert int(t.abs().sum().item()) == 0


def test_streams_run_side_by_side(ips4o):
    """Calls on two streams from two host threads (separate workspaces)
    give the same results as calls made one after the other."""
    import threading
    arrays = [inputs.u64(3_000_017, "uniform", seed=21), inputs.u64(2_500_000, "two_dup", seed=22)]
    tens = [to_dev(a) for a in arrays]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    errors = []

    def work(i):
        try:
            with torch.cuda.stream(streams[i]):
                for _ in range(3):
                    ips4o.sort(tens[i], "u64")
        except Exception as e:          # reported below
            errors.append(e)

    th = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors
    for a, t in zip(arrays, tens):
        assert np.array_equal(to_host(t, a), oracle.sort(a, "u64"))


def test_scheduler_heavy_duplicates_and_deep_segments(ips4o):
    """The segment scheduler on arrays whose buckets need further
    distribution steps by the same CTA (Exponential keys leave some buckets
    above the base case) and on arrays of one repeated key."""
    ips4o.set_params(segment_scheduler=2)
    try:
        lengths = np.array([4_000_000, 1 << 20, 300_000, 70_001, 16_385, 9, 2_000_000], dtype=np.uint64)
        off = offsets_for(lengths)
        for dist in ("exponential", "ones", "two_dup", "root_dup"):
            a = inputs.u64_segments(lengths, dist)
            t = to_dev(a)
            ips4o.sort_segmented(t, off, "u64")
            check_segments(to_host(t, a), a, off, "u64")
    finally:
        ips4o.reset_params()


def _async_sort(ips4o, t, d_off, nseg, kt, stream):
    rc = ips4o.ips4o_sort_segmented_async(t.data_ptr(), d_off.data_ptr(), nseg, ips4o.KEY_TYPES[kt],
                                          stream.cuda_stream)
    assert rc == 0, ips4o.STATUS.get(rc)


@pytest.mark.parametrize("kt,dist", [("u64", "uniform"), ("pair", "two_dup"), ("f64", "exponential")])
def test_segmented_async_and_stream_status(ips4o, kt, dist):
    lengths = inputs.log_uniform_lengths(700, 4, 18)
    off = offsets_for(lengths)
    a = inputs.make(kt, int(off[-1]), dist)
    t = to_dev(a)
    d_off = torch.from_numpy(off.view(np.int64).copy()).cuda()
    stream = torch.cuda.Stream()
    # nothing reserved on this stream yet: refused before any work
    assert ips4o.ips4o_sort_segmented_async(t.data_ptr(), d_off.data_ptr(), len(lengths),
                                            ips4o.KEY_TYPES[kt], stream.cuda_stream) == 8
    assert ips4o.ips4o_reserve_workspace(int(off[-1]), len(lengths), ips4o.KEY_TYPES[kt], stream.cuda_stream) == 0
    torch.cuda.synchronize()
    _async_sort(ips4o, t, d_off, len(lengths), kt, stream)
    assert ips4o.ips4o_stream_status(stream.cuda_stream) == 0
    check_segments(to_host(t, a), a, off, kt)


@pytest.mark.parametrize("dist", ["uniform", "two_dup", "exponential"])
def test_segmented_async_deep_recursion(ips4o, dist):
    # a base case of 64 keys and 4 buckets per step: many levels planned on the
    # device, and subproblems the enqueued rounds leave go to the segment
    # scheduler; every segment equals the oracle's sort of it
    lengths = inputs.log_uniform_lengths(300, 4, 17)
    off = offsets_for(lengths)
    a = inputs.make("u64", int(off[-1]), dist)
    t = to_dev(a)
    d_off = torch.from_numpy(off.view(np.int64).copy()).cuda()
    stream = torch.cuda.Stream()
    ips4o.set_params(base_case_max=64, k_max=4)
    try:
        assert ips4o.ips4o_reserve_workspace(int(off[-1]), len(lengths), ips4o.U64, stream.cuda_stream) == 0
        torch.cuda.synchronize()
        _async_sort(ips4o, t, d_off, len(lengths), "u64", stream)
        assert ips4o.ips4o_stream_status(stream.cuda_stream) == 0
    finally:
        ips4o.reset_params()
    check_segments(to_host(t, a), a, off, "u64")


def test_segmented_async_more_keys_than_reserved(ips4o):
    # the level queues are sized for the reserved total: segments holding
    # more keys than that are reported as an internal error by
    # ips4o_stream_status (no fault); a later call within the reservation works
    lengths = np.full(64, 40_000, dtype=np.uint64)
    off = offsets_for(lengths)
    a = inputs.make("u64", int(off[-1]), "uniform")
    t = to_dev(a)
    d_off = torch.from_numpy(off.view(np.int64).copy()).cuda()
    stream = torch.cuda.Stream()
    assert ips4o.ips4o_reserve_workspace(100_000, len(lengths), ips4o.U64, stream.cuda_stream) == 0
    torch.cuda.synchronize()
    _async_sort(ips4o, t, d_off, len(lengths), "u64", stream)
    assert ips4o.ips4o_stream_status(stream.cuda_stream) == 7
    assert ips4o.ips4o_reserve_workspace(int(off[-1]), len(lengths), ips4o.U64, stream.cuda_stream) == 0
    t = to_dev(a)
    _async_sort(ips4o, t, d_off, len(lengths), "u64", stream)
    assert ips4o.ips4o_stream_status(stream.cuda_stream) == 0
    check_segments(to_host(t, a), a, off, "u64")


def test_segmented_async_reports_decreasing_offsets(ips4o):
    t = torch.zeros(1000, dtype=torch.int64).cuda()
    off = torch.tensor([0, 500, 400, 1000], dtype=torch.int64).cuda()
    stream = torch.cuda.Stream()
    assert ips4o.ips4o_reserve_workspace(1000, 3, ips4o.U64, stream.cuda_stream) == 0
    torch.cuda.synchronize()
    assert ips4o.ips4o_sort_segmented_async(t.data_ptr(), off.data_ptr(), 3, ips4o.U64, stream.cuda_stream) == 0
    assert ips4o.ips4o_stream_status(stream.cuda_stream) == 7


def test_segmented_async_in_a_cuda_graph(ips4o):
    """Captured once into a CUDA graph, replayed on new contents of the same
    buffers: every replay sorts every array."""
    lengths = inputs.log_uniform_lengths(2000, 4, 16)
    off = offsets_for(lengths)
    n = int(off[-1])
    t = torch.zeros(n, dtype=torch.int64, device="cuda")
    d_off = torch.from_numpy(off.view(np.int64).copy()).cuda()
    stream = torch.cuda.Stream()
    assert ips4o.ips4o_reserve_workspace(n, len(lengths), ips4o.U64, stream.cuda_stream) == 0
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        _async_sort(ips4o, t, d_off, len(lengths), "u64", stream)
    for seed in (31, 32, 33):
        a = inputs.u64_segments(lengths, "uniform", seed=seed)
        t.copy_(torch.from_numpy(a.view(np.int64)))
        g.replay()
        torch.cuda.synchronize()
        check_segments(t.cpu().numpy().view(np.uint64), a, off, "u64")
    assert ips4o.ips4o_stream_status(stream.cuda_stream) == 0
