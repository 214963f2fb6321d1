"""Failure detection without a GPU fault.

Every device-side wait of the sort is a bounded poll that, when it runs out,
records IPS4O_ERR_TIMEOUT in a status word instead of hanging.  These tests
make waits run out on purpose -- a flag that nothing sets, and a poll limit
of one -- and check that the error comes back and the context stays usable;
and they inject a failure on the host into the sort service.
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
    yield m
    m.reset_params()


def _sort_ok(ips4o, a):
    t = torch.from_numpy(a.view(np.int64).copy()).cuda()
    ips4o.sort(t, "u64")
    torch.cuda.synchronize()
    return np.array_equal(t.cpu().numpy().view(np.uint64), oracle.sort(a, "u64"))


def test_wait_on_a_flag_nothing_sets_times_out(ips4o):
    stream = torch.cuda.Stream()
    for limit in (0, 10, 100_000):
        assert ips4o.ips4o_check_bounded_wait(limit, stream.cuda_stream) == 6      # IPS4O_ERR_TIMEOUT
    # the context is still usable
    assert _sort_ok(ips4o, inputs.u64(1_000_003, "uniform"))


@pytest.mark.parametrize("dist", ["root_dup", "two_dup", "uniform"])
def test_tiny_poll_limit_reports_or_completes(ips4o, dist):
    """With one poll per wait, a sort either completes correctly (no wait
    was needed) or reports IPS4O_ERR_TIMEOUT through the stream status; it
    never hangs.  ips4o_sort only enqueues, so the device-side outcome is
    read with ips4o_stream_status."""
    a = inputs.u64(3_000_017, dist)
    ips4o.set_params(spin_limit=1)
    try:
        t = torch.from_numpy(a.view(np.int64).copy()).cuda()
        stream = torch.cuda.current_stream().cuda_stream
        rc = ips4o.ips4o_sort(t.data_ptr(), len(a), ips4o.U64, stream)
        assert rc == 0, ips4o.STATUS.get(rc)
        rc = ips4o.ips4o_stream_status(stream)
        assert rc in (0, 6), ips4o.STATUS.get(rc)
        if rc == 0:
            assert np.array_equal(t.cpu().numpy().view(np.uint64), oracle.sort(a, "u64"))
    finally:
        ips4o.reset_params()
    assert _sort_ok(ips4o, a)


def test_service_propagates_a_host_failure(ips4o):
    from paper_1705_02257_gb300 import serve
    srv = serve.SortServer(budget_bytes=1 << 40, workers=2, max_batch_requests=4, max_batch_keys=1 << 18)
    reqs = [serve.Request(i, "u64", 5000 + i, 0.0) for i in range(40)]

    def fill(r, buf):
        if r.rid == 17:
            raise RuntimeError("injected input failure")
        buf.copy_(torch.from_numpy(inputs.u64(r.n, "uniform", seed=r.rid + 1).view(np.uint8)).cuda())

    with pytest.raises(RuntimeError, match="injected"):
        srv.run(reqs, fill)
    # the service object still works afterwards
    ok = [serve.Request(i, "u64", 3000, 0.0) for i in range(8)]
    srv.run(ok, lambda r, buf: buf.copy_(torch.from_numpy(inputs.u64(3000, seed=r.rid + 1).view(np.uint8)).cuda()))
    assert all(r.sorted_ok for r in ok)
