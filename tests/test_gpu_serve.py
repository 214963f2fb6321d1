"""The continuous-batching sort service on the GPU.

A burst of requests of mixed key types and distributions goes through the
service under an HBM budget far smaller than the burst, so that requests
wait for memory, are admitted while others are on the device, and are
sorted in batches on several streams.  Every result must equal the oracle's
sort of the request's input and the result of sorting the same request alone
(keys bit for bit; for pairs also the (key, payload) multiset).
"""
import numpy as np
import pytest

import oracle
from paper_1705_02257_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DTYPES = {"u64": np.uint64, "f64": np.float64, "pair": inputs.PAIR_DTYPE}


@pytest.fixture(scope="module")
def serve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_02257_gb300 import build
    build.build()
    from paper_1705_02257_gb300 import ips4o, serve as s
    ips4o.reset_params()
    return s


def _pools(hi):
    pools = {}
    for kt in ("u64", "f64", "pair"):
        for d in inputs.DISTRIBUTIONS:
            a = inputs.make(kt, hi, d)
            pools[kt, d] = (a, torch.from_numpy(a.view(np.uint8).reshape(-1).copy()).cuda())
    return pools


def _requests(serve, count, lo, hi, rate):
    sizes, types, dists, arr = inputs.request_stream(count, lo, hi, rate)
    reqs = [serve.Request(i, types[i], int(sizes[i]), float(arr[i])) for i in range(count)]
    return reqs, dists


def _host(r):
    return r.buf.cpu().numpy().view(DTYPES[r.key_type])


@pytest.mark.parametrize("rate", [5000.0, 1e9])
def test_service_results_equal_alone_and_oracle(serve, rate):
    lo, hi = 10, 18
    pools = _pools(1 << hi)
    reqs, dists = _requests(serve, 240, lo, hi, rate)
    dist_of = {r.rid: dists[r.rid] for r in reqs}

    def fill(r, buf):
        buf.copy_(pools[r.key_type, dist_of[r.rid]][1][: r.nbytes])

    # 4 MiB for resident requests (the budget left after the workspaces)
    srv = serve.SortServer(budget_bytes=1 << 40, workers=3, max_batch_requests=16, max_batch_keys=1 << 20)
    srv.budget = 4 << 20
    mixed = srv.run(reqs, fill, keep=lambda r: True)
    summary = serve.summarize(mixed)
    assert summary["all_sorted"]
    assert all(r.t_done >= r.t_start >= r.t_admit >= r.arrival for r in mixed)
    # the budget made requests wait for memory, and batches overlapped
    assert max(r.t_admit - r.arrival for r in mixed) > 0
    alone, _ = _requests(serve, 240, lo, hi, rate)
    srv.run_one_at_a_time(alone, fill, keep=lambda r: True)
    for m, a in zip(mixed, alone):
        assert m.rid == a.rid
        src = pools[m.key_type, dist_of[m.rid]][0][: m.n]
        gm, ga = _host(m), _host(a)
        exp = oracle.sort(src, m.key_type)
        if m.key_type == "pair":
            assert np.array_equal(gm["key"], exp["key"]) and np.array_equal(ga["key"], exp["key"])
            ms = np.sort(gm, order=["key", "payload"])
            assert np.array_equal(ms, np.sort(ga, order=["key", "payload"]))
            assert np.array_equal(ms, np.sort(src, order=["key", "payload"]))
        else:
            assert np.array_equal(gm.view(np.uint64), exp.view(np.uint64)), (m.rid, m.key_type, m.n)
            assert np.array_equal(gm.view(np.uint64), ga.view(np.uint64))


def test_service_rejects_request_larger_than_budget(serve):
    srv = serve.SortServer(budget_bytes=1 << 40, workers=1, max_batch_requests=4, max_batch_keys=1 << 16)
    srv.budget = 1024
    r = serve.Request(0, "u64", 4096, 0.0)
    with pytest.raises(ValueError):
        srv.run([r], lambda r, buf: buf.zero_())
