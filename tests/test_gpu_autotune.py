"""The autotuner of the distribution step per size class (GPU): it returns a
valid table, installs it, and the sort with the tuned table still matches
the oracle."""
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
    m.ips4o_set_class_params(None)


def test_autotune_small_classes_and_sort_with_table(ips4o):
    from paper_1705_02257_gb300 import autotune
    res = autotune.tune("u64", classes=range(14, 17), batch_keys=1 << 21, reps=1, leaves=(8, 32, 128),
                        alphas=(8, 16))
    table = res["table"]
    assert len(table) == ips4o.NUM_CLASSES
    for c, (L, a) in enumerate(table):
        if L:
            assert c in res["results"] and L in (8, 32, 128) and a in (8, 16)
    assert ips4o.ips4o_get_class_params() == [tuple(x) for x in table]
    # sorting with the tuned table installed: both segmented forms and a plain sort
    lengths = inputs.log_uniform_lengths(300, 10, 17)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.uint64)
    a = inputs.u64(int(off[-1]), "exponential")
    for mode in (1, 2):
        ips4o.set_params(segment_scheduler=mode)
        t = torch.from_numpy(a.view(np.int64).copy()).cuda()
        ips4o.sort_segmented(t, off, "u64")
        got = t.cpu().numpy().view(np.uint64)
        for i in range(len(lengths)):
            lo, hi = int(off[i]), int(off[i + 1])
            assert np.array_equal(got[lo:hi], oracle.sort(a[lo:hi], "u64"))
    ips4o.reset_params()
    b = inputs.u64(100_003, "two_dup")
    t = torch.from_numpy(b.view(np.int64).copy()).cuda()
    ips4o.sort(t, "u64")
    assert np.array_equal(t.cpu().numpy().view(np.uint64), oracle.sort(b, "u64"))
    assert ips4o.ips4o_set_class_params(None) == 0
    assert all(x == (0, 0) for x in ips4o.ips4o_get_class_params())
