"""The C-ABI library builds, loads and exports every entry point that
include/ips4o.h declares; argument errors are reported before any device
work (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ips4o.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(ips4o_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_02257_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared_functions()
    for expected in ("ips4o_sort", "ips4o_sort_host", "ips4o_partition", "ips4o_workspace_bytes",
                     "ips4o_get_stats", "ips4o_status_string"):
        assert expected in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared in ips4o.h but not exported: {missing}"


def test_argument_errors_without_device_work(lib):
    from paper_1705_02257_gb300 import ips4o
    assert ips4o.ips4o_sort(0, 10, ips4o.U64, 0) == 1          # null pointer, n > 0
    assert ips4o.ips4o_sort(0, 10, 17, 0) == 2                  # unknown key type
    assert ips4o.ips4o_sort(8 * 1024 + 4, 10, ips4o.U64, 0) == 3  # misaligned
    assert ips4o.ips4o_sort(8 * 1024 + 2, 10, ips4o.REC100_K10, 0) == 3   # records: 4-byte alignment
    assert ips4o.ips4o_sort(0, 0, ips4o.U64, 0) == 0            # empty input: no-op
    assert ips4o.ips4o_sort(0, 1, ips4o.U64, 0) == 0
    # more than 16 GiB of elements in one call (the packed pointer word's
    # region limit): refused before any device work
    assert ips4o.ips4o_sort(8 * 1024, (16 << 30) // 8 + 1, ips4o.U64, 0) == 8
    assert ips4o.ips4o_sort(16 * 1024, (16 << 30) // 16 + 1, ips4o.PAIR_U64, 0) == 8
    assert ips4o.ips4o_sort_host(8 * 1024, (16 << 30) // 8 + 1, ips4o.U64, 0) == 8
    assert ips4o.ips4o_status_string(6) == "bounded device wait timed out"


def test_params_validation(lib):
    from paper_1705_02257_gb300 import ips4o
    p = ips4o.ips4o_get_params()
    assert p.k_max == 256
    bad = ips4o.Params(100, 0, 0, 2, 0, 1)      # k_max not a power of two
    assert ips4o.ips4o_set_params(bad) == 1
    assert ips4o.ips4o_get_params().k_max == 256


def test_base_case_capacity(lib):
    from paper_1705_02257_gb300 import ips4o
    assert ips4o.ips4o_base_case_capacity(ips4o.U64) == 16384
    assert ips4o.ips4o_base_case_capacity(ips4o.PAIR_U64) == 8192


def test_class_params_validation(lib):
    from paper_1705_02257_gb300 import ips4o
    before = ips4o.ips4o_get_class_params()
    assert ips4o.ips4o_set_class_params([(100, 1)]) == 1       # leaves not a power of two
    assert ips4o.ips4o_set_class_params([(2, 1)]) == 1         # fewer than 4 leaves
    assert ips4o.ips4o_set_class_params([(256, 17)]) == 1      # alpha * leaves > 4096
    assert ips4o.ips4o_get_class_params() == before            # rejected tables change nothing


def test_strict_workspace_is_independent_of_n(lib):
    """Section 4.6: the strictly in-place sort keeps no list whose length
    depends on n, so its workspace is the same for every n above the base
    case (host computation, no GPU needed)."""
    lib.ips4o_workspace_bytes_strict.restype = ctypes.c_size_t
    lib.ips4o_workspace_bytes_strict.argtypes = [ctypes.c_size_t, ctypes.c_int]
    for kt in (0, 1, 2, 3, 4):
        w = [lib.ips4o_workspace_bytes_strict(1 << k, kt) for k in (27, 28, 30, 33)]
        assert len(set(w)) == 1 and w[0] > 0, (kt, w)
        # and no larger than the device-planned sort's at 2^28 (u64, f64, pair,
        # quartet; records there go through key + index pairs)
        if kt != 3:
            assert w[0] <= lib.ips4o_workspace_bytes(1 << 28, kt), (kt, w[0])


def test_workspace_is_sublinear_in_n(lib):
    """Theorem 2: the extra space of the sort is O(k b t + log_k(n / n0)).
    Here t is a fixed number of stripes per SM, so the leftover pool and the
    per-chunk tables do not grow with n; only the two level queues grow, by
    n / (base-case size) task entries of 16 bytes each (computed on the host,
    no GPU needed; 152 SMs when no device is present)."""
    lib.ips4o_workspace_bytes.restype = ctypes.c_size_t
    lib.ips4o_workspace_bytes.argtypes = [ctypes.c_size_t, ctypes.c_int]
    for kt, s, cap in ((0, 8, 16384), (1, 8, 16384), (2, 16, 8192)):
        w = {k: lib.ips4o_workspace_bytes(1 << k, kt) for k in (24, 26, 28, 30)}
        for k in (26, 28, 30):
            queues = 4 * 16 * ((1 << k) - (1 << 24)) // (cap + 1)     # two queues, the fallback list (2x)
            assert w[k] - w[24] <= queues + 4096, (kt, k, w)
        # at 2^28 elements: well below 5% of the input
        assert w[28] < 0.05 * (1 << 28) * s, (kt, w[28])
