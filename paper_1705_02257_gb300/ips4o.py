"""Thin ctypes binding of ``libips4o_gb300.so`` (declared in include/ips4o.h).

The functions named ``ips4o_*`` mirror the C entry points one to one and
only marshal arguments; every step of the sort runs in the library's CUDA
kernels.  ``sort``/``partition`` are conveniences that take a torch CUDA
tensor and pass its pointer, size and the current stream.

There is no fallback: if the library is missing or fails to load, importing
this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# IPS4O_LIBRARY names another build of the same library (e.g. one compiled
# with different tuning constants); by default the in-tree build is loaded.
LIB_PATH = os.environ.get("IPS4O_LIBRARY") or os.path.join(_HERE, "libips4o_gb300.so")

U64, F64, PAIR_U64, REC100_K10, QUARTET_U64 = 0, 1, 2, 3, 4
KEY_TYPES = {"u64": U64, "f64": F64, "pair": PAIR_U64, "rec100": REC100_K10, "quartet": QUARTET_U64}
ELEM_SIZE = {U64: 8, F64: 8, PAIR_U64: 16, REC100_K10: 100, QUARTET_U64: 32}

STATUS = {
    0: "IPS4O_OK", 1: "IPS4O_ERR_INVALID_ARG", 2: "IPS4O_ERR_UNSUPPORTED_TYPE",
    3: "IPS4O_ERR_MISALIGNED", 4: "IPS4O_ERR_OOM", 5: "IPS4O_ERR_CUDA",
    6: "IPS4O_ERR_TIMEOUT", 7: "IPS4O_ERR_INTERNAL", 8: "IPS4O_ERR_TOO_LARGE",
}
PHASES = ("sample", "classify", "prefix", "empty_block_fix", "block_permutation",
          "cleanup", "base_case", "other")


class Ips4oError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = f"{where}: {STATUS.get(status, status)}"
        if status in (5, 6, 7):
            detail = last_cuda_error()
            if detail:
                msg += f" ({detail})"
        super().__init__(msg)
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int), ("alpha", ctypes.c_int), ("base_case_max", ctypes.c_int),
                ("stripes_per_sm", ctypes.c_int), ("profile", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("segment_scheduler", ctypes.c_int), ("spin_limit", ctypes.c_uint32), ("record_path", ctypes.c_int),
                ("strict_window", ctypes.c_uint64)]


class ClassParams(ctypes.Structure):
    _fields_ = [("leaves", ctypes.c_uint16), ("alpha", ctypes.c_uint16)]


NUM_CLASSES = 64


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("levels", ctypes.c_uint32), ("chunks", ctypes.c_uint32),
                ("subproblems", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("blocks_moved", ctypes.c_uint64), ("blocks_skipped", ctypes.c_uint64),
                ("fix_blocks_moved", ctypes.c_uint64), ("base_case_buckets", ctypes.c_uint64),
                ("elements_distributed", ctypes.c_uint64), ("workspace_bytes", ctypes.c_uint64),
                ("phase_ms", ctypes.c_double * 8), ("phase_launches", ctypes.c_uint64 * 8)]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_ if name not in ("phase_ms", "phase_launches")}
        d["phase_ms"] = {p: self.phase_ms[i] for i, p in enumerate(PHASES)}
        d["phase_launches"] = {p: int(self.phase_launches[i]) for i, p in enumerate(PHASES)}
        return d


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    vp, sz, i32, u64p = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)
    lib.ips4o_sort.restype = i32
    lib.ips4o_sort.argtypes = [vp, sz, i32, vp]
    lib.ips4o_sort_strict.restype = i32
    lib.ips4o_sort_strict.argtypes = [vp, sz, i32, vp]
    lib.ips4o_workspace_bytes_strict.restype = sz
    lib.ips4o_workspace_bytes_strict.argtypes = [sz, i32]
    lib.ips4o_sort_host.restype = i32
    lib.ips4o_sort_host.argtypes = [vp, sz, i32, vp]
    lib.ips4o_sort_noalloc.restype = i32
    lib.ips4o_sort_noalloc.argtypes = [vp, sz, i32, vp]
    lib.ips4o_sort_segmented.restype = i32
    lib.ips4o_sort_segmented.argtypes = [vp, vp, sz, i32, vp]
    lib.ips4o_sort_segmented_async.restype = i32
    lib.ips4o_sort_segmented_async.argtypes = [vp, vp, sz, i32, vp]
    lib.ips4o_sort_batched.restype = i32
    lib.ips4o_sort_batched.argtypes = [vp, vp, sz, i32, vp]
    lib.ips4o_stream_status.restype = i32
    lib.ips4o_stream_status.argtypes = [vp]
    lib.ips4o_partition.restype = i32
    lib.ips4o_partition.argtypes = [vp, sz, i32, vp, vp, ctypes.POINTER(sz), vp, ctypes.POINTER(sz),
                                    ctypes.POINTER(i32)]
    lib.ips4o_workspace_bytes.restype = sz
    lib.ips4o_workspace_bytes.argtypes = [sz, i32]
    lib.ips4o_reserve_workspace.restype = i32
    lib.ips4o_reserve_workspace.argtypes = [sz, sz, i32, vp]
    lib.ips4o_release_workspace.restype = i32
    lib.ips4o_release_workspace.argtypes = []
    lib.ips4o_set_params.restype = i32
    lib.ips4o_set_params.argtypes = [ctypes.POINTER(Params)]
    lib.ips4o_get_params.restype = i32
    lib.ips4o_get_params.argtypes = [ctypes.POINTER(Params)]
    lib.ips4o_set_class_params.restype = i32
    lib.ips4o_set_class_params.argtypes = [ctypes.POINTER(ClassParams), sz]
    lib.ips4o_get_class_params.restype = i32
    lib.ips4o_get_class_params.argtypes = [ctypes.POINTER(ClassParams), sz]
    lib.ips4o_get_stats.restype = i32
    lib.ips4o_get_stats.argtypes = [ctypes.POINTER(Stats)]
    lib.ips4o_base_case_capacity.restype = sz
    lib.ips4o_base_case_capacity.argtypes = [i32]
    lib.ips4o_status_string.restype = ctypes.c_char_p
    lib.ips4o_status_string.argtypes = [i32]
    lib.ips4o_check_bounded_wait.restype = i32
    lib.ips4o_check_bounded_wait.argtypes = [ctypes.c_uint32, vp]
    lib.ips4o_last_cuda_error.restype = ctypes.c_char_p
    lib.ips4o_last_cuda_error.argtypes = []
    return lib


_lib = _load()


def lib():
    return _lib


# ------------------------------------------------------ C ABI, same names
def ips4o_sort(d_ptr: int, n: int, key_type: int, stream: int = 0) -> int:
    return _lib.ips4o_sort(d_ptr, n, key_type, stream)


def ips4o_sort_strict(d_ptr: int, n: int, key_type: int, stream: int = 0) -> int:
    return _lib.ips4o_sort_strict(d_ptr, n, key_type, stream)


def ips4o_workspace_bytes_strict(n: int, key_type: int) -> int:
    return _lib.ips4o_workspace_bytes_strict(n, key_type)


def ips4o_sort_host(h_ptr: int, n: int, key_type: int, stream: int = 0) -> int:
    return _lib.ips4o_sort_host(h_ptr, n, key_type, stream)


def ips4o_sort_noalloc(d_ptr: int, n: int, key_type: int, stream: int = 0) -> int:
    """The sort without any memory allocation (fixed scratch, n <= 2^20)."""
    return _lib.ips4o_sort_noalloc(d_ptr, n, key_type, stream)


def ips4o_sort_segmented(d_base: int, offsets: int, num_segments: int, key_type: int, stream: int = 0) -> int:
    """offsets: address of num_segments + 1 uint64 element indices (host or device)."""
    return _lib.ips4o_sort_segmented(d_base, offsets, num_segments, key_type, stream)


def ips4o_sort_segmented_async(d_base: int, d_offsets: int, num_segments: int, key_type: int, stream: int = 0) -> int:
    """Enqueue-only segmented sort (device offsets; reserve the workspace first)."""
    return _lib.ips4o_sort_segmented_async(d_base, d_offsets, num_segments, key_type, stream)


def ips4o_sort_batched(ptrs: int, lens: int, count: int, key_type: int, stream: int = 0) -> int:
    """ptrs, lens: addresses of `count` device pointers and uint64 lengths (host or device)."""
    return _lib.ips4o_sort_batched(ptrs, lens, count, key_type, stream)


def ips4o_stream_status(stream: int = 0) -> int:
    return _lib.ips4o_stream_status(stream)


def check(stream: int | None = None) -> None:
    """Wait for the stream and raise the device-side error of the last
    enqueue-only sort on it, if any (ips4o_stream_status)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    rc = ips4o_stream_status(stream)
    if rc:
        raise Ips4oError(rc, "ips4o_stream_status")


def ips4o_partition(d_ptr: int, n: int, key_type: int, stream: int = 0):
    """Returns (status, bounds, splitters, eq)."""
    bounds = np.zeros(257, dtype=np.uint64)
    spl = np.zeros(256, dtype=np.uint64)
    nb, ns, eq = ctypes.c_size_t(0), ctypes.c_size_t(0), ctypes.c_int(0)
    rc = _lib.ips4o_partition(d_ptr, n, key_type, stream, bounds.ctypes.data, ctypes.byref(nb),
                              spl.ctypes.data, ctypes.byref(ns), ctypes.byref(eq))
    return rc, bounds[: nb.value + 1].astype(np.int64), spl[: ns.value].copy(), bool(eq.value)


def ips4o_workspace_bytes(n: int, key_type: int) -> int:
    return int(_lib.ips4o_workspace_bytes(n, key_type))


def ips4o_reserve_workspace(n: int, num_segments: int, key_type: int, stream: int = 0) -> int:
    return _lib.ips4o_reserve_workspace(n, num_segments, key_type, stream)


def ips4o_release_workspace() -> int:
    return _lib.ips4o_release_workspace()


def ips4o_set_params(p: Params | None) -> int:
    return _lib.ips4o_set_params(ctypes.byref(p) if p is not None else None)


def ips4o_get_params() -> Params:
    p = Params()
    rc = _lib.ips4o_get_params(ctypes.byref(p))
    if rc:
        raise Ips4oError(rc, "ips4o_get_params")
    return p


def ips4o_set_class_params(table) -> int:
    """table: sequence of (leaves, alpha) per size class floor(log2 n), or None to reset."""
    if table is None:
        return _lib.ips4o_set_class_params(None, 0)
    arr = (ClassParams * NUM_CLASSES)()
    for c, (leaves, alpha) in enumerate(table):
        arr[c].leaves, arr[c].alpha = int(leaves), int(alpha)
    return _lib.ips4o_set_class_params(arr, len(table))


def ips4o_get_class_params():
    arr = (ClassParams * NUM_CLASSES)()
    rc = _lib.ips4o_get_class_params(arr, NUM_CLASSES)
    if rc:
        raise Ips4oError(rc, "ips4o_get_class_params")
    return [(arr[c].leaves, arr[c].alpha) for c in range(NUM_CLASSES)]


def ips4o_get_stats() -> Stats:
    s = Stats()
    rc = _lib.ips4o_get_stats(ctypes.byref(s))
    if rc:
        raise Ips4oError(rc, "ips4o_get_stats")
    return s


def ips4o_base_case_capacity(key_type: int) -> int:
    return int(_lib.ips4o_base_case_capacity(key_type))


def ips4o_status_string(status: int) -> str:
    return _lib.ips4o_status_string(status).decode()


def ips4o_check_bounded_wait(spin_limit: int, stream: int = 0) -> int:
    return _lib.ips4o_check_bounded_wait(spin_limit, stream)


def last_cuda_error() -> str:
    return _lib.ips4o_last_cuda_error().decode()


# -------------------------------------------------- torch conveniences
def _kt(key_type) -> int:
    return KEY_TYPES[key_type] if isinstance(key_type, str) else int(key_type)


def _count(t, kt: int) -> int:
    nbytes = t.numel() * t.element_size()
    if nbytes % ELEM_SIZE[kt]:
        raise ValueError("tensor size is not a whole number of elements of the key type")
    return nbytes // ELEM_SIZE[kt]


def _stream_of(t) -> int:
    import torch
    return torch.cuda.current_stream(t.device).cuda_stream


def sort(t, key_type="u64", stream: int | None = None):
    """Sort a contiguous CUDA tensor in place, viewing its bytes as elements
    of ``key_type`` ('u64', 'f64', 'pair', 'rec100').  For u64, f64 and
    pairs the call only enqueues the work on the stream (device-side errors:
    ``check(stream)``)."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    kt = _kt(key_type)
    n = _count(t, kt)
    rc = ips4o_sort(t.data_ptr(), n, kt, _stream_of(t) if stream is None else stream)
    if rc:
        raise Ips4oError(rc, "ips4o_sort")
    return t


def sort_strict(t, key_type="u64", stream: int | None = None):
    """Sort a contiguous CUDA tensor in place with extra memory independent
    of its size (Section 4.6); returns when the tensor is sorted."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    kt = _kt(key_type)
    n = _count(t, kt)
    rc = ips4o_sort_strict(t.data_ptr(), n, kt, _stream_of(t) if stream is None else stream)
    if rc:
        raise Ips4oError(rc, "ips4o_sort_strict")
    return t


def workspace_bytes_strict(n: int, key_type="u64") -> int:
    return ips4o_workspace_bytes_strict(n, _kt(key_type))


def sort_segmented(t, offsets, key_type="u64", stream: int | None = None):
    """Sort the segments t[offsets[i]:offsets[i+1]] of a contiguous CUDA
    tensor (viewed as elements of ``key_type``) independently, in place.
    ``offsets`` is a sequence or array of num_segments + 1 element indices
    (host memory) or a uint64/int64 CUDA tensor."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    kt = _kt(key_type)
    if hasattr(offsets, "is_cuda") and offsets.is_cuda:
        if offsets.element_size() != 8 or not offsets.is_contiguous():
            raise ValueError("offsets tensor must be contiguous 64-bit")
        addr, count, keep = offsets.data_ptr(), offsets.numel() - 1, offsets
    else:
        keep = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
        addr, count = keep.ctypes.data, len(keep) - 1
    if count < 0:
        raise ValueError("offsets needs at least one entry")
    if len(keep) and int(keep[-1]) > _count(t, kt):
        raise ValueError("segments extend past the tensor")
    rc = ips4o_sort_segmented(t.data_ptr(), addr, count, kt, _stream_of(t) if stream is None else stream)
    if rc:
        raise Ips4oError(rc, "ips4o_sort_segmented")
    return t


def sort_batched(tensors, key_type="u64", stream: int | None = None):
    """Sort each contiguous CUDA tensor of ``tensors`` in place, in one call."""
    kt = _kt(key_type)
    tensors = list(tensors)
    if not tensors:
        return tensors
    for t in tensors:
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("expected contiguous CUDA tensors")
    ptrs = np.array([t.data_ptr() for t in tensors], dtype=np.uint64)
    lens = np.array([_count(t, kt) for t in tensors], dtype=np.uint64)
    rc = ips4o_sort_batched(ptrs.ctypes.data, lens.ctypes.data, len(tensors), kt,
                            _stream_of(tensors[0]) if stream is None else stream)
    if rc:
        raise Ips4oError(rc, "ips4o_sort_batched")
    return tensors


def partition(t, key_type="u64", stream: int | None = None):
    """One distribution step in place; returns (bounds, splitters, eq)."""
    kt = _kt(key_type)
    n = _count(t, kt)
    rc, bounds, spl, eq = ips4o_partition(t.data_ptr(), n, kt, _stream_of(t) if stream is None else stream)
    if rc:
        raise Ips4oError(rc, "ips4o_partition")
    return bounds, spl, eq


def sort_host(a: np.ndarray, key_type="u64", stream: int = 0) -> np.ndarray:
    """Sort a host numpy array in place through the device."""
    kt = _kt(key_type)
    if not a.flags.c_contiguous:
        raise ValueError("expected a C-contiguous array")
    if a.nbytes % ELEM_SIZE[kt]:
        raise ValueError("array size is not a whole number of elements of the key type")
    rc = ips4o_sort_host(a.ctypes.data, a.nbytes // ELEM_SIZE[kt], kt, stream)
    if rc:
        raise Ips4oError(rc, "ips4o_sort_host")
    return a


def set_params(**kw) -> None:
    p = ips4o_get_params()
    for k, v in kw.items():
        setattr(p, k, v)
    rc = ips4o_set_params(p)
    if rc:
        raise Ips4oError(rc, "ips4o_set_params")


def reset_params() -> None:
    rc = _lib.ips4o_set_params(None)
    if rc:
        raise Ips4oError(rc, "ips4o_set_params")


def stats() -> dict:
    return ips4o_get_stats().as_dict()
