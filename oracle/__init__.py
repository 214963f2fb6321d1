"""CPU oracle for the IPS4o distribution path — TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never loads it and the
two share no code.  The arithmetic lives in ``ips4o_oracle.c`` (a plain
sequential samplesort, Sections 3, 4.4 and 4.7 of the paper), compiled with gcc
on first use; this file only marshals numpy arrays to it.

Key types: 'u64', 'f64', 'pair' (16-byte key/payload), 'rec100' (100-byte
record, 10-byte key compared as unsigned bytes), 'quartet' (32 bytes: three
64-bit key words compared lexicographically, one payload word).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

KEY_TYPES = {"u64": 0, "f64": 1, "pair": 2, "rec100": 3, "quartet": 4}
ELEM_SIZE = {"u64": 8, "f64": 8, "pair": 16, "rec100": 100, "quartet": 32}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ips4o_oracle.c")
_LIB = os.path.join(_HERE, "libips4o_oracle.so")
_lock = threading.Lock()
_lib = None


class OracleParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("n0", ctypes.c_int), ("alpha", ctypes.c_int),
                ("adaptive", ctypes.c_int), ("seed", ctypes.c_uint64)]


def build(force: bool = False, extra_flags: tuple = (), out: str | None = None) -> str:
    """Compile the oracle into a shared library next to its source."""
    target = out or _LIB
    if force or out or not os.path.exists(target) or os.path.getmtime(target) < os.path.getmtime(_SRC):
        tmp = target + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", *extra_flags, _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, target)
    return target


def _declare(lib):
    vp, sz, i32, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64
    pp = ctypes.POINTER(OracleParams)
    lib.oracle_sort.restype = i32
    lib.oracle_sort.argtypes = [vp, sz, i32, pp]
    lib.oracle_partition.restype = i32
    lib.oracle_partition.argtypes = [vp, sz, i32, pp, vp, vp, ctypes.POINTER(sz),
                                     ctypes.POINTER(i32), vp, ctypes.POINTER(sz), vp]
    lib.oracle_key.restype = None
    lib.oracle_key.argtypes = [vp, i32, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64)]
    lib.oracle_rank_counts.restype = i32
    lib.oracle_rank_counts.argtypes = [vp, sz, i32, vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
    lib.oracle_multiset_hash.restype = i32
    lib.oracle_multiset_hash.argtypes = [vp, sz, i32, vp]
    lib.oracle_is_sorted.restype = i32
    lib.oracle_is_sorted.argtypes = [vp, sz, i32]
    return lib


def load(path: str | None = None):
    """The oracle library (built on first use).  ``path`` (or the environment
    variable IPS4O_ORACLE_LIB) loads another build of the same source, e.g. a
    copy with a deliberately planted bug used to show that the pins catch it."""
    global _lib
    path = path or os.environ.get("IPS4O_ORACLE_LIB") or None
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _params(k=256, n0=16, alpha=0, adaptive=True, seed=0x1234567):
    return OracleParams(int(k), int(n0), int(alpha), 1 if adaptive else 0, int(seed))


def _kt(key_type: str) -> int:
    if key_type not in KEY_TYPES:
        raise ValueError(f"unknown key type {key_type!r}")
    return KEY_TYPES[key_type]


def _count(a: np.ndarray, key_type: str) -> int:
    if key_type == "rec100":
        return a.shape[0]
    return a.shape[0] if a.ndim else 0


def sort(a: np.ndarray, key_type: str = "u64", lib=None, **params) -> np.ndarray:
    """Return a sorted copy of ``a`` (the oracle's output)."""
    out = np.ascontiguousarray(a).copy()
    rc = (lib or load()).oracle_sort(out.ctypes.data, _count(out, key_type), _kt(key_type),
                                     ctypes.byref(_params(**params)))
    if rc != 0:
        raise RuntimeError(f"oracle_sort failed ({rc})")
    return out


def partition(a: np.ndarray, key_type: str = "u64", lib=None, **params):
    """One distribution step.  Returns (arranged copy, splitter keys as an
    (m, 3) uint64 array of (hi, lo, lo2) key words, equality flag, bucket
    bounds)."""
    out = np.ascontiguousarray(a).copy()
    k = params.get("k", 256)
    hi = np.zeros(k, dtype=np.uint64)
    lo = np.zeros(k, dtype=np.uint64)
    lo2 = np.zeros(k, dtype=np.uint64)
    bounds = np.zeros(2 * k + 2, dtype=np.uint64)
    m = ctypes.c_size_t(0)
    eq = ctypes.c_int(0)
    nb = ctypes.c_size_t(0)
    rc = (lib or load()).oracle_partition(out.ctypes.data, _count(out, key_type), _kt(key_type),
                                          ctypes.byref(_params(**params)), hi.ctypes.data,
                                          lo.ctypes.data, ctypes.byref(m), ctypes.byref(eq),
                                          bounds.ctypes.data, ctypes.byref(nb), lo2.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_partition failed ({rc})")
    spl = np.stack([hi[: m.value], lo[: m.value], lo2[: m.value]], axis=1)
    return out, spl, bool(eq.value), bounds[: nb.value + 1].astype(np.int64)


def keys(a: np.ndarray, key_type: str = "u64") -> np.ndarray:
    """Comparable keys of every element as an (n, 3) uint64 array of key
    words (hi, lo, lo2), compared lexicographically."""
    lib = load()
    n = _count(a, key_type)
    a = np.ascontiguousarray(a)
    raw = a.view(np.uint8).reshape(n, ELEM_SIZE[key_type]) if n else np.zeros((0, 1), np.uint8)
    out = np.zeros((n, 3), dtype=np.uint64)
    h, l_, l2 = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    for i in range(n):
        lib.oracle_key(raw[i].ctypes.data, _kt(key_type), ctypes.byref(h), ctypes.byref(l_), ctypes.byref(l2))
        out[i, 0], out[i, 1], out[i, 2] = h.value, l_.value, l2.value
    return out


def rank_counts(a: np.ndarray, key_type: str, elem) -> tuple[int, int]:
    """(#elements with key < key(elem), #elements with key <= key(elem))."""
    e = np.ascontiguousarray(elem)
    lt, le = ctypes.c_uint64(), ctypes.c_uint64()
    rc = load().oracle_rank_counts(np.ascontiguousarray(a).ctypes.data, _count(a, key_type),
                                   _kt(key_type), e.ctypes.data, ctypes.byref(lt), ctypes.byref(le))
    if rc != 0:
        raise RuntimeError("oracle_rank_counts failed")
    return lt.value, le.value


def multiset_hash(a: np.ndarray, key_type: str) -> tuple[int, int]:
    out = np.zeros(2, dtype=np.uint64)
    rc = load().oracle_multiset_hash(np.ascontiguousarray(a).ctypes.data, _count(a, key_type),
                                     _kt(key_type), out.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle_multiset_hash failed")
    return int(out[0]), int(out[1])


def is_sorted(a: np.ndarray, key_type: str) -> bool:
    return bool(load().oracle_is_sorted(np.ascontiguousarray(a).ctypes.data, _count(a, key_type),
                                        _kt(key_type)))
