"""Seeded synthetic inputs shaped like the paper's workloads (Section 5).

This module holds no arithmetic of the sorting method.  It is the one piece
shared by the CPU oracle's tests and the GPU path's tests and benchmarks:
both sort exactly the arrays it returns.  The generators are written in C
(``gen_inputs.c``, compiled on first use with gcc) so that 2^28-element
inputs take seconds, not minutes.

Distributions (Section 5): Uniform, Exponential, AlmostSorted, Sorted,
ReverseSorted, Ones, RootDup, TwoDup, EightDup.  Element types: 64-bit
unsigned keys, float64 keys, 16-byte (key, payload) pairs, and 100-byte
records whose first 10 bytes are the key (compared as unsigned bytes).
The exact definitions and seeds are documented in ``gen_inputs.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

DISTRIBUTIONS = (
    "uniform", "exponential", "almost_sorted", "sorted", "reverse_sorted",
    "ones", "root_dup", "two_dup", "eight_dup",
)
_DIST_ID = {name: i for i, name in enumerate(DISTRIBUTIONS)}

# Seeds: 1 input values, 2 AlmostSorted swaps, 3 payloads, 4 batch lengths,
# 5 arrival times, 6 and 7 the second and third key words of quartets.
SEED_VALUES, SEED_SWAPS, SEED_PAYLOAD, SEED_LENGTHS, SEED_ARRIVALS = 1, 2, 3, 4, 5
SEED_QUARTET_K1, SEED_QUARTET_K2 = 6, 7

PAIR_DTYPE = np.dtype([("key", "<u8"), ("payload", "<u8")])
QUARTET_DTYPE = np.dtype([("k0", "<u8"), ("k1", "<u8"), ("k2", "<u8"), ("payload", "<u8")])
REC100_DTYPE = np.dtype((np.void, 100))

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen_inputs.c")
_LIB = os.path.join(_HERE, "libips4o_inputs.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen_inputs.c into an in-tree shared library (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, u64p, i32 = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
            lib.gen_splitmix64_at.restype = u64
            lib.gen_splitmix64_at.argtypes = [u64, u64]
            for name in ("gen_u64", "gen_f64"):
                f = getattr(lib, name)
                f.restype = i32
                f.argtypes = [u64p, u64, i32, u64]
            lib.gen_pair.restype = i32
            lib.gen_pair.argtypes = [u64p, u64, i32, u64, u64]
            lib.gen_rec100.restype = i32
            lib.gen_rec100.argtypes = [u64p, u64, i32, u64, u64]
            lib.gen_splitmix64_range.restype = i32
            lib.gen_splitmix64_range.argtypes = [u64p, u64, u64, u64]
            lib.gen_u64_segments.restype = i32
            lib.gen_u64_segments.argtypes = [u64p, u64p, u64, i32, u64, u64]
            lib.gen_log_uniform_lengths.restype = i32
            lib.gen_log_uniform_lengths.argtypes = [u64p, u64, ctypes.c_double, ctypes.c_double, u64]
            _lib = lib
    return _lib


def _dist_id(dist: str) -> int:
    try:
        return _DIST_ID[dist]
    except KeyError:
        raise ValueError(f"unknown distribution {dist!r}; expected one of {DISTRIBUTIONS}") from None


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def splitmix64_at(seed: int, i: int) -> int:
    """Output i (0-based) of the SplitMix64 stream with the given seed."""
    return int(_load().gen_splitmix64_at(seed, i))


def u64(n: int, dist: str = "uniform", seed: int = SEED_VALUES) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _check(_load().gen_u64(out.ctypes.data, n, _dist_id(dist), seed), "gen_u64")
    return out


def f64(n: int, dist: str = "uniform", seed: int = SEED_VALUES) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _check(_load().gen_f64(out.ctypes.data, n, _dist_id(dist), seed), "gen_f64")
    return out


def pair(n: int, dist: str = "uniform", seed: int = SEED_VALUES,
         payload_seed: int = SEED_PAYLOAD) -> np.ndarray:
    out = np.empty(n, dtype=PAIR_DTYPE)
    _check(_load().gen_pair(out.ctypes.data, n, _dist_id(dist), seed, payload_seed), "gen_pair")
    return out


def rec100(n: int, dist: str = "uniform", seed: int = SEED_VALUES,
           payload_seed: int = SEED_PAYLOAD) -> np.ndarray:
    """n records as an (n, 100) uint8 array."""
    out = np.empty((n, 100), dtype=np.uint8)
    _check(_load().gen_rec100(out.ctypes.data, n, _dist_id(dist), seed, payload_seed), "gen_rec100")
    return out


def log_uniform_lengths(count: int, lo_log2: float, hi_log2: float,
                        seed: int = SEED_LENGTHS) -> np.ndarray:
    """count lengths floor(2^U), U uniform in [lo_log2, hi_log2]."""
    out = np.empty(count, dtype=np.uint64)
    _check(_load().gen_log_uniform_lengths(out.ctypes.data, count, lo_log2, hi_log2, seed),
           "gen_log_uniform_lengths")
    return out


def splitmix64_range(count: int, seed: int, first: int = 0) -> np.ndarray:
    """Outputs first .. first + count - 1 of the SplitMix64 stream ``seed``."""
    out = np.empty(count, dtype=np.uint64)
    _check(_load().gen_splitmix64_range(out.ctypes.data, count, seed, first), "gen_splitmix64_range")
    return out


def unit_uniform(count: int, seed: int, first: int = 0) -> np.ndarray:
    """Doubles (x >> 11) * 2^-53 in [0, 1) from the SplitMix64 stream ``seed``."""
    return (splitmix64_range(count, seed, first) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def u64_segments(lengths: np.ndarray, dist: str = "uniform", seed: int = SEED_VALUES, first: int = 0,
                 out: np.ndarray | None = None) -> np.ndarray:
    """Independent arrays back to back: array j has lengths[j] keys of the
    distribution drawn with value seed ``seed + 2^32 * (first + j)``."""
    lengths = np.ascontiguousarray(lengths, dtype=np.uint64)
    total = int(lengths.sum())
    if out is None:
        out = np.empty(total, dtype=np.uint64)
    if out.dtype != np.uint64 or not out.flags.c_contiguous or out.size < total:
        raise ValueError("out must be a contiguous uint64 array with room for every segment")
    _check(_load().gen_u64_segments(out.ctypes.data, lengths.ctypes.data, len(lengths), _dist_id(dist), seed, first),
           "gen_u64_segments")
    return out[:total]


REQUEST_TYPES = ("u64", "u64", "f64", "pair")     # drawn uniformly: u64 : f64 : pair = 2 : 1 : 1


def request_stream(count: int, lo_log2: float = 10, hi_log2: float = 26, rate: float = 1.0):
    """The served workload's requests as (sizes, key types, distributions,
    arrival times in seconds).  Sizes floor(2^U), U ~ U[lo_log2, hi_log2]
    (seed 4); from the seed-5 stream, draw 3j picks the key type (u64 : f64 :
    pair = 2 : 1 : 1), draw 3j+1 the distribution (uniform over the nine) and
    draw 3j+2 the exponential gap before request j (Poisson arrivals at
    ``rate`` requests per second; request 0 arrives at time 0)."""
    sizes = log_uniform_lengths(count, lo_log2, hi_log2)
    u = unit_uniform(3 * count, SEED_ARRIVALS)
    types = [REQUEST_TYPES[int(x * 4)] for x in u[0::3]]
    dists = [DISTRIBUTIONS[int(x * len(DISTRIBUTIONS))] for x in u[1::3]]
    gaps = -np.log1p(-u[2::3]) / rate
    gaps[0] = 0.0
    return sizes, types, dists, np.cumsum(gaps)


def quartet(n: int, dist: str = "uniform", seed: int = SEED_VALUES) -> np.ndarray:
    """n quartets (Section 5: three key words and one word of associated
    information).  The first key word follows the distribution; the second
    takes four values (SplitMix64 stream 6 mod 4), so that elements with equal
    first words are ordered by the later words; the third and the payload are
    the SplitMix64 streams 7 and 3."""
    out = np.empty(n, dtype=QUARTET_DTYPE)
    out["k0"] = u64(n, dist, seed)
    out["k1"] = splitmix64_range(n, SEED_QUARTET_K1) % np.uint64(4)
    out["k2"] = splitmix64_range(n, SEED_QUARTET_K2)
    out["payload"] = splitmix64_range(n, SEED_PAYLOAD)
    return out


def make(key_type: str, n: int, dist: str = "uniform", seed: int = SEED_VALUES) -> np.ndarray:
    """Inputs by key-type name: 'u64', 'f64', 'pair', 'rec100' or 'quartet'."""
    if key_type == "u64":
        return u64(n, dist, seed)
    if key_type == "f64":
        return f64(n, dist, seed)
    if key_type == "pair":
        return pair(n, dist, seed)
    if key_type == "rec100":
        return rec100(n, dist, seed)
    if key_type == "quartet":
        return quartet(n, dist, seed)
    raise ValueError(f"unknown key type {key_type!r}")
