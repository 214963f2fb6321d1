"""Autotuner of the distribution step per size class.

The number of leaves k of a distribution step and the oversampling factor
alpha trade classification cost (log2 k tree levels per element) against
the number of further steps and the spread of bucket sizes (Section 4.7 fixes
k = 256 and alpha = 0.2 log n for the paper's CPUs).  On the GPU the best
choice differs with the subproblem size, so this module measures it: for each
size class c (subproblems of 2^c <= n < 2^(c+1) elements), from the smallest
class that is not sorted by the base case upwards, it times the segmented
sort of a batch of arrays of that class under every candidate (k, alpha),
with the classes below already tuned, and keeps the fastest.  The result is a
table for ips4o_set_class_params; the block size b and the CTA sizes are
fixed at compile time (b = 512 bytes, the buffer blocks of a classification
CTA fill its shared memory).

Every measurement runs the library's CUDA kernels through the C ABI; this
module only generates inputs, times calls and keeps the best candidate.
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import inputs, ips4o

LEAVES = (4, 8, 16, 32, 64, 128, 256)
ALPHAS = (8, 16, 32)


def _time_batch(torch, work, pristine, off, kt, reps):
    best = float("inf")
    stream = torch.cuda.current_stream()
    for _ in range(reps):
        work.copy_(pristine)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        rc = ips4o.ips4o_sort_segmented(work.data_ptr(), off.ctypes.data, len(off) - 1, ips4o.KEY_TYPES[kt],
                                        stream.cuda_stream)
        e.record(stream)
        torch.cuda.synchronize()
        if rc:
            raise ips4o.Ips4oError(rc, "ips4o_sort_segmented")
        best = min(best, s.elapsed_time(e))
    return best


def tune(key_type: str = "u64", classes=range(14, 21), batch_keys: int = 1 << 25, reps: int = 3,
         leaves=LEAVES, alphas=ALPHAS, dist: str = "uniform", scheduler: int = 1, log=None) -> dict:
    """Tune the classes in ``classes`` (ascending) on arrays of ``dist`` keys.
    Returns {"key_type", "table": [[leaves, alpha] x 64], "results": {...}}.
    The table is left installed (ips4o_set_class_params)."""
    import torch
    table = [(0, 0)] * ips4o.NUM_CLASSES
    results = {}
    cap = ips4o.ips4o_base_case_capacity(ips4o.KEY_TYPES[key_type])
    prev = ips4o.ips4o_get_params()
    ips4o.set_params(segment_scheduler=scheduler)
    try:
        for c in classes:
            lo, hi = 1 << c, (1 << (c + 1)) - 1
            if hi <= cap:
                continue                                        # sorted by the base case alone
            count = max(1, batch_keys // ((lo + hi) // 2))
            u = inputs.unit_uniform(count, 6, first=c << 20)   # lengths uniform in the class
            lengths = (lo + (u * (hi - lo + 1)).astype(np.uint64)).astype(np.uint64)
            off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.uint64)
            host = inputs.make(key_type, int(off[-1]), dist)
            raw = np.ascontiguousarray(host).view(np.uint8).reshape(-1)
            pristine = torch.from_numpy(raw).cuda()
            work = torch.empty_like(pristine)
            timings = {}
            for L in leaves:
                for a in alphas:
                    if a * L > 4096:
                        continue
                    trial = list(table)
                    trial[c] = (L, a)
                    rc = ips4o.ips4o_set_class_params(trial)
                    if rc:
                        raise ips4o.Ips4oError(rc, "ips4o_set_class_params")
                    timings[(L, a)] = _time_batch(torch, work, pristine, off, key_type, reps)
            trial = list(table)
            ips4o.ips4o_set_class_params(trial)
            default_ms = _time_batch(torch, work, pristine, off, key_type, reps)
            best = min(timings, key=timings.get)
            if timings[best] < default_ms:
                table[c] = best
            results[c] = {"arrays": count, "keys": int(off[-1]), "default_ms": default_ms,
                          "best": list(best), "best_ms": timings[best],
                          "chosen": list(table[c]),
                          "all_ms": {f"{L},{a}": t for (L, a), t in sorted(timings.items())}}
            if log:
                log(f"class 2^{c}: default {default_ms:.3f} ms, best k={best[0]} alpha={best[1]} "
                    f"{timings[best]:.3f} ms")
            del pristine, work
        ips4o.ips4o_set_class_params(table)
    finally:
        ips4o.ips4o_set_params(prev)
    return {"key_type": key_type, "dist": dist, "table": [list(x) for x in table], "results": results}


def save(result: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(result, f, indent=1)


def load(path: str) -> dict:
    """Install a saved table (ips4o_set_class_params) and return it."""
    with open(path) as f:
        result = json.load(f)
    rc = ips4o.ips4o_set_class_params([tuple(x) for x in result["table"]])
    if rc:
        raise ips4o.Ips4oError(rc, "ips4o_set_class_params")
    return result
