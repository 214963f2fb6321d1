"""A sort service on one GPU with continuous batching.

Requests (an array of n elements of one key type) arrive over time.  The
service keeps every admitted request resident in HBM, admits waiting
requests in arrival order as long as their bytes fit the HBM budget, and
hands the resident requests of one key type as one batch to a free worker.
Each worker owns a CUDA stream (and with it the library's workspace for that
stream) and sorts its batch with one ``ips4o_sort_batched`` call, so that up
to ``workers`` batches are on the device at once, and requests that arrive
while batches run are admitted and batched as soon as memory and a worker
are free.  Every sort runs in the library's CUDA kernels; this module only
moves pointers, memory and timestamps.

The paper has no service; it sorts one array per call (Section 1).  A
request's result is the same whether it is sorted alone or in a batch: the
batched call sorts every array as ``ips4o_sort`` would, and the key sequence
of a sorted array is unique.
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import ips4o

ELEM_BYTES = {"u64": 8, "f64": 8, "pair": 16}


@dataclass
class Request:
    rid: int
    key_type: str           # 'u64', 'f64' or 'pair'
    n: int                  # elements
    arrival: float          # seconds after the start of the run
    t_admit: float = -1.0
    t_start: float = -1.0
    t_done: float = -1.0
    sorted_ok: bool | None = None
    buf: object = field(default=None, repr=False)      # device tensor while resident
    ready: object = field(default=None, repr=False)    # CUDA event: input written

    @property
    def nbytes(self) -> int:
        return self.n * ELEM_BYTES[self.key_type]

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def _sorted_on_device(torch, buf, key_type) -> bool:
    """Non-decreasing keys in the library's order (checked on the current stream)."""
    if key_type == "f64":
        x = buf.view(torch.float64)
    else:
        x = buf.view(torch.int64)
        if key_type == "pair":
            x = x.view(-1, 2)[:, 0]
        x = x ^ (-(1 << 63))            # unsigned order as signed order
    if x.numel() < 2:
        return True
    return not bool((x[1:] < x[:-1]).any().item())


class SortServer:
    """Continuous-batching sort service.

    ``fill(request, buf)`` writes a request's input into its device buffer
    (a uint8 tensor of request.nbytes) on the current stream; the service
    calls it at admission.  ``keep(request)`` decides whether a request's
    buffer is kept after completion (for checks); other buffers are freed.
    """

    def __init__(self, budget_bytes: int, workers: int = 3, max_batch_requests: int = 1024,
                 max_batch_keys: int = 1 << 27, check_sorted: bool = True):
        import torch
        self.torch = torch
        self.workers = workers
        self.max_batch_requests = max_batch_requests
        self.max_batch_keys = max_batch_keys
        self.check_sorted = check_sorted
        self.device = torch.cuda.current_device()
        self.streams = [torch.cuda.Stream() for _ in range(workers)]
        # each worker's workspace is reserved up front (no allocation, and
        # no implicit device synchronisation, while batches run) and counted
        # against the budget
        self.workspace_bytes = 0
        for s in self.streams:
            for kt in ("u64", "pair"):
                rc = ips4o.ips4o_reserve_workspace(max_batch_keys, max_batch_requests, ips4o.KEY_TYPES[kt],
                                                   s.cuda_stream)
                if rc:
                    raise ips4o.Ips4oError(rc, "ips4o_reserve_workspace")
            self.workspace_bytes += max(ips4o.ips4o_workspace_bytes(max_batch_keys, ips4o.KEY_TYPES[kt])
                                        for kt in ("u64", "pair"))
        self.budget = budget_bytes - self.workspace_bytes
        if self.budget <= 0:
            raise ValueError("the HBM budget does not cover the workers' workspaces")

    # -------------------------------------------------------------- workers
    def _worker(self, wid, inq, doneq, t0):
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = self.streams[wid]
        while True:
            batch = inq.get()
            if batch is None:
                return
            try:
                for r in batch:
                    stream.wait_event(r.ready)
                kt = batch[0].key_type
                ptrs = np.array([r.buf.data_ptr() for r in batch], dtype=np.uint64)
                lens = np.array([r.n for r in batch], dtype=np.uint64)
                t_start = time.perf_counter() - t0
                rc = ips4o.ips4o_sort_batched(ptrs.ctypes.data, lens.ctypes.data, len(batch), ips4o.KEY_TYPES[kt],
                                              stream.cuda_stream)
                stream.synchronize()
                t_done = time.perf_counter() - t0
                for r in batch:
                    r.t_start, r.t_done = t_start, t_done
                if rc:
                    raise ips4o.Ips4oError(rc, "ips4o_sort_batched")
                if self.check_sorted:
                    with torch.cuda.stream(stream):
                        for r in batch:
                            r.sorted_ok = _sorted_on_device(torch, r.buf, r.key_type)
                doneq.put((wid, batch, None))
            except Exception as e:      # handed to the dispatcher, which re-raises
                doneq.put((wid, batch, e))

    # ------------------------------------------------------------- dispatch
    def run(self, requests, fill, keep=lambda r: False):
        """Serve ``requests`` (their ``arrival`` times are honoured against
        the wall clock from the call).  Returns the requests with their
        timestamps; ``buf`` is kept for the requests ``keep`` selects."""
        torch = self.torch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        ready = {kt: collections.deque() for kt in ELEM_BYTES}
        free = list(range(self.workers))
        inqs = [queue.Queue() for _ in range(self.workers)]
        doneq = queue.Queue()
        upload = torch.cuda.Stream()
        t0 = time.perf_counter()
        threads = [threading.Thread(target=self._worker, args=(w, inqs[w], doneq, t0), daemon=True)
                   for w in range(self.workers)]
        for t in threads:
            t.start()
        in_use = 0
        outstanding = len(pending)
        error = None
        try:
            while outstanding:
                now = time.perf_counter() - t0
                while pending and pending[0].arrival <= now:
                    waiting.append(pending.popleft())
                # admission in arrival order under the HBM budget
                while waiting and in_use + waiting[0].nbytes <= self.budget:
                    r = waiting.popleft()
                    with torch.cuda.stream(upload):
                        r.buf = torch.empty(r.nbytes, dtype=torch.uint8, device="cuda")
                        fill(r, r.buf)
                        r.ready = torch.cuda.Event()
                        r.ready.record(upload)
                    r.t_admit = time.perf_counter() - t0
                    in_use += r.nbytes
                    ready[r.key_type].append(r)
                if waiting and in_use == 0 and waiting[0].nbytes > self.budget:
                    raise ValueError(f"request {waiting[0].rid} does not fit the HBM budget")
                # continuous batching: the key type with the oldest resident
                # request goes to the next free worker
                while free and any(ready.values()):
                    kt = min((q[0].arrival, kt) for kt, q in ready.items() if q)[1]
                    q = ready[kt]
                    batch, keys = [], 0
                    while q and len(batch) < self.max_batch_requests and (not batch or keys + q[0].n <= self.max_batch_keys):
                        r = q.popleft()
                        batch.append(r)
                        keys += r.n
                    inqs[free.pop()].put(batch)
                # completions
                if pending and not waiting and not any(ready.values()):
                    timeout = max(0.0, min(0.002, pending[0].arrival - (time.perf_counter() - t0)))
                else:
                    timeout = 0.0005
                try:
                    wid, batch, err = doneq.get(timeout=timeout)
                except queue.Empty:
                    continue
                while True:
                    free.append(wid)
                    if err is not None and error is None:
                        error = err
                    for r in batch:
                        in_use -= r.nbytes
                        if not keep(r):
                            r.buf = None
                        r.ready = None
                    outstanding -= len(batch)
                    try:
                        wid, batch, err = doneq.get_nowait()
                    except queue.Empty:
                        break
                if error is not None:
                    raise error
        finally:
            for q in inqs:
                q.put(None)
            for t in threads:
                t.join()
        return requests

    def run_one_at_a_time(self, requests, fill, keep=lambda r: False):
        """The same requests through plain ips4o_sort calls, one at a time in
        arrival order on one stream (the comparison the service must beat)."""
        torch = self.torch
        stream = self.streams[0]
        t0 = time.perf_counter()
        for r in sorted(requests, key=lambda r: r.arrival):
            now = time.perf_counter() - t0
            if r.arrival > now:
                time.sleep(r.arrival - now)
            with torch.cuda.stream(stream):
                r.buf = torch.empty(r.nbytes, dtype=torch.uint8, device="cuda")
                fill(r, r.buf)
                r.t_admit = r.t_start = time.perf_counter() - t0
                rc = ips4o.ips4o_sort(r.buf.data_ptr(), r.n, ips4o.KEY_TYPES[r.key_type], stream.cuda_stream)
                stream.synchronize()
                r.t_done = time.perf_counter() - t0
                if rc:
                    raise ips4o.Ips4oError(rc, "ips4o_sort")
                if self.check_sorted:
                    r.sorted_ok = _sorted_on_device(torch, r.buf, r.key_type)
            if not keep(r):
                r.buf = None
        return requests


def summarize(requests) -> dict:
    lat = np.array([r.latency for r in requests]) * 1e3
    keys = sum(r.n for r in requests)
    t_first = min(r.arrival for r in requests)
    t_last = max(r.t_done for r in requests)
    return {
        "requests": len(requests),
        "keys": keys,
        "keys_per_s": keys / (t_last - t_first),
        "makespan_s": t_last - t_first,
        "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()),
        "max_ms": float(lat.max()),
        "all_sorted": all(r.sorted_ok is not False for r in requests),
    }
