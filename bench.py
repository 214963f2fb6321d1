"""Benchmark: in-place samplesort of 2^28 uint64 keys on one GB300.

A step is one complete sort (every distribution level and the base case) of
a fresh copy of the input, which is already resident in HBM; the copy that
restores the input between steps is not timed.  The input (2 GiB) is larger
than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dist uniform]
  python bench.py --impl reference     # the CPU oracle on a bounded sample
  python bench.py --workload batched [--segments 100000 | --batched-total-log2 28] [--dist two_dup]
      many independent arrays (log-uniform lengths in [16, 2^20]) sorted by
      one ips4o_sort_segmented call per step, against a loop of plain calls
  python bench.py --workload served [--requests 20000] [--load 0.7]
      a stream of requests (Poisson arrivals, sizes log-uniform in [2^10, 2^26],
      u64 : f64 : pair = 2 : 1 : 1, the nine distributions) through the
      continuous-batching service under a 64 GB HBM budget, against the same
      stream through one-at-a-time plain calls; p50/p99 latency and keys/s

Prints one JSON line.  `value` is keys/s over all ranks (N > 1 runs
independent replicas, one per GPU: the sort does not shard).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "keys/s"
# DRAM bytes per launch of the dominant kernels for 2^28 Uniform u64 keys: one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the same
# kernels at 2^26 keys, where a launch processes a quarter of the elements,
# scaled by 4 (averaged over the two distribution levels).  Retake the
# capture when one of these kernels changes.
NOMINAL_HBM_GBS = 7900.0      # the data-sheet HBM3e bandwidth, for context beside the measured peak
TRAFFIC_2P28_U64_UNIFORM = {"classify": 4.050e9, "block_permutation": 4.005e9, "base_case": 3.808e9}
ELEM_BYTES = {"u64": 8, "f64": 8, "pair": 16, "rec100": 100, "quartet": 32}
DTYPE_NAME = {"u64": "u64", "f64": "f64", "pair": "u64 key + u64 payload", "rec100": "80-bit byte key + 90-byte payload",
              "quartet": "3 x u64 key + u64 payload"}
KT_LABEL = {"u64": "uint64 keys", "f64": "float64 keys", "pair": "16-byte (uint64 key, uint64 payload) pairs",
            "rec100": "100-byte records (10-byte key)",
            "quartet": "32-byte quartets (three uint64 key words, one payload word)"}


def _sorted_keys(t, kt) -> bool:
    """Keys non-decreasing in the library's order, checked on the device."""
    import torch
    if kt == "rec100":
        r = t.view(-1, 100)
        b = r[:, :10].to(torch.int64)
        hi = torch.zeros(r.shape[0], dtype=torch.int64, device=t.device)
        for q in range(7):                      # the first 7 bytes fit a signed 64-bit compare
            hi = hi * 256 + b[:, q]
        lo = (b[:, 7] << 16) | (b[:, 8] << 8) | b[:, 9]
        d_hi = hi[1:] - hi[:-1]
        ok = (d_hi > 0) | ((d_hi == 0) & (lo[1:] >= lo[:-1]))
        return bool(ok.all().item())
    if kt == "quartet":
        k = t.view(torch.int64).view(-1, 4)[:, :3] ^ (-(1 << 63))
        a, b = k[:-1], k[1:]
        ok = (a[:, 0] < b[:, 0]) | ((a[:, 0] == b[:, 0]) & ((a[:, 1] < b[:, 1]) | ((a[:, 1] == b[:, 1]) & (a[:, 2] <= b[:, 2]))))
        return bool(ok.all().item())
    if kt == "f64":
        x = t.view(torch.float64)
    else:
        x = t.view(torch.int64)
        if kt == "pair":
            x = x.view(-1, 2)[:, 0]
        x = x ^ (-(1 << 63))
    return bool((x[1:] >= x[:-1]).all().item())
LOG2N = 28
FALLBACK_HBM_GBS = 6800.0


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]) if parts[3] not in ("[N/A]", "") else 0.0,
                             parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return out
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        loaded = [r for r in rows if r[2] > 200.0] or rows
        reasons = set()
        for r in loaded:
            for nm, v in zip(names, r[3]):
                if v.lower() == "active":
                    reasons.add(nm)
        out.update(sm_mhz=statistics.median(r[0] for r in loaded), sm_max_mhz=max(r[1] for r in rows),
                   reasons=sorted(reasons), samples=len(rows),
                   power_w_max=max(r[2] for r in rows))
        return out


def _transfer_bound(h_buf, d_buf, stream, reps: int) -> dict:
    """Copy-engine time of one host -> device and one device -> host copy of
    the step's bytes between pinned host memory and HBM: the least an end-to-
    end sort that must bring its input in and its result back can take when
    the two transfers do not overlap each other."""
    import torch
    d_tmp = torch.empty_like(d_buf)
    h_tmp = torch.empty_like(h_buf).pin_memory()
    res = {}
    best = {"h2d": float("inf"), "d2h": float("inf")}
    for _ in range(reps):                                      # alternate directions, keep the best of each
        for name, dst, src in (("h2d", d_tmp, h_buf), ("d2h", h_tmp, d_buf)):
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            dst.copy_(src, non_blocking=True)
            e.record(stream)
            torch.cuda.synchronize()
            best[name] = min(best[name], s.elapsed_time(e))
    for name, src in (("h2d", h_buf), ("d2h", d_buf)):
        res[f"{name}_ms"] = best[name]
        res[f"{name}_gbs"] = src.numel() / (best[name] * 1e-3) / 1e9
    res["transfer_bound_ms"] = res["h2d_ms"] + res["d2h_ms"]
    del d_tmp, h_tmp
    return res


def cpu_baseline(log2n_sample: int = 24, reps: int = 1, kt: str = "u64", dist: str = "uniform"):
    """The oracle, as it stands, single-threaded on a bounded sample."""
    import oracle
    from paper_1705_02257_gb300 import inputs
    n = 1 << log2n_sample
    a = inputs.make(kt, n, dist)
    oracle.sort(a[:1024], kt)                         # load/build outside the timing
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.sort(a, kt)
    dt = time.perf_counter() - t0
    return {"value": n * reps / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"2^{log2n_sample} {KT_LABEL[kt]}, {dist} (seed 1), {reps} sort(s), single-threaded C oracle, "
                      f"{dt:.1f} s", "host_cores": os.cpu_count()}


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1705_02257_gb300 import inputs
    kt = args.key_type
    log2s = min(args.ref_log2n, 20) if kt == "rec100" else args.ref_log2n
    n = 1 << log2s
    base = inputs.make(kt, n, args.dist)
    oracle.sort(base[:1024], kt)
    for _ in range(args.warmup):
        oracle.sort(base, kt)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sort(base, kt)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n * args.steps / total
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[kt], "data": "synthetic",
        "impl": "reference",
        "config": {"workload": f"{'sort' if kt == 'rec100' else 'in-place sort'} of 2^{args.log2n} {KT_LABEL[kt]}, "
                               f"{args.dist} (seed 1); reference steps sort a 2^{log2s}-element sample",
                   "n": 1 << args.log2n, "key_type": kt, "distribution": args.dist},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                         "sample": f"2^{log2s} {KT_LABEL[kt]}, {args.dist}, per step, single-threaded C oracle"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    rank, world, local = _dist_env()
    dist_on = world > 1
    if dist_on:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1705_02257_gb300 import build as cuda_build
    cuda_build.build()
    from paper_1705_02257_gb300 import inputs, ips4o

    n = 1 << args.log2n
    kt = args.key_type
    host = inputs.make(kt, n, args.dist)
    elem = ELEM_BYTES[kt]
    pristine = torch.from_numpy(np.ascontiguousarray(host).view(np.uint8).reshape(-1)).cuda()
    work = torch.empty_like(pristine)
    stream = torch.cuda.current_stream()
    ips4o.reset_params()
    base_params = {}
    if args.stripes_per_sm > 0:
        base_params["stripes_per_sm"] = args.stripes_per_sm
    if args.record_path:
        base_params["record_path"] = args.record_path
    if base_params:
        ips4o.set_params(**base_params)
    # ips4o_sort, or the strictly in-place ips4o_sort_strict (Section 4.6)
    sort_fn = ips4o.sort_strict if args.strict else ips4o.sort

    def one_step():
        work.copy_(pristine)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        sort_fn(work, kt)
        e.record(stream)
        torch.cuda.synchronize()
        return s.elapsed_time(e)

    for _ in range(args.warmup):
        one_step()
    launches_per_step = ips4o.stats()["kernel_launches"]

    if dist_on:
        tdist.barrier()
    torch.cuda.synchronize()
    times = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            times.append(one_step())
    torch.cuda.synchronize()
    if dist_on:
        tdist.barrier()
    total_ms = sum(times)
    if dist_on:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        total_ms = float(t.item())
    stats = ips4o.stats()
    levels = stats["levels"]

    # output check on the last timed step: sorted and a permutation
    sorted_ok = _sorted_keys(work, kt)

    # per-kernel times (CUDA events around each launch on the sort's stream)
    ips4o.set_params(profile=1, **base_params)
    prof_steps = max(1, min(3, args.steps))
    phase_ms = {p: 0.0 for p in ips4o.PHASES}
    phase_launches = {p: 0 for p in ips4o.PHASES}
    for _ in range(prof_steps):
        one_step()
        st = ips4o.stats()
        for p in ips4o.PHASES:
            phase_ms[p] += st["phase_ms"][p]
            phase_launches[p] += st["phase_launches"][p]
    ips4o.reset_params()
    if base_params:
        ips4o.set_params(**base_params)
    # algorithmic bytes per launch (Appendix B I/O volume): classification and
    # block permutation each read and write the elements of the launch once.
    # Records are distributed as 16-byte (key prefix, index) pairs.
    rec_blocks = kt == "rec100" and (args.record_path == 1 or args.strict)   # records moved in place, not pairs
    dist_elem = 16 if kt == "rec100" and not rec_blocks else elem
    # elements classified over all levels of one sort (a deeper level often
    # holds only a few buckets): the classification and permutation volume
    distributed = stats["elements_distributed"] or n * levels
    per_level = 2.0 * distributed * dist_elem * prof_steps
    alg = {
        "classify": per_level,
        "block_permutation": per_level,
        "base_case": 2.0 * n * dist_elem * prof_steps,
    }
    dominant = max(alg, key=lambda p: phase_ms[p])
    traffic = None
    if kt == "u64" and args.log2n == 28 and args.dist == "uniform":
        traffic = TRAFFIC_2P28_U64_UNIFORM.get(dominant)
    peak, peak_kind = _peaks()
    achieved = alg[dominant] / (phase_ms[dominant] * 1e-3) / 1e9 if phase_ms[dominant] > 0 else None
    ms_per_step = total_ms / args.steps
    value = n * world * args.steps / (total_ms * 1e-3)
    # the sort's roofline uses the nominal number of levels, log_k(n / base
    # case) with k = 256, the same bar for every distribution
    base_cap = 1024 if rec_blocks else ips4o.ips4o_base_case_capacity(ips4o.KEY_TYPES["pair" if kt == "rec100" else kt])
    nominal_levels, m = 0, n
    while m > base_cap:
        m = (m + 255) // 256
        nominal_levels += 1
    alg_sort = (4 * nominal_levels + 2) * n * dist_elem
    if kt == "rec100" and not rec_blocks:
        # key extraction (12 bytes read, 16 written), input copy (read + write)
        # and the gather (pair read, record read + write)
        alg_sort += n * (12 + 16) + 2 * n * elem + n * (16 + 2 * elem)
    sort_frac = alg_sort / (ms_per_step * 1e-3) / 1e9 / peak
    # the distribution levels alone (sampling through cleanup, no base case):
    # 4 n s per nominal level over the device time of those phases
    level_phases = ("sample", "classify", "prefix", "empty_block_fix", "block_permutation", "cleanup")
    levels_ms = sum(phase_ms[p] for p in level_phases if p in phase_ms) / prof_steps
    levels_alg = 4.0 * nominal_levels * n * dist_elem
    levels_gbs = levels_alg / (levels_ms * 1e-3) / 1e9 if levels_ms > 0 else None

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        h_in = torch.from_numpy(np.ascontiguousarray(host).view(np.uint8).reshape(-1)).pin_memory()
        h_work = torch.empty_like(h_in).pin_memory()
        e2e_times = []
        for i in range(args.warmup + args.steps):
            h_work.copy_(h_in)
            t0 = time.perf_counter()
            rc = ips4o.ips4o_sort_host(h_work.data_ptr(), n, ips4o.KEY_TYPES[kt], stream.cuda_stream)
            dt = time.perf_counter() - t0
            if rc:
                raise ips4o.Ips4oError(rc, "ips4o_sort_host")
            if i >= args.warmup:
                e2e_times.append(dt)
        e2e_total = sum(e2e_times)
        # the last call's host result: non-decreasing, and for key-only types
        # equal to the device-timed sort of the same input
        t_chk = h_work.cuda()
        e2e_sorted = bool(_sorted_keys(t_chk, kt))
        e2e_same = bool(torch.equal(t_chk, work)) if kt in ("u64", "f64") else None
        del t_chk
        if dist_on:
            t = torch.tensor([e2e_total], device="cuda", dtype=torch.float64)
            tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
            e2e_total = float(t.item())
        e2e = {"value": n * world * args.steps / e2e_total, "unit": METRIC,
               "h2d_bytes_per_step": n * elem, "d2h_bytes_per_step": n * elem,
               "ms_per_step": 1e3 * e2e_total / args.steps, "host_memory": "pinned",
               "output_sorted": e2e_sorted, "equals_device_result": e2e_same}
        # the transfer bound: the same bytes copied host -> device and back
        # by the copy engines (pinned buffers, CUDA events), no sort between
        e2e.update(_transfer_bound(h_in, pristine, stream, 4))
        e2e["frac_of_transfer_bound"] = e2e["transfer_bound_ms"] / e2e["ms_per_step"]
        del h_in, h_work

    if rank != 0:
        if dist_on:
            tdist.destroy_process_group()
        return 0
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(
        min(args.cpu_log2n, 22) if kt == "rec100" else args.cpu_log2n, kt=kt, dist=args.dist)
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_NAME[kt], "data": "synthetic",
        "config": {"workload": f"{'sort' if kt == 'rec100' and not rec_blocks else 'in-place sort'} of 2^{args.log2n} "
                               f"{KT_LABEL[kt]}, {args.dist} (seed 1)"
                               f"{' (in-place block path)' if rec_blocks else (' (key + index indirection)' if kt == 'rec100' else '')}"
                               f"{', strictly in place (ips4o_sort_strict)' if args.strict else ''}",
                   "n": n, "key_type": kt, "distribution": args.dist,
                   "l2": f"input {n * elem / 2**30:.2f} GiB per step, larger than the 129 MB L2 (no flush needed)",
                   "parallelism": f"replicas x{world}", "levels": levels},
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": traffic,
                     "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the same "
                                        "kernels at 2^26 keys, scaled by 4 to 2^28") if traffic else None,
                     "alg_bytes_per_launch": alg[dominant] / (prof_steps * (levels if dominant != "base_case" else 1)),
                     "launches": levels if dominant != "base_case" else 1,
                     "alg_bytes_per_sort": alg[dominant] / prof_steps,
                     "sort_alg_bytes": alg_sort, "sort_frac": sort_frac, "nominal_levels": nominal_levels,
                     "levels_alg_bytes": levels_alg, "levels_ms": levels_ms, "levels_gbs": levels_gbs,
                     "levels_frac": (levels_gbs / peak) if levels_gbs else None,
                     "levels_frac_of_nominal_7900": (levels_gbs / NOMINAL_HBM_GBS) if levels_gbs else None},
        "phase_ms_per_step": {p: phase_ms[p] / prof_steps for p in ips4o.PHASES},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": launches_per_step * args.steps,
        "output_sorted": sorted_ok,
        "stats": {k: stats[k] for k in ("levels", "chunks", "subproblems", "blocks_moved", "blocks_skipped",
                                        "fix_blocks_moved", "base_case_buckets", "workspace_bytes")},
    }
    print(json.dumps(line), flush=True)
    if dist_on:
        tdist.destroy_process_group()
    return 0


def _segment_lengths(args, inputs):
    """Log-uniform lengths floor(2^U), U ~ U[4, 20] (seed 4): either a fixed
    number of arrays or as many as it takes to reach 2^batched_total_log2 keys."""
    if args.batched_total_log2 <= 0:
        return inputs.log_uniform_lengths(args.segments, 4, 20)
    target = 1 << args.batched_total_log2
    count = 4096
    while True:
        lengths = inputs.log_uniform_lengths(count, 4, 20)
        csum = np.cumsum(lengths)
        if csum[-1] >= target:
            return lengths[: int(np.searchsorted(csum, target)) + 1]
        count *= 2


def run_batched(args):
    import torch
    rank, world, local = _dist_env()
    dist_on = world > 1
    if dist_on:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1705_02257_gb300 import build as cuda_build
    cuda_build.build()
    from paper_1705_02257_gb300 import inputs, ips4o
    import oracle

    lengths = _segment_lengths(args, inputs)
    nseg = len(lengths)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.uint64)
    total = int(off[-1])
    pristine = torch.empty(total, dtype=torch.int64, device="cuda")
    work = torch.empty_like(pristine)
    # generate on the host in groups of at most 2^27 keys, copy into HBM
    group = 1 << 27
    h_buf = torch.empty(group + (1 << 20), dtype=torch.int64).pin_memory()
    h_np = h_buf.numpy().view(np.uint64)
    j = 0
    while j < nseg:
        j1 = j
        while j1 < nseg and (j1 == j or off[j1 + 1] - off[j] <= group):
            j1 += 1
        cnt = int(off[j1] - off[j])
        buf = h_np if cnt <= h_np.size else np.empty(cnt, dtype=np.uint64)
        inputs.u64_segments(lengths[j:j1], args.dist, first=j, out=buf)
        src = torch.from_numpy(buf[:cnt].view(np.int64))
        pristine[int(off[j]):int(off[j1])].copy_(src)
        torch.cuda.synchronize()
        j = j1
    stream = torch.cuda.current_stream()
    ips4o.reset_params()
    tuned = None
    if args.autotune:
        from paper_1705_02257_gb300 import autotune
        tuned = autotune.tune("u64", classes=range(14, 21), dist=args.dist,
                              scheduler=args.segment_scheduler or 1)
    if args.segment_scheduler in (1, 2):
        ips4o.set_params(segment_scheduler=args.segment_scheduler)
    off_host = np.ascontiguousarray(off)
    enqueue_only = args.segment_scheduler == 3
    if enqueue_only:
        # ips4o_sort_segmented_async: offsets on the device, workspace reserved
        d_off = torch.from_numpy(off_host.view(np.int64).copy()).cuda()
        rc = ips4o.ips4o_reserve_workspace(total, nseg, ips4o.U64, stream.cuda_stream)
        if rc:
            raise ips4o.Ips4oError(rc, "ips4o_reserve_workspace")

    def one_step():
        work.copy_(pristine)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        if enqueue_only:
            rc = ips4o.ips4o_sort_segmented_async(work.data_ptr(), d_off.data_ptr(), nseg, ips4o.U64,
                                                  stream.cuda_stream)
        else:
            rc = ips4o.ips4o_sort_segmented(work.data_ptr(), off_host.ctypes.data, nseg, ips4o.U64, stream.cuda_stream)
        e.record(stream)
        torch.cuda.synchronize()
        if rc == 0 and enqueue_only:
            rc = ips4o.ips4o_stream_status(stream.cuda_stream)
        if rc:
            raise ips4o.Ips4oError(rc, "ips4o_sort_segmented")
        return s.elapsed_time(e)

    for _ in range(args.warmup):
        one_step()
    if dist_on:
        tdist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        times = [one_step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    total_ms = sum(times)
    if dist_on:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        total_ms = float(t.item())
    stats = ips4o.stats()
    value = total * world * args.steps / (total_ms * 1e-3)

    # parity on the last timed step: every segment non-decreasing (on the
    # device), and a seeded sample of segments equal to the oracle's sort
    sorted_ok = True
    seg_starts = off[1:-1].astype(np.int64)
    chunk = 1 << 28
    for c0 in range(0, total - 1, chunk):
        c1 = min(total, c0 + chunk + 1)
        x = work[c0:c1] ^ (-(1 << 63))          # unsigned order as signed order
        desc = x[1:] < x[:-1]                   # desc[i]: element c0+i+1 below its predecessor
        lo, hi = np.searchsorted(seg_starts, [c0 + 1, c1])
        if hi > lo:
            desc[torch.from_numpy(seg_starts[lo:hi] - c0 - 1).cuda()] = False   # a new array starts there
        if bool(desc.any().item()):
            sorted_ok = False
        del x, desc
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(nseg, size=min(nseg, args.verify_segments), replace=False))
    oracle_ok = True
    for q in sample:
        lo, hi = int(off[q]), int(off[q + 1])
        got = work[lo:hi].cpu().numpy().view(np.uint64)
        src = pristine[lo:hi].cpu().numpy().view(np.uint64)
        if not np.array_equal(got, oracle.sort(src, "u64")):
            oracle_ok = False
            break

    # the same arrays through a loop of plain ips4o_sort calls
    lib = ips4o.lib()
    base = work.data_ptr()
    sptr = stream.cuda_stream

    def plain_loop(count):
        work.copy_(pristine)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q in range(count):
            rc = lib.ips4o_sort(base + 8 * int(off[q]), int(lengths[q]), ips4o.U64, sptr)
            if rc:
                raise ips4o.Ips4oError(rc, "ips4o_sort")
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    plain_loop(min(nseg, 2000))
    plain_s = plain_loop(nseg)
    plain_value = total / plain_s

    if rank != 0:
        if dist_on:
            tdist.destroy_process_group()
        return 0
    # the oracle on the host cores: the first arrays of the batch up to ~2^24 keys
    cpu = None
    if not args.no_cpu_baseline:
        k = int(np.searchsorted(off, 1 << 24)) or 1
        keys = int(off[k])
        data = inputs.u64_segments(lengths[:k], args.dist)
        t0 = time.perf_counter()
        for q in range(k):
            oracle.sort(data[int(off[q]):int(off[q + 1])], "u64")
        dt = time.perf_counter() - t0
        cpu = {"value": keys / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
               "sample": f"the batch's first {k} arrays ({keys} keys), one oracle call each, single-threaded C oracle"}
    peak, peak_kind = _peaks()
    alg = (4 * stats["elements_distributed"] + 2 * total) * 8
    ms = total_ms / args.steps
    achieved = alg / (ms * 1e-3) / 1e9
    label = (f"{nseg} uint64 arrays" if args.batched_total_log2 <= 0
             else f"{nseg} uint64 arrays (lengths drawn until 2^{args.batched_total_log2} keys)")
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"batched segmented sort: {label}, log-uniform lengths [16, 2^20] (seed 4), "
                               f"{args.dist} keys per array, one ips4o_sort_segmented call "
                               f"({['automatic', 'level by level', 'segment scheduler', 'enqueue-only ips4o_sort_segmented_async'][args.segment_scheduler]})",
                   "segments": nseg, "n": total, "key_type": "u64", "distribution": args.dist,
                   "l2": f"{total * 8 / 2**30:.1f} GiB per step, larger than L2",
                   "parallelism": f"replicas x{world}"},
        "vs_plain_loop": {"value": plain_value, "unit": METRIC, "ratio": value / plain_value,
                          "ms": plain_s * 1e3, "calls": nseg},
        "roofline": {"bound": "hbm", "kernel": "whole call", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "alg_bytes": alg, "elements_distributed": stats["elements_distributed"]},
        "cpu_baseline": cpu, "e2e": None, "clocks": clk.summary(),
        "gpu_launches": stats["kernel_launches"] * args.steps,
        "output_sorted": sorted_ok, "oracle_sample_ok": oracle_ok, "oracle_sample_segments": int(len(sample)),
        "autotuned": None if tuned is None else {
            "classes": {c: r["chosen"] for c, r in tuned["results"].items()},
            "default_vs_best_ms": {c: [round(r["default_ms"], 3), round(r["best_ms"], 3)]
                                   for c, r in tuned["results"].items()}},
        "stats": {k: stats[k] for k in ("levels", "chunks", "subproblems", "blocks_moved", "base_case_buckets",
                                        "workspace_bytes")},
    }
    print(json.dumps(line), flush=True)
    if dist_on:
        tdist.destroy_process_group()
    return 0


def run_served(args):
    import torch
    rank, world, local = _dist_env()
    if world > 1 and rank != 0:
        return 0        # the service runs on one GPU; other ranks have no work
    torch.cuda.set_device(local)
    from paper_1705_02257_gb300 import build as cuda_build
    cuda_build.build()
    from paper_1705_02257_gb300 import inputs, ips4o, serve
    import oracle

    lo, hi = 10, args.served_max_log2
    dtypes = {"u64": np.uint64, "f64": np.float64, "pair": inputs.PAIR_DTYPE}
    # resident inputs: one array of 2^hi elements per (key type, distribution);
    # a request of n elements of type t and distribution d sorts the first n
    pools = {}
    for kt in ("u64", "f64", "pair"):
        for d in inputs.DISTRIBUTIONS:
            a = inputs.make(kt, 1 << hi, d)
            pools[kt, d] = torch.from_numpy(a.view(np.uint8).reshape(-1)).cuda()
            del a
    torch.cuda.synchronize()
    srv = serve.SortServer(budget_bytes=args.budget_gb * 10**9, workers=args.workers,
                           max_batch_requests=1024, max_batch_keys=1 << 27)
    sizes, types, dists, unit_arr = inputs.request_stream(args.requests, lo, hi, rate=1.0)

    def make_reqs(rate):
        return [serve.Request(i, types[i], int(sizes[i]), float(unit_arr[i]) / rate) for i in range(args.requests)]

    def fill(r, buf):
        buf.copy_(pools[r.key_type, dists[r.rid]][: r.nbytes])

    # calibration: plain one-at-a-time keys/s on the first requests, all
    # present at time 0; the arrival rate then offers `load` times that
    calib = [serve.Request(i, types[i], int(sizes[i]), 0.0) for i in range(min(args.requests, 400))]
    srv.run_one_at_a_time(calib[:50], fill)
    plain_kps = serve.summarize(srv.run_one_at_a_time(calib, fill))["keys_per_s"]

    rng = np.random.default_rng(7)
    small = [i for i in range(args.requests) if sizes[i] <= (1 << 22)]
    sample = set(rng.choice(small, size=min(len(small), args.verify_requests), replace=False).tolist())
    keep = lambda r: r.rid in sample   # noqa: E731
    loads = [float(x) for x in str(args.load).split(",")]
    sweep, oracle_ok, alone_ok, unsorted = [], True, True, []
    clocks = None
    for li, load in enumerate(loads):
        rate = load * plain_kps / float(np.mean(sizes))
        with ClockSampler(torch.cuda.current_device()) as clk:
            served = srv.run(make_reqs(rate), fill, keep=keep if li == 0 else (lambda r: False))
        if li == 0:
            clocks = clk.summary()
        plain = srv.run_one_at_a_time(make_reqs(rate), fill, keep=keep if li == 0 else (lambda r: False))
        s_sum, p_sum = serve.summarize(served), serve.summarize(plain)
        unsorted += [[load, run, r.rid, r.key_type, r.n, dists[r.rid]] for run, reqs in (("served", served),
                     ("alone", plain)) for r in reqs if r.sorted_ok is False]
        sweep.append({"load": load, "arrival_rate_per_s": rate, "served": s_sum, "one_at_a_time": p_sum,
                      "ratio_keys_per_s": s_sum["keys_per_s"] / p_sum["keys_per_s"],
                      "ratio_p99": p_sum["p99_ms"] / s_sum["p99_ms"]})
        if li > 0:
            continue
        # each sampled result: the oracle's sort of the input, and the same
        # as the request sorted alone (one-at-a-time run)
        for m, a in zip(served, plain):
            if m.rid not in sample:
                continue
            src = pools[m.key_type, dists[m.rid]][: m.nbytes].cpu().numpy().view(dtypes[m.key_type])
            gm = m.buf.cpu().numpy().view(dtypes[m.key_type])
            ga = a.buf.cpu().numpy().view(dtypes[m.key_type])
            exp = oracle.sort(src, m.key_type)
            if m.key_type == "pair":
                oracle_ok &= bool(np.array_equal(gm["key"], exp["key"]))
                alone_ok &= bool(np.array_equal(np.sort(gm, order=["key", "payload"]),
                                                np.sort(ga, order=["key", "payload"])))
            else:
                oracle_ok &= bool(np.array_equal(gm.view(np.uint64), exp.view(np.uint64)))
                alone_ok &= bool(np.array_equal(gm.view(np.uint64), ga.view(np.uint64)))
            m.buf = a.buf = None
    head = sweep[0]
    peak, peak_kind = _peaks()
    line = {
        "metric": METRIC, "value": head["served"]["keys_per_s"], "unit": METRIC, "n_gpus": 1, "steps": 1,
        "warmup": 1, "ms_per_step": head["served"]["makespan_s"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64/f64/pair", "data": "synthetic",
        "config": {"workload": f"served sort stream: {args.requests} requests, Poisson arrivals at {loads[0]} x "
                               f"the one-at-a-time keys/s, sizes log-uniform [2^{lo}, 2^{hi}] (seed 4), "
                               "u64 : f64 : pair = 2 : 1 : 1 and the nine distributions (seed 5), "
                               f"{args.budget_gb} GB HBM budget, {args.workers} workers",
                   "requests": args.requests, "keys": head["served"]["keys"],
                   "l2": "requests resident in HBM; most are larger than L2"},
        "latency_ms": {k: head["served"][k] for k in ("p50_ms", "p99_ms", "mean_ms", "max_ms")},
        "vs_one_at_a_time": {"keys_per_s": head["one_at_a_time"]["keys_per_s"],
                             "p50_ms": head["one_at_a_time"]["p50_ms"], "p99_ms": head["one_at_a_time"]["p99_ms"],
                             "calibration_keys_per_s": plain_kps},
        "sweep": sweep,
        "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clocks,
        "gpu_launches": None, "peak_hbm_gbs": peak, "peak_kind": peak_kind,
        "all_sorted": not unsorted, "unsorted": unsorted[:20],
        "oracle_sample_ok": oracle_ok, "alone_equals_mixed": alone_ok, "sample_requests": len(sample),
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dist", default="uniform")
    ap.add_argument("--log2n", type=int, default=LOG2N)
    ap.add_argument("--key-type", default="u64", choices=["u64", "f64", "pair", "rec100", "quartet"],
                    help="plain workload: element type (f64 and pair at 2^27, rec100 at 2^24 in the paper's table)")
    ap.add_argument("--ref-log2n", type=int, default=22)
    ap.add_argument("--cpu-log2n", type=int, default=24)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stripes-per-sm", type=int, default=0, help="override the library's stripes per SM")
    ap.add_argument("--workload", default="plain", choices=["plain", "batched", "served"])
    ap.add_argument("--requests", type=int, default=20_000, help="served: number of requests")
    ap.add_argument("--load", default="0.7,1.5",
                    help="served: offered loads (comma-separated), each a multiple of the one-at-a-time keys/s")
    ap.add_argument("--budget-gb", type=int, default=64, help="served: HBM budget (GB) for requests + workspaces")
    ap.add_argument("--workers", type=int, default=3, help="served: batches on the device at once")
    ap.add_argument("--served-max-log2", type=int, default=26, help="served: largest request, 2^x elements")
    ap.add_argument("--verify-requests", type=int, default=200, help="served: requests checked against the oracle")
    ap.add_argument("--segments", type=int, default=100_000, help="batched: number of arrays")
    ap.add_argument("--batched-total-log2", type=int, default=0,
                    help="batched: draw arrays until this many keys (2^x) instead of --segments")
    ap.add_argument("--verify-segments", type=int, default=200, help="batched: arrays checked against the oracle")
    ap.add_argument("--autotune", action="store_true",
                    help="batched: tune leaves / alpha per size class first and sort with that table")
    ap.add_argument("--record-path", type=int, default=0, choices=[0, 1],
                    help="100-byte records: 0 key + index indirection (default), 1 in-place blocks")
    ap.add_argument("--strict", action="store_true",
                    help="plain workload: time ips4o_sort_strict (Section 4.6, workspace independent of n)")
    ap.add_argument("--segment-scheduler", type=int, default=0, choices=[0, 1, 2, 3],
                    help="batched: 0 automatic, 1 level by level, 2 one CTA per array, "
                         "3 the enqueue-only ips4o_sort_segmented_async")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
