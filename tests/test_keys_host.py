"""The order-preserving key maps of the element types (ips4o_common.cuh, host
and device code) against the plain definitions of their total orders, on
the CPU: IEEE '<' for f64 with -0.0 < +0.0 and NaNs at the ends, memcmp of
bytes [0, 10) for 100-byte records, lexicographic (k0, k1, k2) for quartets
(tests/host/keys_check.cu, built with nvcc for the host only; no GPU)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1705_02257_gb300", "csrc")


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_key_maps_follow_the_total_orders(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "keys_check")
    cmd = [nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
           os.path.join(HERE, "host", "keys_check.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok "), r.stdout + r.stderr
    assert int(r.stdout.split()[1]) > 300_000
