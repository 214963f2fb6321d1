"""The splitter lookup table of the local classification, on the CPU.

`tests/host/lut_check.cu` includes the library's own `ips4o_common.cuh`
(the lut_* functions are host and device code) and checks both cell maps
against brute-force counting of the splitters <= e, for random and
adversarial splitter sets.  It is built with nvcc for the host only; no GPU
is used.
"""
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


def test_lookup_table_equals_brute_force_count(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "lut_check")
    cmd = [nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
           os.path.join(HERE, "host", "lut_check.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe, "600"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok "), r.stdout + r.stderr
    assert int(r.stdout.split()[1]) > 1_000_000


def test_noalloc_scratch_holds_every_accepted_sort(tmp_path):
    """ips4o_sort_noalloc refuses sizes above 2^20 elements; below that its
    fixed 16 MiB device scratch and 1 MiB host staging must hold the
    workspace the driver's sizing rules ask for, for every element type and
    any SM count up to 160 (tests/host/noalloc_fit.cu, host only)."""
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "noalloc_fit")
    cmd = [nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
           os.path.join(HERE, "host", "noalloc_fit.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok "), r.stdout + r.stderr


def test_exhausted_bitmap_search_equals_bit_by_bit(tmp_path):
    """first_live_bucket, the block permutation's search for the next bucket
    with unprocessed blocks, against testing the bits one at a time for
    every start and many bitmaps (tests/host/bitmap_check.cu, host only)."""
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "bitmap_check")
    cmd = [nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
           os.path.join(HERE, "host", "bitmap_check.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok "), r.stdout + r.stderr
    assert int(r.stdout.split()[1]) > 1_000_000
