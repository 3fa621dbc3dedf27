"""Host check of the request server's device-memory arena (row a12: served
requests take their workspace and staging buffers from one arena allocated
at creation): a first-fit allocator with coalescing, driven by random
allocations and releases against a granule model (arena_check.cu, compiled
here with nvcc; the library calls the server file makes are stubbed, and
nothing runs on a GPU).  Every allocation lies inside the arena on free
granules at the first free run that holds it, an allocation fails only when
no free run holds it, and releasing everything restores one block."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_arena_first_fit_and_coalescing(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "arena_check")
    cmd = [nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=compute_103a",
           "-I", os.path.join(ROOT, "include"), "-o", exe, os.path.join(HERE, "arena_check.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.splitlines()[-1] == "OK 0", r.stdout[-3000:]
