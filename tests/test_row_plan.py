"""Host sweep of the final-pass planners of the row schedule (Sec. 4): the
tile plans of k_rowx and of the bulk-staged k_rowx_bulk for every row length
the kernels take (16 .. 1024 elements of 4 bytes, 16 .. 512 of 8; 128 .. 1024
for the bulk pass) over a grid of slice heights, slice counts, windows along
n_{d-1} and SM counts.  A host program (row_plan_check.cu, compiled here with
nvcc, launching nothing) checks each plan against what its kernel relies on:
shared memory within a block's limit and holding the tile, tiles covering
every row of a slice with none empty, staged rows holding the window's halo,
strips covering a row, grids below 2^31 blocks; and that a plan is refused
only where the grid would overflow (the bulk pass also where a wide window
leaves no room, which k_rowx then takes)."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_final_pass_plans_hold_their_tiles(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "row_plan_check")
    cmd = [nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=compute_103a",
           "-I", os.path.join(ROOT, "include"), "-o", exe, os.path.join(HERE, "row_plan_check.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.splitlines()
    bad = [ln for ln in lines if ln.startswith("V ")]
    assert lines[-1] == "BAD 0", "\n".join(bad)
    counts = {tuple(ln.split()[:2]): [int(v) for v in ln.split()[2:]] for ln in lines if ln[:2] in ("R ", "B ")}
    # every sweep planned most of its cases
    assert set(counts) == {("R", "f32"), ("R", "i64"), ("B", "f32")}
    for key, (ok, refused) in counts.items():
        assert ok > refused, key
