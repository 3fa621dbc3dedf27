"""The paper's comparison methods on the GPU: summed-area tables with
inclusion-exclusion (SAT / SATC, Sec. 1) and corners (App. A).

CPU: the corner regions tile the complement of the box exactly -- every one
of the 3^d cells (below / inside / above the box in each dimension) but the
box itself lies in exactly one region, for d = 2 and 3 -- and the entry
points reject what they do not handle before any device work.
GPU: both against the oracle, element by element (bit-exact for integers
and max, the floored 1e-5 bound for fp +).
"""

import itertools
import zlib

import numpy as np
import pytest

import paper_2106_00124_gb300 as ex
from helpers import check, oracle_sum, seeded, to_device

# region r of a dimension covers these cells: B below x, I inside [x, x+k), A from x+k on
REGION_CELLS = {0: {"B"}, 1: {"B", "I"}, 2: {"I", "A"}, 3: {"A"}}


@pytest.mark.parametrize("d", [2, 3])
def test_corner_regions_tile_the_complement(d):
    regions = [[ex.exsum_corner_region(d, c, i) for i in range(d)] for c in range(1 << d)]
    assert all(0 <= r <= 3 for reg in regions for r in reg)
    # distinct prefix / suffix patterns: one corner tensor per region
    patterns = {tuple(r >= 2 for r in reg) for reg in regions}
    assert len(patterns) == 1 << d
    for cell in itertools.product("BIA", repeat=d):
        hits = sum(all(cell[i] in REGION_CELLS[reg[i]] for i in range(d)) for reg in regions)
        assert hits == (0 if all(c == "I" for c in cell) else 1), cell


def test_corner_region_rejects_out_of_range():
    assert ex.exsum_corner_region(4, 0, 0) == -1
    assert ex.exsum_corner_region(2, 4, 0) == -1
    assert ex.exsum_corner_region(3, 0, 3) == -1


def test_comparators_reject_without_gpu():
    sh, k = [4, 4], [2, 2]
    assert ex.exsum_sat(16, 32, 2, sh, k, 1, ex.F32) == ex.EXSUM_EUNSUPPORTED
    assert ex.exsum_sat(16, 32, 2, sh, [5, 2], 1, ex.I64) == ex.EXSUM_EINVAL
    assert ex.exsum_corners(16, 32, 4, [2, 2, 2, 2], [1, 1, 1, 1], ex.OP_ADD, ex.I64) == ex.EXSUM_EUNSUPPORTED
    assert ex.exsum_corners(0, 32, 2, sh, k, ex.OP_ADD, ex.I64) == ex.EXSUM_EINVAL


SAT_CASES = [((1000,), (37,)), ((37, 41), (5, 40)), ((19, 23, 29), (4, 23, 1)), ((6, 7, 8, 9), (2, 3, 4, 5)),
             ((256, 256), (16, 16)), ((3, 5, 2, 4, 3), (2, 2, 2, 2, 2)),
             # long lines in few of them: segmented scans with carries
             ((100000,), (777,)), ((4096, 8), (100, 3)), ((3, 20000), (2, 999))]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["i32", "i64"])
@pytest.mark.parametrize("excluded", [0, 1])
@pytest.mark.parametrize("shape,k", SAT_CASES, ids=[str(c[0]) + "k" + str(c[1]) for c in SAT_CASES])
def test_sat_matches_oracle(shape, k, excluded, dtype):
    seed = zlib.crc32(repr((shape, k, dtype, "sat")).encode()) & 0xFFFFFF
    dev, vals = seeded(shape, dtype, seed, "add")
    got = ex.sat(to_device(dev, dtype), k, excluded=bool(excluded)).cpu().numpy()
    ref = oracle_sum("excluded" if excluded else "included", vals, k, "add")
    check(got, ref, dtype, "add", "sat %s %s k=%s excluded=%d" % (dtype, shape, k, excluded))


CORNER_CASES = [((37, 41), (5, 40)), ((256, 256), (16, 16)), ((1, 9), (1, 9)), ((50, 3), (50, 1)),
                ((19, 23, 29), (4, 23, 1)), ((64, 64, 64), (8, 8, 8)), ((5, 1, 7), (2, 1, 7)),
                ((30, 31, 33), (30, 5, 2)),
                # segmented scans (few long lines), both directions
                ((2000, 5), (30, 2)), ((3, 20000), (2, 999)), ((5000, 2, 3), (7, 2, 1))]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,op", [("i64", "add"), ("i32", "max"), ("i32", "add"), ("i64", "max"),
                                      ("f32", "add"), ("f32", "max"), ("bf16", "add")])
@pytest.mark.parametrize("shape,k", CORNER_CASES, ids=[str(c[0]) + "k" + str(c[1]) for c in CORNER_CASES])
def test_corners_match_oracle(shape, k, dtype, op):
    seed = zlib.crc32(repr((shape, k, dtype, op, "corners")).encode()) & 0xFFFFFF
    dev, vals = seeded(shape, dtype, seed, op)
    got = ex.corners(to_device(dev, dtype), k, op).cpu().numpy()
    ref = oracle_sum("excluded", vals, k, op)
    check(got, ref.astype(np.float64) if dtype in ("f32", "bf16") else ref, dtype, op,
          "corners %s %s %s k=%s" % (dtype, op, shape, k))


def test_slowed_operator_rejects_without_gpu():
    assert ex.exsum_slow_extra(-1) == ex.EXSUM_EINVAL
    assert ex.exsum_slow_run(16, 32, 2, [4, 4], [2, 2], 9, 0) == ex.EXSUM_EINVAL
    assert ex.exsum_slow_run(16, 32, 4, [2, 2, 2, 2], [1, 1, 1, 1], ex.SLOW_CORNERS, 0) == ex.EXSUM_EUNSUPPORTED


@pytest.mark.gpu
@pytest.mark.parametrize("extra", [0, 3])
@pytest.mark.parametrize("shape,k", [((37, 41), (5, 40)), ((19, 23, 29), (4, 23, 1)), ((9, 8, 7, 6), (2, 3, 4, 5))])
def test_slowed_operator_pipelines_match_oracle(shape, k, extra):
    """The slowed int64 + gives the plain sums: box-complement, BDBS and
    corners through it match the oracle bit for bit, and the calibration
    kernel applies the operator the stated number of times."""
    import torch
    seed = zlib.crc32(repr((shape, k, "slow")).encode()) & 0xFFFFFF
    dev, vals = seeded(shape, "i64", seed, "add")
    x = to_device(dev, "i64")
    out = torch.empty_like(x)
    s = torch.cuda.current_stream().cuda_stream
    assert ex.exsum_slow_extra(extra) == ex.EXSUM_OK
    try:
        methods = [(ex.SLOW_BOX_COMPLEMENT, "excluded"), (ex.SLOW_BDBS, "included")]
        if len(shape) in (2, 3):
            methods.append((ex.SLOW_CORNERS, "excluded"))
        for m, kind in methods:
            out.fill_(5)
            assert ex.exsum_slow_run(x.data_ptr(), out.data_ptr(), len(shape), shape, k, m, s) == ex.EXSUM_OK
            torch.cuda.synchronize()
            check(out.cpu().numpy(), oracle_sum(kind, vals, k, "add"), "i64", "add", "slowed %d %s" % (m, shape))
        assert ex.exsum_slow_run(x.data_ptr(), out.data_ptr(), len(shape), shape, k, ex.SLOW_CALIBRATE, s) == 0
        torch.cuda.synchronize()
        assert torch.equal(out, x * (ex.SLOW_CALIBRATE_REPS + 1))
    finally:
        ex.exsum_slow_extra(0)
