"""GPU parity: the CUDA library against the CPU oracle, element by element,
on seeded inputs that span several tiles and ragged tails, for every dtype,
operator and problem (included / excluded)."""

import zlib

import numpy as np
import pytest

from helpers import check, gpu_sum, oracle_sum, seeded, to_device

pytestmark = pytest.mark.gpu

DTYPES = ["i32", "i64", "f32", "bf16"]
OPS = ["add", "max"]
KINDS = ["included", "excluded"]

# (shape, k): ragged sizes, k = 1, k = n, k not dividing n, k larger than the
# segment and chunk lengths of the kernels, and up to eight dimensions.
CASES = [
    ((1,), (1,)),
    ((7,), (3,)),
    ((33,), (33,)),
    ((100,), (45,)),
    ((1000,), (64,)),
    ((5000,), (1,)),
    ((4099,), (700,)),
    ((37, 29), (5, 29)),
    ((64, 64), (16, 16)),
    ((1, 300), (1, 17)),
    ((300, 1), (299, 1)),
    ((9, 17, 33), (2, 8, 5)),
    ((40, 5, 70), (40, 1, 3)),
    ((3, 130, 2), (2, 65, 1)),
    ((5, 6, 7, 8), (2, 3, 4, 5)),
    ((3, 4, 5, 3, 4), (1, 2, 5, 3, 2)),
    ((2, 2, 2, 2, 2, 2, 2, 3), (1, 2, 1, 2, 2, 1, 2, 3)),
    ((300000,), (4500,)),
    ((300000,), (32,)),
    ((5000, 3), (100, 2)),
    ((3, 517), (2, 32)),
    ((70, 300), (33, 31)),
    ((7, 129, 131), (7, 17, 9)),
    # last dimension peeled first (rows of 16 .. 1024): several slices per
    # block with a ragged last group, several row tiles with the window along
    # dimension d-1 fused (widths up to 32) or run as its own pass, k_d = 1,
    # k_d = n_d, strips that do not fill 4-element vectors
    ((33, 16), (7, 16)),
    ((29, 3, 20), (3, 2, 5)),
    ((3, 100, 256), (2, 9, 17)),
    ((130, 64), (20, 5)),
    ((12, 40), (9, 3)),
    ((3, 1024), (2, 100)),
    ((4, 257), (3, 256)),
    ((20, 50), (4, 1)),
    ((3, 4, 5, 40), (2, 3, 4, 7)),
    ((4, 5, 64), (1, 1, 8)),
    # the lower-dimensional problem one-dimensional but too long (or its box
    # too wide) to fold into the final pass
    ((5000, 20), (3, 4)),
    ((300, 40), (100, 5)),
    # rows longer than the peeled schedule takes
    ((5, 1500), (2, 40)),
    ((4, 6, 1100), (3, 2, 9)),
]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape,k", CASES, ids=[str(c[0]) + "k" + str(c[1]) for c in CASES])
def test_parity_small(shape, k, dtype, op, kind):
    seed = zlib.crc32(repr((shape, k, dtype, op)).encode()) & 0xFFFFFF
    dev, vals = seeded(shape, dtype, seed, op)
    got = gpu_sum(kind, to_device(dev, dtype), k, op)
    ref = oracle_sum(kind, vals, k, op)
    check(got, ref, dtype, op, "%s %s %s %s k=%s" % (kind, dtype, op, shape, k))


@pytest.mark.parametrize("kind", KINDS)
def test_int32_add_wraps(kind):
    from paper_2106_00124_gb300 import synth
    shape, k = (50, 60), (7, 9)
    vals = synth.uniform_int(shape, -(1 << 31), (1 << 31) - 1, seed=12, dtype=np.int32)
    got = gpu_sum(kind, to_device(vals, "i32"), k, "add")
    check(got, oracle_sum(kind, vals, k, "add"), "i32", "add", kind)


def test_repeat_calls_identical():
    """The same call twice gives identical bits (deterministic reduction order)."""
    dev, _ = seeded((31, 40, 50), "f32", 5, "add")
    x = to_device(dev, "f32")
    a = gpu_sum("excluded", x, (4, 8, 16), "add")
    b = gpu_sum("excluded", x, (4, 8, 16), "add")
    assert np.array_equal(a, b)


# Inputs and outputs one element past an aligned allocation: the staged,
# vectorised and 16-byte-store paths must fall back to element accesses.
MISALIGNED = [((9, 17, 33), (2, 8, 5)), ((3, 100, 256), (2, 9, 17)), ((29, 3, 20), (3, 2, 5)),
              ((64, 64), (16, 16)), ((40, 5, 72), (3, 1, 8)), ((300, 3), (7, 2))]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("shape,k", MISALIGNED, ids=[str(c[0]) + "k" + str(c[1]) for c in MISALIGNED])
def test_parity_misaligned(shape, k, dtype, kind):
    import torch
    import paper_2106_00124_gb300 as ex
    dev, vals = seeded(shape, dtype, 991, "add")
    x0 = to_device(dev, dtype)
    n = x0.numel()
    x = torch.empty(n + 1, dtype=x0.dtype, device="cuda")[1:].view(shape)
    x.copy_(x0)
    out_dt = torch.float32 if dtype == "bf16" else x0.dtype
    out = torch.empty(n + 1, dtype=out_dt, device="cuda")[1:].view(shape)
    assert x.data_ptr() % 16 != 0 and out.data_ptr() % 16 != 0
    fn = ex.excluded if kind == "excluded" else ex.included
    fn(x, k, "add", out=out)
    torch.cuda.synchronize()
    check(out.cpu().numpy(), oracle_sum(kind, vals, k, "add"), dtype, "add",
          "misaligned %s %s %s k=%s" % (kind, dtype, shape, k))


# Enough slices that every block of the final pass stages and computes many
# tiles in turn (its shared buffers reused), with rows padded to the strip
# width (76, 36, 300) or filling it exactly (256, 32, 128); windows along the
# second-to-last dimension fused in every case.
MANY_TILES = [
    ((40, 40, 40, 76), (2, 3, 4, 5)),
    ((24, 24, 40, 36), (3, 2, 5, 7)),
    ((12, 12, 12, 32, 32), (2, 2, 2, 4, 4)),
    ((600, 40, 128), (3, 8, 16)),
    ((300, 64, 256), (2, 8, 8)),
    ((200, 20, 300), (5, 6, 30)),
]


@pytest.mark.parametrize("dtype,op", [("f32", "add"), ("i32", "max"), ("bf16", "add")])
@pytest.mark.parametrize("shape,k", MANY_TILES, ids=[str(c[0]) + "k" + str(c[1]) for c in MANY_TILES])
def test_parity_many_tiles_per_block(shape, k, dtype, op):
    seed = zlib.crc32(repr((shape, k, dtype, op, "many")).encode()) & 0xFFFFFF
    dev, vals = seeded(shape, dtype, seed, op)
    got = gpu_sum("excluded", to_device(dev, dtype), k, op)
    check(got, oracle_sum("excluded", vals, k, op), dtype, op,
          "many tiles %s %s %s k=%s" % (dtype, op, shape, k))


# Lower problems of many planes: the two-dimensional excluded sum runs one
# warp per plane (d = 2 tensors of >= 1216 rows, and d = 3 tensors whose
# first dimension is that long), including planes of one column, boxes
# covering the whole plane and windows reaching past the last plane.
MANY_PLANES = [
    ((1500, 37), (5, 7)),
    ((4000, 60), (64, 3)),
    ((1300, 700), (16, 600)),
    ((2048, 1), (9, 1)),
    ((1300, 20, 16), (10, 3, 4)),
    ((1250, 9, 33), (64, 9, 2)),
]


@pytest.mark.parametrize("dtype,op", [("f32", "add"), ("i64", "max"), ("i32", "add"), ("bf16", "add")])
@pytest.mark.parametrize("shape,k", MANY_PLANES, ids=[str(c[0]) + "k" + str(c[1]) for c in MANY_PLANES])
def test_parity_many_planes(shape, k, dtype, op):
    seed = zlib.crc32(repr((shape, k, dtype, op, "planes")).encode()) & 0xFFFFFF
    dev, vals = seeded(shape, dtype, seed, op)
    got = gpu_sum("excluded", to_device(dev, dtype), k, op)
    check(got, oracle_sum("excluded", vals, k, op), dtype, op,
          "many planes %s %s %s k=%s" % (dtype, op, shape, k))


# Boxes longer than 32 along a dimension: the strided passes keep each
# block's suffixes in the output (one thread per block of k lines), the
# contiguous passes run one warp per segment of whole blocks of a row.
# Rows longer than a segment, boxes that do not divide the side, a box of the
# whole side, boxes over 32 along every dimension, and d = 1.
BIG_K = [
    ((300, 40), (33, 37)),
    ((5, 3000), (2, 255)),
    ((70, 9, 130), (64, 9, 100)),
    ((257, 33), (256, 33)),
    ((3, 4, 2500), (3, 1, 1000)),
    ((40, 50, 60), (40, 50, 60)),
    ((12000,), (4000,)),
    ((64, 1100), (1, 300)),
]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype,op", [("f32", "add"), ("i64", "add"), ("i32", "max"), ("bf16", "add"),
                                      ("f32", "max")])
@pytest.mark.parametrize("shape,k", BIG_K, ids=[str(c[0]) + "k" + str(c[1]) for c in BIG_K])
def test_parity_boxes_over_32(shape, k, dtype, op, kind):
    seed = zlib.crc32(repr((shape, k, dtype, op, kind, "bigk")).encode()) & 0xFFFFFF
    dev, vals = seeded(shape, dtype, seed, op)
    got = gpu_sum(kind, to_device(dev, dtype), k, op)
    check(got, oracle_sum(kind, vals, k, op), dtype, op,
          "boxes over 32 %s %s %s %s k=%s" % (kind, dtype, op, shape, k))


# Rows of 128 .. 1024 elements whose length is not a multiple of 4: the
# bulk-staged final pass copies each tile from the 16-byte boundary before
# it (the tile's data shifted by 0 .. 3 elements), loads the last elements
# after the last boundary one by one, and writes every warp's rows as one
# run realigned to 16-byte stores.  Windows along n_2 of each compile-time
# bound (1, 4, 8, 16, 32), suffix offsets k_d both multiples of 4 and not,
# several tiles per slice and a short last tile.
ODD_ROWS = [
    ((3, 70, 129), (2, 1, 5)),
    ((2, 100, 131), (1, 4, 8)),
    ((4, 33, 130), (3, 8, 130)),
    ((2, 90, 255), (2, 16, 3)),
    ((2, 40, 997), (1, 32, 500)),
    ((1, 77, 1023), (1, 5, 1)),
    ((5, 300, 150), (3, 7, 4)),
    ((300, 131), (3, 9)),
]


@pytest.mark.parametrize("dtype,op", [("f32", "add"), ("i32", "max"), ("i32", "add"), ("f32", "max"),
                                      ("bf16", "add")])
@pytest.mark.parametrize("shape,k", ODD_ROWS, ids=[str(c[0]) + "k" + str(c[1]) for c in ODD_ROWS])
def test_parity_odd_rows(shape, k, dtype, op):
    seed = zlib.crc32(repr((shape, k, dtype, op, "odd")).encode()) & 0xFFFFFF
    dev, vals = seeded(shape, dtype, seed, op)
    got = gpu_sum("excluded", to_device(dev, dtype), k, op)
    check(got, oracle_sum("excluded", vals, k, op), dtype, op,
          "odd rows %s %s %s k=%s" % (dtype, op, shape, k))


def test_no_bulk_copy_wait_gave_up():
    """The bulk final pass's bounded waits for its tile copies never run out
    (the library's counter of blocks that gave up stays at zero) over calls
    through every bulk variant: even and odd row lengths, one and two
    staging buffers."""
    import torch

    import paper_2106_00124_gb300 as ex
    for shape, k in [((64, 256, 256), (8, 8, 8)), ((3, 70, 129), (2, 1, 5)), ((2, 40, 997), (1, 32, 500)),
                     ((8, 300, 1024), (2, 16, 9))]:
        x = torch.rand(shape, device="cuda") - 0.5
        ex.excluded(x, k, "add")
    torch.cuda.synchronize()
    assert ex.exsum_device_timeouts() == 0


# Rows longer than one warp scans (1025 .. 16384 elements; 8-byte local
# types up to 8192): the row schedule with one block per row in the final
# pass (strips of 4 .. 32 elements per thread, compensated scans across
# them).  Suffix offsets inside a strip, across strips and past the row end;
# d = 2 (a one-dimensional lower problem) and d = 3.
LONG_ROWS = [
    ((5, 1025), (2, 1)),
    ((7, 2048), (3, 700)),
    ((3, 3001), (1, 33)),
    ((4, 4097), (4, 4097)),
    ((2, 3, 8192), (2, 2, 5)),
    ((3, 2, 16384), (1, 2, 9000)),
    ((6, 5000), (6, 1)),
]


@pytest.mark.parametrize("dtype,op", [("f32", "add"), ("i64", "add"), ("i32", "max"), ("bf16", "add"),
                                      ("i64", "max")])
@pytest.mark.parametrize("shape,k", LONG_ROWS, ids=[str(c[0]) + "k" + str(c[1]) for c in LONG_ROWS])
def test_parity_long_rows(shape, k, dtype, op, monkeypatch):
    # every shape the long-row pass can hold (by default only d = 2 rows of
    # at most 4096 elements take it; the others take the dimension-1 schedule,
    # which the rest of this file covers)
    monkeypatch.setenv("EXSUM_LONGROW", "2")
    seed = zlib.crc32(repr((shape, k, dtype, op, "long")).encode()) & 0xFFFFFF
    dev, vals = seeded(shape, dtype, seed, op)
    got = gpu_sum("excluded", to_device(dev, dtype), k, op)
    check(got, oracle_sum("excluded", vals, k, op), dtype, op,
          "long rows %s %s %s k=%s" % (dtype, op, shape, k))
