"""Weak excluded sums (BDBS complement, Sec. 1 / Sec. 6 "BDBSC"): total minus
included, integer + only.  Checked against the oracle's BDBSC and against the
strong excluded sum, which it equals exactly for wrapping integer +."""

import zlib

import numpy as np
import pytest

import paper_2106_00124_gb300 as ex
from helpers import seeded, to_device
from oracle import oracle as O

CASES = [((1,), (1,)), ((1000,), (64,)), ((37, 29), (5, 29)), ((9, 17, 33), (2, 8, 5)),
         ((64, 96, 256), (8, 8, 8)), ((5, 6, 7, 8), (2, 3, 4, 5)), ((70, 300), (33, 31))]


def test_weak_rejects_float_and_bad_args():
    shape, k = (4, 5), (2, 2)
    for dt in (ex.F32, ex.BF16):
        assert ex.exsum_excluded_weak(1, 1, 2, shape, k, dt) == ex.EXSUM_EUNSUPPORTED
    assert ex.exsum_excluded_weak(1, 1, 2, shape, (9, 2), ex.I32) == ex.EXSUM_EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["i32", "i64"])
@pytest.mark.parametrize("shape,k", CASES, ids=[str(c[0]) + "k" + str(c[1]) for c in CASES])
def test_weak_equals_oracle_and_strong(shape, k, dtype):
    import torch
    dev, vals = seeded(shape, dtype, zlib.crc32(repr((shape, k, dtype)).encode()) & 0xFFFF, "add")
    x = to_device(dev, dtype)
    weak = ex.excluded_weak(x, k)
    strong = ex.excluded(x, k, "add")
    torch.cuda.synchronize()
    assert torch.equal(weak, strong)
    ref = O.bdbsc(np.asarray(vals, dtype=np.int64), k)
    got = weak.cpu().numpy().astype(np.int64)
    if dtype == "i32":
        ref = ref.astype(np.int32).astype(np.int64)   # int32 + wraps modulo 2^32
    assert np.array_equal(got, ref)
