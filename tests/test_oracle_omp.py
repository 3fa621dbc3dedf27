"""The OpenMP variant of the box-complement oracle (used to time the
all-core CPU baseline) gives the single-threaded oracle's results bit for
bit: it performs the same steps with the same operand order, only on
several host threads.  CPU only."""

import zlib

import numpy as np
import pytest

from oracle import oracle as O

CASES = [
    ((7, 9, 11), (3, 4, 5), "add", "float"),
    ((7, 9, 11), (7, 9, 11), "max", "float"),
    ((5, 6, 7, 8), (2, 3, 4, 5), "max", "int"),
    ((5, 6, 7, 8), (1, 1, 1, 1), "add", "int"),
    ((300,), (17,), "add", "int"),
    ((1,), (1,), "add", "float"),
    ((40, 50), (40, 1), "add", "float"),
    ((6, 5, 4, 3, 2), (6, 1, 4, 1, 2), "max", "float"),
    ((33, 34, 35), (8, 8, 8), "add", "float"),
]


@pytest.mark.parametrize("shape,k,op,kind", CASES)
def test_omp_oracle_equals_single_threaded(shape, k, op, kind):
    rng = np.random.default_rng(zlib.crc32(repr((shape, k, op, kind)).encode()))
    a = rng.uniform(-1, 1, shape) if kind == "float" else rng.integers(-1000, 1000, shape)
    ref = O.box_complement(a, k, op)
    got = O.box_complement_omp(a, k, op)
    assert np.array_equal(ref.view(np.int64), got.view(np.int64))


def test_omp_oracle_reports_threads():
    assert O.omp_threads() >= 1
