"""C-ABI checks that need no GPU: the library loads, exports every function
that include/exsum.h declares, sizes workspaces and rejects bad arguments
before touching the device."""

import ctypes
import os
import re

import pytest

import paper_2106_00124_gb300 as ex

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(exsum_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(ex.LIB_PATH):
        from paper_2106_00124_gb300 import build
        build.build()
    return ex._load()


def test_header_declares_functions():
    names = _header_functions()
    assert "exsum_included" in names and "exsum_excluded" in names
    assert len(names) >= 10


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(ex.LIB_PATH)
    missing = [n for n in _header_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_binding_covers_header(lib):
    """The Python binding mirrors every C entry point under the same name."""
    assert set(_header_functions()) <= set(ex.declared_symbols())
    for name in _header_functions():
        assert hasattr(ex, name), name


def test_version_and_strings(lib):
    assert ex.exsum_version() >= 10000
    assert ex.strerror(ex.EXSUM_EINVAL) == "invalid argument"
    assert ex.exsum_out_dtype(ex.BF16) == ex.F32
    assert ex.exsum_out_dtype(ex.I64) == ex.I64
    assert ex.exsum_out_dtype(9) == -1
    assert [ex.exsum_dtype_size(t) for t in (ex.I32, ex.I64, ex.F32, ex.BF16)] == [4, 8, 4, 2]


@pytest.mark.parametrize("d,shape,k", [
    (0, [], []), (9, [2] * 9, [1] * 9), (2, [4, 0], [1, 1]), (2, [4, 4], [0, 1]),
    (2, [4, 4], [5, 1]), (1, [3], [4]),
])
def test_invalid_shapes_rejected_without_gpu(lib, d, shape, k):
    shape = shape or [1]
    k = k or [1]
    nbytes, st = ex.exsum_workspace_bytes(d, shape, k, ex.OP_ADD, ex.F32, 1)
    assert st == ex.EXSUM_EINVAL and nbytes == 0
    # argument checks happen before any device work, so a null pointer is never touched
    assert ex.exsum_excluded(1, 2, d, shape, k, ex.OP_ADD, ex.F32, 0) == ex.EXSUM_EINVAL
    assert ex.exsum_included(1, 2, d, shape, k, ex.OP_ADD, ex.F32, 0) == ex.EXSUM_EINVAL


def test_invalid_op_dtype_rejected(lib):
    assert ex.exsum_workspace_bytes(2, [4, 4], [2, 2], 7, ex.F32, 1)[1] == ex.EXSUM_EINVAL
    assert ex.exsum_workspace_bytes(2, [4, 4], [2, 2], ex.OP_ADD, 11, 1)[1] == ex.EXSUM_EINVAL
    assert ex.exsum_excluded(None, None, 2, [4, 4], [2, 2], ex.OP_ADD, ex.F32, 0) == ex.EXSUM_EINVAL


def test_workspace_sizes(lib):
    # included d = 1 needs no workspace; multi-dimensional sums need an N-element buffer
    assert ex.exsum_workspace_bytes(1, [1000], [10], ex.OP_ADD, ex.F32, 0) == (0, 0)
    inc2, st = ex.exsum_workspace_bytes(2, [256, 256], [16, 16], ex.OP_ADD, ex.I64, 0)
    assert st == 0 and inc2 >= 256 * 256 * 8
    exc3, st = ex.exsum_workspace_bytes(3, [256] * 3, [8] * 3, ex.OP_ADD, ex.F32, 1)
    assert st == 0 and exc3 >= 256 ** 3 * 4
    # the workspace stays a small multiple of the tensor (Theta(N) space, Sec. 5)
    assert exc3 <= 3 * 256 ** 3 * 4


def test_workspace_query_is_deterministic(lib):
    a = ex.exsum_workspace_bytes(4, [7, 9, 11, 13], [3, 2, 5, 13], ex.OP_MAX, ex.BF16, 1)
    b = ex.exsum_workspace_bytes(4, [7, 9, 11, 13], [3, 2, 5, 13], ex.OP_MAX, ex.BF16, 1)
    assert a == b and a[1] == 0
