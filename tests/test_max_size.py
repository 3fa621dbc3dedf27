"""Beyond 2^31 elements: 64-bit indexing end to end.

A 2-D int32 tensor of 65536 x 32769 = 2,147,549,184 elements (more than
2^31) is summed at full size on the GPU.  Properties that hold at any size
are checked on every element: for integer + (wrapping modulo 2^32),
included + excluded = the tensor total; for max, max(included, excluded) =
the global max.  A few sampled outputs are also checked against the
oracle's point queries (which reduce the whole tensor per point).
"""

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

SHAPE = (65536, 32769)
K = (300, 17)


@pytest.fixture(scope="module")
def big():
    import torch
    if torch.cuda.get_device_properties(0).total_memory < 60 * (1 << 30):
        pytest.skip("needs a large-memory GPU")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2106)
    x = torch.randint(-1000, 1001, SHAPE, generator=gen, device="cuda", dtype=torch.int32)
    yield x
    del x
    torch.cuda.empty_cache()


def test_add_included_plus_excluded_is_total(big):
    import torch
    import paper_2106_00124_gb300 as ex
    inc = ex.included(big, K, "add")
    exc = ex.excluded(big, K, "add")
    total = big.sum(dtype=torch.int64).item()
    total32 = np.array([total], dtype=np.int64).astype(np.int32)[0]
    s = inc + exc                        # int32 wraps, as the library does
    assert bool((s == int(total32)).all())
    # sampled points against the oracle's definition (on a host copy)
    host = big.cpu().numpy()
    rng = np.random.default_rng(1)
    for _ in range(2):
        x = (int(rng.integers(0, SHAPE[0])), int(rng.integers(0, SHAPE[1])))
        ref = O.included_at(host, K, "add", x)
        assert int(inc[x].item()) == int(np.int64(ref).astype(np.int32))
    x = (SHAPE[0] - 1, SHAPE[1] - 5)
    ref = O.excluded_at(host, K, "add", x)
    assert int(exc[x].item()) == int(np.int64(ref).astype(np.int32))
    del inc, exc, s
    torch.cuda.empty_cache()


def test_max_included_excluded_cover_global_max(big):
    import torch
    import paper_2106_00124_gb300 as ex
    inc = ex.included(big, K, "max")
    exc = ex.excluded(big, K, "max")
    gmax = big.max().item()
    assert bool((torch.maximum(inc, exc) == gmax).all())
    del inc, exc
    torch.cuda.empty_cache()


# The row schedule beyond 2^31 elements: rows of 1024 (the longest it takes),
# 2,097,155 rows.  The excluded sum's lower problem is then a line of
# 2,097,155 row totals.
SHAPE_R = (2097155, 1024)
K_R = (5, 7)


@pytest.fixture(scope="module")
def big_rows():
    import torch
    if torch.cuda.get_device_properties(0).total_memory < 60 * (1 << 30):
        pytest.skip("needs a large-memory GPU")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2107)
    x = torch.randint(-1000, 1001, SHAPE_R, generator=gen, device="cuda", dtype=torch.int32)
    yield x
    del x
    torch.cuda.empty_cache()


def test_row_schedule_beyond_2_31(big_rows):
    import torch
    import paper_2106_00124_gb300 as ex
    x = big_rows
    inc = ex.included(x, K_R, "add")
    exc = ex.excluded(x, K_R, "add")
    total = x.sum(dtype=torch.int64).item()
    total32 = int(np.array([total], dtype=np.int64).astype(np.int32)[0])
    assert bool(((inc + exc) == total32).all())
    # points near the start, the middle, 2^31 and the end, each against the
    # oracle's included sum of its box (a small host slice of the tensor)
    pts = [(0, 0), (SHAPE_R[0] // 2, 511), ((1 << 31) // SHAPE_R[1], 1000),
           (SHAPE_R[0] - 1, SHAPE_R[1] - 1), (SHAPE_R[0] - 3, 1020)]
    for p in pts:
        box = x[p[0]:p[0] + K_R[0], p[1]:p[1] + K_R[1]].cpu().numpy()
        kk = tuple(min(a, b) for a, b in zip(K_R, box.shape))  # the box clipped at the edge
        s_box = int(O.included_at(box, kk, "add", (0, 0)))
        assert int(inc[p].item()) == int(np.int64(s_box).astype(np.int32)), p
        assert int(exc[p].item()) == int(np.int64(total - s_box).astype(np.int32)), p
    del inc, exc
    torch.cuda.empty_cache()
    mx_inc = ex.included(x, K_R, "max")
    mx_exc = ex.excluded(x, K_R, "max")
    assert bool((torch.maximum(mx_inc, mx_exc) == x.max()).all())
    del mx_inc, mx_exc
    torch.cuda.empty_cache()
