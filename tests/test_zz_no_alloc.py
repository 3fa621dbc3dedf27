"""exsum_excluded_noalloc: excluded sums for callers that cannot allocate.

Some callers of this library cannot call cudaMalloc when they need a result
(a plugin whose host framework owns all device memory, a real-time loop that
cannot take cudaMalloc's implicit synchronisation).  The no-allocation entry
point runs the excluded-sum pipeline on a static device buffer built into the
library.  These checks call it through the C ABI and compare it with the
regular entry point, twice in a row on the shared buffer.  The file is named
to run last in a suite.
"""

import numpy as np
import pytest

import paper_2106_00124_gb300 as ex
from helpers import check, seeded, to_device

pytestmark = pytest.mark.gpu

CASES = [
    ((37, 41, 29), (5, 8, 3), "f32", "add"),
    ((64, 300), (16, 17), "i64", "max"),
    ((5000,), (333,), "bf16", "add"),
]


def _noalloc(x, shape, k, op, dtype):
    import torch
    out_dtype = {"i32": torch.int32, "i64": torch.int64}.get(dtype, torch.float32)
    out = torch.full(shape, -7, dtype=out_dtype, device=x.device)
    rc = ex.exsum_excluded_noalloc(x.data_ptr(), out.data_ptr(), len(shape), shape, k,
                                   ex.OPS[op], ex.DTYPES[dtype],
                                   torch.cuda.current_stream().cuda_stream)
    assert rc == ex.EXSUM_OK, ex.strerror(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("shape,k,dtype,op", CASES)
def test_noalloc_matches_excluded_two_calls(shape, k, dtype, op):
    import torch
    dev, _ = seeded(shape, dtype, 99, op)
    x = to_device(dev, dtype)
    ref = ex.excluded(x, k, op)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    for call in range(2):
        got = _noalloc(x, shape, k, op, dtype)
        check(got, ref.astype(np.float64) if ref.dtype.kind == "f" else ref, dtype, op,
              "noalloc call %d" % call)


def test_noalloc_rejects_oversize_without_work():
    import torch
    shape, k = (512, 512, 512), (8, 8, 8)
    need, st = ex.exsum_workspace_bytes(3, shape, k, ex.OP_ADD, ex.F32, 1)
    assert st == 0 and need > ex.NOALLOC_SCRATCH_BYTES
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    rc = ex.exsum_excluded_noalloc(x.data_ptr(), x.data_ptr() + 16, 3, shape, k, ex.OP_ADD,
                                   ex.F32, 0)
    assert rc == ex.EXSUM_ENOMEM


def test_noalloc_allocates_nothing_and_forks_nothing():
    """The promise itself: with the library's cached workspaces released and
    the launch trace off, calls on a stream the library has never seen leave
    the device's free memory and the library's side-stream count unchanged
    (the first call on the device, which loads the library image holding the
    static buffer, is made before measuring)."""
    import torch
    shape, k, dtype, op = CASES[0]
    dev, _ = seeded(shape, dtype, 98, op)
    x = to_device(dev, dtype)
    _noalloc(x, shape, k, op, dtype)          # first call on this device
    assert ex.exsum_release_cached_workspace() == ex.EXSUM_OK
    ex.exsum_trace_enable(False)
    s = torch.cuda.Stream()
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    streams0 = ex.exsum_side_streams_created()
    for _ in range(2):
        rc = ex.exsum_excluded_noalloc(x.data_ptr(), out.data_ptr(), len(shape), shape, k,
                                       ex.OPS[op], ex.DTYPES[dtype], s.cuda_stream)
        assert rc == ex.EXSUM_OK, ex.strerror(rc)
    s.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert ex.exsum_side_streams_created() == streams0
