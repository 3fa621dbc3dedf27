"""Graphs instantiated by the library (exsum_graph_instantiate): a captured
excluded sum, replayed through exsum_graph_launch, equals the direct call
bit for bit, and the helpers reject null handles."""

import numpy as np
import pytest

import paper_2106_00124_gb300 as ex
from helpers import seeded, to_device


def test_graph_helpers_reject_null():
    with pytest.raises(ex.ExsumError):
        ex.exsum_graph_launch(0)
    with pytest.raises(ex.ExsumError):
        ex.exsum_graph_exec_destroy(0)


@pytest.mark.gpu
@pytest.mark.parametrize("shape,k", [((64, 96, 256), (8, 8, 8)), ((40, 300), (7, 9)), ((9, 17, 33), (2, 8, 5))])
def test_captured_graph_equals_direct_call(shape, k):
    import torch
    dev, _ = seeded(shape, "f32", 77, "add")
    x = to_device(dev, "f32")
    ref = ex.excluded(x, k, "add")
    torch.cuda.synchronize()
    out = torch.empty_like(x)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())

    def call(s):
        ex.exsum_excluded(x.data_ptr(), out.data_ptr(), x.dim(), list(shape), list(k), ex.OP_ADD,
                          ex.F32, s)

    with torch.cuda.stream(st):
        call(st.cuda_stream)  # side streams exist before the capture
    st.synchronize()
    g = torch.cuda.CUDAGraph(keep_graph=True)
    with torch.cuda.graph(g, stream=st):
        call(st.cuda_stream)
    exe = ex.exsum_graph_instantiate(g.raw_cuda_graph())
    try:
        for _ in range(3):
            out.fill_(float("nan"))
            ex.exsum_graph_launch(exe, st.cuda_stream)
            st.synchronize()
            assert torch.equal(out, ref)
    finally:
        ex.exsum_graph_exec_destroy(exe)
