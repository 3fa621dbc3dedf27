"""GPU parity at the full sizes of the named workloads, against the whole
fp64 / int64 oracle tensor (box-complement run on the host), with the error
of every floating-point result stated.

The fp32/bf16 + results are checked against the fp64 oracle with the floored
relative bound of the other parity tests (|got - ref| <= 1e-5 * max(|ref|,
RMS(ref))); the unfloored maximum relative error and the normwise error
||got - ref|| / ||ref|| are printed beside it (run pytest with -s to see
them).  Integer + and max are bit-exact.
"""

import numpy as np
import pytest

from helpers import check, oracle_sum, to_device
from paper_2106_00124_gb300 import synth

pytestmark = pytest.mark.gpu

FULL = ["d2_256x256_i64_add_k16", "d3_256cube_f32_add_k8", "d3_256cube_i32_max_k8",
        "d1_2p25_f32_add_k64", "d1_2p25_bf16_add_k64", "d4_76p4_f32_add_k4", "d4_76p4_bf16_add_k4",
        "d5_32p5_f32_add_k4", "d5_32p5_bf16_add_k4", "d3_256x512x301_f32_add_k484"]


def _errors(got, ref):
    g = got.astype(np.float64).ravel()
    r = ref.astype(np.float64).ravel()
    diff = np.abs(g - r)
    nz = np.abs(r) > 0
    unfloored = float(np.max(diff[nz] / np.abs(r[nz]))) if nz.any() else 0.0
    normwise = float(np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300))
    return unfloored, normwise


@pytest.mark.parametrize("name", FULL)
@pytest.mark.parametrize("kind", ["excluded", "included"])
def test_full_size_workload(name, kind):
    import torch
    import paper_2106_00124_gb300 as ex
    dev, vals, spec = synth.workload_input(name)
    k, op, dtype = spec["k"], spec["op"], spec["dtype"]
    x = to_device(dev, dtype)
    out = (ex.excluded if kind == "excluded" else ex.included)(x, k, op)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = oracle_sum(kind, vals, k, op)
    worst = check(got, ref, dtype, op, "%s %s" % (kind, name))
    if dtype in ("f32", "bf16") and op == "add":
        unfloored, normwise = _errors(got, ref)
        print("\n%s %s: floored-relative %.3g, unfloored max relative %.3g, normwise %.3g"
              % (kind, name, worst, unfloored, normwise))
        assert normwise <= 1e-6


def test_server_stress_scheduled_arrivals():
    """400 mixed requests with scheduled arrivals on 4 slots and a budget that
    holds only a few at a time: all complete, each equal to its lone result,
    and the result of every distinct shape equal to the oracle's."""
    import torch
    import paper_2106_00124_gb300 as ex
    shapes = synth.batched_shapes(12, seed=21, side_lo=16, side_hi=96)
    inputs = [synth.make_input(s_, "f32", 30 + i) for i, (s_, _) in enumerate(shapes)]
    xs = [to_device(dev, "f32") for dev, _ in inputs]
    outs = [torch.full_like(x, float("nan")) for x in xs]
    alone = []
    for x, (s_, k) in zip(xs, shapes):
        r = ex.excluded(x, k, "add")
        torch.cuda.synchronize()
        alone.append(r)
    need = max(ex.exsum_workspace_bytes(len(s_), s_, k, ex.OP_ADD, ex.F32, 1)[0] for s_, k in shapes)
    srv = ex.exsum_server_create(3 * need, 4)
    assert srv
    rng = np.random.default_rng(5)
    t0 = ex.exsum_server_now_ns() + 20_000_000
    arrivals = t0 + np.cumsum(rng.exponential(20_000, size=400)).astype(np.int64)
    tickets = []
    served = set()
    try:
        for i in range(400):
            j = i if i < len(shapes) else int(rng.integers(0, len(shapes)))
            served.add(j)
            s_, k = shapes[j]
            dsc = ex.make_desc(xs[j].data_ptr(), outs[j].data_ptr(), s_, k, ex.OP_ADD, ex.F32)
            rc, t = ex.exsum_server_submit_at(srv, dsc, 0, int(arrivals[i]))
            assert rc == ex.EXSUM_OK
            tickets.append(t)
        for t in tickets:
            assert ex.exsum_server_wait(srv, t, 30 * 10 ** 9) == ex.EXSUM_OK
        for t in tickets:
            rc, sub, st, done = ex.exsum_server_ticket_times(srv, t)
            assert rc == 0 and sub <= st <= done
    finally:
        ex.exsum_server_destroy(srv)
    torch.cuda.synchronize()
    for j in served:
        assert torch.equal(outs[j], alone[j])
        s_, k = shapes[j]
        check(outs[j].cpu().numpy(), oracle_sum("excluded", inputs[j][1], k, "add"), "f32", "add",
              "served shape %d" % j)
    assert len(served) == len(shapes)
