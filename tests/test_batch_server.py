"""Batched (one graph launch over uneven tensors) and served (continuous
batching) excluded sums.

CPU: argument checks that return before any device work.
GPU: every tensor of a batch and every request of a served mix (device and
host pointers, int64 max among them) is checked against the oracle, element
by element: bit-exact for integers and max, the floored 1e-5 relative bound
for fp32/bf16 +.  Beside that, each served result and each tensor of a
batch planned on lanes gives the same bits as the same tensor computed alone
by exsum_excluded (the kernels and their reduction order do not depend on
what else runs), so that comparison is exact equality.  A level-scheduled
batch (one launch per pass level for all its tensors) may pick
other tile heights than a lone call, so its tensors are held to the oracle
bound only.
"""

import numpy as np
import pytest

import paper_2106_00124_gb300 as ex
from helpers import check, oracle_sum, seeded, to_device


def test_server_rejects_bad_arguments_without_gpu():
    assert not ex.exsum_server_create(0, 4)
    assert not ex.exsum_server_create(1 << 20, 0)
    dsc = ex.make_desc(16, 32, [4, 4], [2, 2], ex.OP_ADD, ex.F32)
    assert ex.exsum_server_submit(None, dsc)[0] == ex.EXSUM_EINVAL
    assert ex.exsum_server_wait(None, 1, 0) == ex.EXSUM_EINVAL


def test_batch_rejects_bad_descriptors_without_gpu():
    bad = ex.make_desc(16, 32, [4, 4], [5, 2], ex.OP_ADD, ex.F32)       # k > n
    assert ex.exsum_batch_create([bad], lanes=1)[0] == ex.EXSUM_EINVAL
    nul = ex.make_desc(0, 32, [4, 4], [2, 2], ex.OP_ADD, ex.F32)        # null input
    assert ex.exsum_batch_create([nul], lanes=1)[0] == ex.EXSUM_EINVAL
    assert ex.exsum_batch_create([], lanes=1)[0] == ex.EXSUM_EINVAL


MIX = [
    ((40, 33, 21), (8, 5, 3), "f32", "add"),
    ((100, 64), (16, 2), "f32", "add"),
    ((7, 300), (7, 31), "i64", "max"),
    ((2000,), (100,), "bf16", "add"),
    ((33, 34, 35), (32, 2, 9), "i32", "add"),
    ((64, 64, 64), (8, 8, 8), "f32", "add"),
    ((5, 6, 7, 8), (2, 3, 4, 5), "i32", "max"),
    ((129, 131), (30, 17), "bf16", "max"),
    ((300, 257), (3, 32), "f32", "add"),
    ((50, 40, 30), (10, 10, 10), "i64", "add"),
]


def _tensors(cases, seed0=0):
    import torch
    xs, outs = [], []
    for i, (shape, k, dtype, op) in enumerate(cases):
        dev, _ = seeded(shape, dtype, seed0 + i, op)
        x = to_device(dev, dtype)
        out_dtype = {"i32": torch.int32, "i64": torch.int64}.get(dtype, torch.float32)
        xs.append(x)
        outs.append(torch.full(shape, 3, dtype=out_dtype, device="cuda"))
    return xs, outs


_ORACLE = {}


def _oracle(case, seed):
    """Oracle excluded sum of the seeded input of `case` (cached per seed)."""
    shape, k, dtype, op = case
    key = (tuple(shape), tuple(k), dtype, op, seed)
    if key not in _ORACLE:
        _, vals = seeded(shape, dtype, seed, op)
        _ORACLE[key] = oracle_sum("excluded", vals, k, op)
    return _ORACLE[key]


def _alone(x, k, op):
    import torch
    r = ex.excluded(x, k, op)
    torch.cuda.synchronize()
    return r.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("lanes", [1, 3, 0, ex.BATCH_LEVELS])
def test_batch_matches_single_calls(lanes):
    import torch
    xs, outs = _tensors(MIX)
    descs = [ex.make_desc(x.data_ptr(), o.data_ptr(), c[0], c[1], ex.OPS[c[3]], ex.DTYPES[c[2]])
             for x, o, c in zip(xs, outs, MIX)]
    s = torch.cuda.current_stream().cuda_stream
    rc, plan = ex.exsum_batch_create(descs, lanes=lanes, stream=s)
    assert rc == ex.EXSUM_OK, ex.strerror(rc)
    try:
        rc, mode, nlevel = ex.exsum_batch_schedule(plan)[:3]
        assert rc == 0 and mode in (0, 1)
        if lanes == ex.BATCH_LEVELS:
            # the fp32 + tensors of d = 2 and 3 join the level set
            assert mode == 1 and nlevel == 4
        for rep in range(2):
            for o in outs:
                o.fill_(3)
            assert ex.exsum_batch_launch(plan, s) == ex.EXSUM_OK
            torch.cuda.synchronize()
            for i, (x, o, c) in enumerate(zip(xs, outs, MIX)):
                got = o.cpu().numpy()
                check(got, _oracle(c, i), c[2], c[3], "batch tensor %d, replay %d" % (i, rep))
                if mode == 0:
                    assert np.array_equal(got, _alone(x, c[1], c[3])), c
        rc, nl, order, wsb, kern = ex.exsum_batch_info(plan)
        assert rc == 0 and 0 <= nl <= len(MIX)
        assert kern >= (len(MIX) if mode == 0 else len(MIX) - nlevel + 1)
    finally:
        ex.exsum_batch_destroy(plan)


@pytest.mark.gpu
def test_server_mix_equals_alone_device_and_host():
    import torch
    cases = MIX * 4
    xs, outs = _tensors(cases, seed0=100)
    alone = [_alone(x, c[1], c[3]) for x, c in zip(xs, cases)]
    srv = ex.exsum_server_create(512 << 20, 6)
    assert srv
    try:
        tickets = []
        for x, o, (shape, k, dtype, op) in zip(xs, outs, cases):
            dsc = ex.make_desc(x.data_ptr(), o.data_ptr(), shape, k, ex.OPS[op], ex.DTYPES[dtype])
            rc, t = ex.exsum_server_submit(srv, dsc)
            assert rc == ex.EXSUM_OK
            tickets.append(t)
        # host-pointer requests staged through the server's arena
        host_in = [x.cpu().pin_memory() for x in xs[:5]]
        host_out = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs[:5]]
        htickets = []
        for hi, ho, (shape, k, dtype, op) in zip(host_in, host_out, cases[:5]):
            dsc = ex.make_desc(hi.data_ptr(), ho.data_ptr(), shape, k, ex.OPS[op], ex.DTYPES[dtype])
            rc, t = ex.exsum_server_submit(srv, dsc, ex.SERVE_HOST)
            assert rc == ex.EXSUM_OK
            htickets.append(t)
        for t in tickets + htickets:
            assert ex.exsum_server_wait(srv, t, 30 * 10 ** 9) == ex.EXSUM_OK
        torch.cuda.synchronize()
        for i, (o, a, c) in enumerate(zip(outs, alone, cases)):
            got = o.cpu().numpy()
            check(got, _oracle(c, 100 + i), c[2], c[3], "served request %d" % i)
            assert np.array_equal(got, a)
        for i, (ho, a, c) in enumerate(zip(host_out, alone[:5], cases[:5])):
            got = ho.numpy()
            check(got, _oracle(c, 100 + i), c[2], c[3], "served host request %d" % i)
            assert np.array_equal(got, a)
        rc, t_sub, t_start, t_done = ex.exsum_server_ticket_times(srv, tickets[0])
        assert rc == 0 and t_sub <= t_start <= t_done
        assert ex.exsum_server_release(srv, tickets[0]) == ex.EXSUM_OK
        assert ex.exsum_server_wait(srv, tickets[0], 0) == ex.EXSUM_EINVAL
        assert ex.exsum_server_completed(srv) == len(tickets) + len(htickets)
    finally:
        ex.exsum_server_destroy(srv)


@pytest.mark.gpu
def test_server_timeout_budget_and_shutdown():
    import torch
    shape, k = (256, 256, 256), (8, 8, 8)
    x = to_device(seeded(shape, "f32", 77, "add")[0], "f32")
    outs = [torch.empty(shape, device="cuda") for _ in range(3)]
    need, st = ex.exsum_workspace_bytes(3, shape, k, ex.OP_ADD, ex.F32, 1)
    # budget for one request at a time: the other two wait for memory
    srv = ex.exsum_server_create(need + need // 2, 4)
    assert srv
    tickets = []
    for o in outs:
        rc, t = ex.exsum_server_submit(srv, ex.make_desc(x.data_ptr(), o.data_ptr(), shape, k,
                                                         ex.OP_ADD, ex.F32))
        assert rc == ex.EXSUM_OK
        tickets.append(t)
    # the last request cannot have finished: two full excluded sums run before it
    assert ex.exsum_server_wait(srv, tickets[-1], 0) == ex.EXSUM_ETIMEDOUT
    # larger than the whole budget: refused at submission
    big = (512, 512, 512)
    assert ex.exsum_server_submit(srv, ex.make_desc(x.data_ptr(), outs[0].data_ptr(), big, k,
                                                    ex.OP_ADD, ex.F32))[0] == ex.EXSUM_ENOMEM
    for t in tickets:
        assert ex.exsum_server_wait(srv, t, 60 * 10 ** 9) == ex.EXSUM_OK
    ref = ex.excluded(x, k, "add")
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o, ref)
    # shutdown while busy: queued work is finished before the server goes away
    for o in outs:
        o.zero_()
    torch.cuda.synchronize()
    for o in outs:
        rc, t = ex.exsum_server_submit(srv, ex.make_desc(x.data_ptr(), o.data_ptr(), shape, k,
                                                         ex.OP_ADD, ex.F32))
        assert rc == ex.EXSUM_OK
    ex.exsum_server_destroy(srv)
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o, ref)


@pytest.mark.gpu
def test_server_injected_launch_failure_is_reported():
    """A request whose launch fails (injected on the host: nothing reaches
    the GPU) completes with that error, frees its slot and memory, and the
    requests around it still give the oracle's result."""
    import torch
    cases = MIX[:3]
    xs, outs = _tensors(cases, seed0=200)
    srv = ex.exsum_server_create(256 << 20, 2)
    assert srv
    try:
        assert ex.exsum_server_fail_next(srv, 1, ex.EXSUM_ECUDA) == ex.EXSUM_OK
        assert ex.exsum_server_fail_next(srv, -1, ex.EXSUM_ECUDA) == ex.EXSUM_EINVAL
        assert ex.exsum_server_fail_next(srv, 1, 0) == ex.EXSUM_EINVAL
        tickets = []
        for x, o, (shape, k, dtype, op) in zip(xs, outs, cases):
            rc, t = ex.exsum_server_submit(srv, ex.make_desc(x.data_ptr(), o.data_ptr(), shape, k,
                                                             ex.OPS[op], ex.DTYPES[dtype]))
            assert rc == ex.EXSUM_OK
            tickets.append(t)
        # the first admitted request is the first submitted (arrival order)
        assert ex.exsum_server_wait(srv, tickets[0], 30 * 10 ** 9) == ex.EXSUM_ECUDA
        for t in tickets[1:]:
            assert ex.exsum_server_wait(srv, t, 30 * 10 ** 9) == ex.EXSUM_OK
        torch.cuda.synchronize()
        for i in (1, 2):
            check(outs[i].cpu().numpy(), _oracle(cases[i], 200 + i), cases[i][2], cases[i][3],
                  "request %d after an injected failure" % i)
        # the slot and memory of the failed request were released: more work runs
        rc, t = ex.exsum_server_submit(srv, ex.make_desc(xs[0].data_ptr(), outs[0].data_ptr(),
                                                         cases[0][0], cases[0][1],
                                                         ex.OPS[cases[0][3]], ex.DTYPES[cases[0][2]]))
        assert rc == ex.EXSUM_OK
        assert ex.exsum_server_wait(srv, t, 30 * 10 ** 9) == ex.EXSUM_OK
        torch.cuda.synchronize()
        check(outs[0].cpu().numpy(), _oracle(cases[0], 200), cases[0][2], cases[0][3],
              "request after the failed one")
        assert ex.exsum_server_completed(srv) == 4
    finally:
        ex.exsum_server_destroy(srv)


def test_server_fail_next_rejects_null_without_gpu():
    assert ex.exsum_server_fail_next(None, 1, ex.EXSUM_ECUDA) == ex.EXSUM_EINVAL
