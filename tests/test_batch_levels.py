"""Level-scheduled batches: one launch per pass level (and register class)
of the row schedule (Sec. 4) for every tensor of a batch, each launch taking
(tensor, pass, tile) items from a device work list.

GPU: every tensor of uneven batches is compared with the oracle, element by
element (floored 1e-5 relative bound for fp32 +, bit-exact for the integer
and max tensors that run on the lane beside the level set), over replays of
the same plan; the plan stays within a handful of kernels whatever the
batch size, and the autotuner's choice is written to the tuning cache.
"""

import os

import numpy as np
import pytest

import paper_2106_00124_gb300 as ex
from helpers import check, oracle_sum, seeded, to_device
from paper_2106_00124_gb300 import synth

pytestmark = pytest.mark.gpu

# Shapes that reach every body of the level kernels: the bulk-staged final
# pass (rows of 128 .. 1024 elements, a multiple of 4), k_rowx (short or odd
# rows), a final pass that does not take the window along n_2 (a second
# strided pass: 32-row window over 512-element rows), boxes of 1 (no
# strided pass), 4-wide strided passes and the small d = 2 path.
EDGE = [
    ((4, 16, 128), (3, 5, 7)),
    ((3, 20, 256), (2, 8, 4)),
    ((2, 64, 512), (2, 32, 5)),
    ((5, 7, 16), (1, 1, 1)),
    ((9, 13, 17), (9, 13, 17)),
    ((6, 40, 33), (4, 1, 32)),
    ((33, 24, 20), (31, 16, 3)),
    ((1, 1, 16), (1, 1, 16)),
    ((64, 1024), (1, 1)),
    ((1, 16), (1, 16)),
    ((128, 77), (20, 31)),
    # rows whose length is not a multiple of 4, bulk-staged
    ((3, 70, 129), (2, 1, 5)),
    ((2, 100, 131), (2, 4, 8)),
    ((4, 33, 130), (3, 8, 130)),
    ((2, 90, 255), (2, 16, 3)),
    ((2, 40, 997), (2, 32, 500)),
]


def _small_uneven(count, seed):
    spec = synth.batched_shapes(count, seed=seed, side_lo=2, side_hi=100, k_lo=1, k_hi=32, cap=1 << 16)
    # sides below 16 along the last dimension leave the row schedule; keep them
    # in the batch (they run on the lane beside the level set)
    return spec


def _run(spec, lanes, seed0, replays=2, extra=()):
    import torch
    cases = [(sh, k, "f32", "add") for sh, k in spec] + list(extra)
    xs, outs, vals = [], [], []
    for i, (sh, k, dt, op) in enumerate(cases):
        dev, v = seeded(sh, dt, seed0 + i, op)
        xs.append(to_device(dev, dt))
        vals.append(v)
        out_dtype = {"i32": torch.int32, "i64": torch.int64}.get(dt, torch.float32)
        outs.append(torch.full(sh, 7, dtype=out_dtype, device="cuda"))
    descs = [ex.make_desc(x.data_ptr(), o.data_ptr(), c[0], c[1], ex.OPS[c[3]], ex.DTYPES[c[2]])
             for x, o, c in zip(xs, outs, cases)]
    s = torch.cuda.current_stream().cuda_stream
    rc, plan = ex.exsum_batch_create(descs, lanes=lanes, stream=s)
    assert rc == ex.EXSUM_OK, ex.strerror(rc)
    try:
        sched = ex.exsum_batch_schedule(plan)
        info = ex.exsum_batch_info(plan)
        refs = [oracle_sum("excluded", v, c[1], c[3]) for v, c in zip(vals, cases)]
        for rep in range(replays):
            for o in outs:
                o.fill_(7)
            assert ex.exsum_batch_launch(plan, s) == ex.EXSUM_OK
            torch.cuda.synchronize()
            for i, (o, c) in enumerate(zip(outs, cases)):
                check(o.cpu().numpy(), refs[i], c[2], c[3], "tensor %d %s, replay %d" % (i, c[:2], rep))
    finally:
        ex.exsum_batch_destroy(plan)
    return sched, info


def test_levels_64_small_uneven_tensors_match_oracle():
    spec = _small_uneven(64, seed=5)
    assert all(int(np.prod(sh)) <= 1 << 16 for sh, _ in spec)
    sched, info = _run(spec, ex.BATCH_LEVELS, 1000)
    rc, mode, nlevel = sched[:3]
    assert rc == 0 and mode == 1
    # every d = 2 tensor and every d = 3 tensor with rows of 16 .. 1024 joins
    # at most thirteen level kernels and a memset, plus what the other tensors take alone
    lane = [(sh, k) for sh, k in spec if not (len(sh) == 2 or sh[-1] >= 16)]
    assert nlevel == len(spec) - len(lane)
    alone = 0
    for sh, k in lane:
        import torch
        x = torch.zeros(sh, dtype=torch.float32, device="cuda")
        n0 = ex.exsum_launch_count()
        ex.excluded(x, k, "add")
        alone += ex.exsum_launch_count() - n0
    assert info[4] <= 14 + alone


def test_levels_edge_shapes_and_a_mixed_lane():
    extra = [((7, 300), (7, 31), "i64", "max"),
             ((5, 6, 7, 8), (2, 3, 4, 5), "i32", "add"),
             ((2000,), (100,), "bf16", "add"),
             ((40, 33, 21), (8, 5, 3), "i32", "max")]
    sched, info = _run(EDGE, ex.BATCH_LEVELS, 2000, replays=3, extra=extra)
    assert sched[1] == 1 and sched[2] == len(EDGE)


def test_levels_batch_of_256_stays_within_a_few_kernels():
    spec = synth.batched_shapes(256, seed=9, side_lo=16, side_hi=64, k_lo=1, k_hi=32, cap=1 << 16)
    sched, info = _run(spec, ex.BATCH_LEVELS, 3000, replays=1)
    assert sched[1] == 1 and sched[2] == len(spec)
    assert info[4] <= 13


def test_autotune_caches_its_choice(tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("EXSUM_TUNE_CACHE", str(path))
    spec = [((17, 19, 23), (3, 4, 5)), ((40, 41), (6, 7)), ((8, 9, 130), (2, 9, 3))]
    s1, _ = _run(spec, 0, 4000, replays=1)
    lines = [ln.split() for ln in path.read_text().splitlines() if ln.strip()]
    assert len(lines) == 1 and len(lines[0]) == 9
    key, fields = lines[0][0], [int(v) for v in lines[0][1:]]
    assert fields[0] == s1[1]                         # mode
    if fields[0] == 1:
        assert fields[3:8] == list(s1[3:8])           # lc, interleave, tiles per block, tall, persist
    # the same signature again: the remembered schedule, no second entry
    s2, _ = _run(spec, 0, 4000, replays=1)
    assert s2[1:] == s1[1:]
    assert len([ln for ln in path.read_text().splitlines() if ln.strip()]) == 1
