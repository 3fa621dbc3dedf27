"""Shared helpers of the GPU parity tests: moving seeded inputs to the device,
calling the library through its binding, and comparing with the oracle."""

import numpy as np

from oracle import oracle as O
from paper_2106_00124_gb300 import synth

# Floating-point + is checked against the fp64 oracle to 1e-5 relative.
# Each element's error is measured against max(|ref|, RMS of the reference
# tensor): an excluded sum of uniform[-1, 1) values can cancel to near zero,
# where a relative bound would be meaningless.
FP_REL_TOL = 1e-5


def to_device(dev_array, dtype):
    import torch
    if dtype == "bf16":
        t = torch.from_numpy(np.ascontiguousarray(dev_array).view(np.int16)).view(torch.bfloat16)
    else:
        t = torch.from_numpy(np.ascontiguousarray(dev_array))
    return t.cuda()


def gpu_sum(kind, x, k, op):
    import torch
    import paper_2106_00124_gb300 as ex
    fn = ex.excluded if kind == "excluded" else ex.included
    out = fn(x, k, op)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def oracle_sum(kind, values, k, op):
    if kind == "excluded":
        return O.box_complement(values, k, op)
    return O.bdbs(values, k, op)


def check(got, ref, dtype, op, what=""):
    """Bit-exact for integers and for max; floored relative tolerance for +."""
    if dtype in ("i32", "i64"):
        want = ref.astype(np.int32 if dtype == "i32" else np.int64)
        if op == "max" and dtype == "i32":
            # the oracle's identity for max is INT64_MIN; the int32 identity is INT32_MIN
            want = np.where(ref == np.iinfo(np.int64).min, np.iinfo(np.int32).min, want).astype(np.int32)
        bad = np.flatnonzero(got.ravel() != want.ravel())
        assert bad.size == 0, "%s: %d mismatches, first at %d: got %r want %r" % (
            what, bad.size, bad[0], got.ravel()[bad[0]], want.ravel()[bad[0]])
        return 0.0
    if op == "max":
        want = ref.astype(np.float32)
        bad = np.flatnonzero(got.ravel() != want.ravel())
        assert bad.size == 0, "%s: %d mismatches, first at %d: got %r want %r" % (
            what, bad.size, bad[0], got.ravel()[bad[0]], want.ravel()[bad[0]])
        return 0.0
    g = got.astype(np.float64).ravel()
    r = ref.astype(np.float64).ravel()
    rms = float(np.sqrt(np.mean(r * r))) if r.size else 0.0
    scale = np.maximum(np.abs(r), rms)
    scale[scale == 0] = 1.0
    rel = np.abs(g - r) / scale
    worst = int(np.argmax(rel)) if rel.size else 0
    assert rel.size == 0 or rel[worst] <= FP_REL_TOL, "%s: error %.3g at %d (got %r want %r)" % (
        what, rel[worst], worst, g[worst], r[worst])
    return float(rel.max()) if rel.size else 0.0


def seeded(shape, dtype, seed, op):
    lo, hi = (-1000, 1000)
    if op == "max" and dtype == "i32":
        lo, hi = 0, (1 << 20) - 1
    return synth.make_input(shape, dtype, seed, lo, hi)
