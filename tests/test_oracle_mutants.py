"""Planted-mistake checks for the oracle's pins (CPU only).

Each case copies the oracle's C source, plants one plausible mistake (an
off-by-one, a dropped term, a wrong offset or bound, a wrong operand), builds
the copy into a temporary library and runs a battery of independent pins
against it.  Every mutant must fail at least one pin; the unmodified source
must pass them all.  Nothing here touches the oracle used by other tests.
"""

import ctypes
import itertools
import os
import subprocess

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "exsum_oracle.c")

MUTANTS = {
    "block_start_test_off_by_one": ("if (x % k != 0) {", "if (x % k != 1) {"),
    "padded_next_block_bound": ("else if (next_block <= len - 1)", "else if (next_block < len - 1)"),
    "prefix_dropped_term": ("Ap[x] = combine(mon, Ap[x - 1], r[x * s]);", "Ap[x] = r[x * s];"),
    "contribution_lower_bound": ("if (t >= 0 && t < n[dim]) {", "if (t > 0 && t < n[dim]) {"),
    "suffix_offset": ("add_contribution(B, Aw, d, n, st, i, k[i], mon);",
                      "add_contribution(B, Aw, d, n, st, i, k[i] - 1, mon);"),
    "prefix_offset": ("add_contribution(B, Aw, d, n, st, i, -1, mon);",
                      "add_contribution(B, Aw, d, n, st, i, 0, mon);"),
    "bdbs_dims_from_i": ("for (j = i + 1; j < d; j++)                  /* BDBS-Along-Dim",
                         "for (j = i; j < d; j++)                  /* BDBS-Along-Dim"),
    "skip_saving_prefix": ("copy_view(Apre, Aw, d, n, st, i);            /* save prefix",
                           "/* */            /* save prefix"),
    "box_clip_short": ("hi[i] = x[i] + k[i] < n[i] ? x[i] + k[i] : n[i];",
                       "hi[i] = x[i] + k[i] - 1 < n[i] ? x[i] + k[i] - 1 : n[i];"),
    "box_membership_bound": ("if (y[i] < x[i] || y[i] >= x[i] + k[i]) return 0;",
                             "if (y[i] < x[i] || y[i] > x[i] + k[i]) return 0;"),
    "max_becomes_min": ("case ORC_MAX_I64: r.i = a.i > b.i ? a.i : b.i; break;",
                        "case ORC_MAX_I64: r.i = a.i < b.i ? a.i : b.i; break;"),
    "corner_rule_own_dim": ("return (mask >> ((dim + 1) % 3)) & 1u;",
                            "return (mask >> dim) & 1u;"),
    "suffix_step_uses_prefix_input": ("copy_view(Aw, Asuf, d, n, st, i);",
                                      "copy_view(Aw, Apre, d, n, st, i);"),
}


def _build(tmp_path, name, source):
    c = tmp_path / (name + ".c")
    so = tmp_path / ("lib" + name + ".so")
    c.write_text(source)
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", "-o", str(so), str(c),
                           "-lm"])
    lib = ctypes.CDLL(str(so))
    i64p = ctypes.POINTER(ctypes.c_int64)
    for fn_name in ("orc_included_brute", "orc_excluded_brute", "orc_bdbs", "orc_box_complement",
                    "orc_corners"):
        fn = getattr(lib, fn_name)
        fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, i64p, i64p, ctypes.c_int]
        fn.restype = ctypes.c_int
    return lib


def _run(lib, fn_name, a, k, mon):
    a = np.ascontiguousarray(a, dtype=np.int64)
    out = np.empty_like(a)
    arr = lambda seq: (ctypes.c_int64 * len(seq))(*[int(v) for v in seq])
    rc = getattr(lib, fn_name)(a.ctypes.data, out.ctypes.data, a.ndim, arr(a.shape), arr(k), mon)
    assert rc == 0
    return out


def _np_def(a, k, op, excluded):
    out = np.empty(a.shape, dtype=np.int64)
    for x in itertools.product(*[range(n) for n in a.shape]):
        box = tuple(slice(xi, min(xi + ki, ni)) for xi, ki, ni in zip(x, k, a.shape))
        if excluded:
            mask = np.ones(a.shape, dtype=bool)
            mask[box] = False
            vals = a[mask]
        else:
            vals = a[box].ravel()
        if op == "add":
            out[x] = vals.sum() if vals.size else 0
        else:
            out[x] = vals.max() if vals.size else np.iinfo(np.int64).min
    return out


def _pins_pass(lib):
    """True when every pin holds for the library."""
    rng = np.random.default_rng(2024)
    for shape in [(7,), (5, 6), (4, 3, 5), (3, 2, 3, 2)]:
        a = rng.integers(-100, 100, size=shape).astype(np.int64)
        for op, mon in (("add", 0), ("max", 1)):
            for _ in range(3):
                k = [int(rng.integers(1, n + 1)) for n in shape]
                inc, exc = _np_def(a, k, op, False), _np_def(a, k, op, True)
                if not np.array_equal(_run(lib, "orc_included_brute", a, k, mon), inc):
                    return False
                if not np.array_equal(_run(lib, "orc_excluded_brute", a, k, mon), exc):
                    return False
                if not np.array_equal(_run(lib, "orc_bdbs", a, k, mon), inc):
                    return False
                if not np.array_equal(_run(lib, "orc_box_complement", a, k, mon), exc):
                    return False
                if len(shape) in (2, 3) and not np.array_equal(
                        _run(lib, "orc_corners", a, k, mon), exc):
                    return False
    return True


def test_unmodified_oracle_passes_battery(tmp_path):
    lib = _build(tmp_path, "orig", open(SRC).read())
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not unique: %s" % name
    lib = _build(tmp_path, name, src.replace(old, new))
    assert not _pins_pass(lib), "pins missed planted mistake %s" % name
