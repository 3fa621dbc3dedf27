"""Host checks of the level planner: the work lists that the level-batched
schedule builds for a batch of excluded sums (the passes of the row schedule,
Sec. 4, grouped by level).

A host program (level_plan_check.cu, compiled here with nvcc, launching
nothing) plans batches with fake device addresses and lists every work item.
For each item this file knows which ranges the pass body reads and writes
(its view of the source, the row or plane totals, the destination); the
tests check, for batches of edge shapes, random uneven batches and every
tuning knob, that

* every range lies inside its tensor's input or output, or the workspace,
  and the workspace the planner sized is the one it carves;
* ranges written by different passes never overlap, and no pass writes an
  input tensor;
* every workspace byte a pass reads was written by a pass of a level that
  runs before it (levels 1 | 1b, 2, 2h | 3 | 4, the order of the launches);
* every tensor's output is written whole, by exactly one pass;
* the pieces of a pass cover its virtual grid once, in order;
* the vector and bulk-copy bodies get 16-byte aligned rows.

A last test plants mistakes in a plan (in Python) and checks that the
checker reports each.
"""

import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2106_00124_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

FIELDS = ("lv", "kind", "vbase", "count", "vgrid", "src", "dst", "t", "r", "O", "I", "n", "k", "Lc",
          "nchunks", "L", "n2", "k2", "k3", "TR", "GO", "ntile", "ntiles", "lpr")


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("lvplan") / "level_plan_check")
    # PTX only: the program launches no kernel, so no machine code is needed
    cmd = [nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=compute_103a",
           "-I", os.path.join(ROOT, "include"), "-o", exe, os.path.join(HERE, "level_plan_check.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    return exe


def plan(exe, spec, lc=0, interleave=1, tpv=2, tall=0, skew=0):
    """Runs the planner on [(shape, k)]; returns a dict with the tensors,
    the workspace and the items."""
    lines = [str(len(spec))]
    for sh, k in spec:
        lines.append(" ".join(str(v) for v in (len(sh),) + tuple(sh) + tuple(k)))
    env = dict(os.environ, LC=str(lc), IL=str(interleave), TPV=str(tpv), TALL=str(tall), SKEW=str(skew))
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    out = dict(kinds={}, levels={}, tensors=[], items=[])
    for ln in r.stdout.splitlines():
        f = ln.split()
        if f[0] == "S":
            out["F"], out["C"] = int(f[1]), int(f[2])
        elif f[0] == "K":
            out["kinds"][int(f[2])] = f[1]
        elif f[0] == "L":
            out["levels"][int(f[2])] = f[1]
        elif f[0] == "T":
            t, a_in, a_out, N, acc = (int(v) for v in f[1:])
            out["tensors"].append(dict(id=t, inp=a_in, out=a_out, N=N, accepted=bool(acc),
                                       shape=tuple(spec[t][0]), k=tuple(spec[t][1])))
        elif f[0] == "W":
            out["base"], out["sized"], out["carved"] = (int(v) for v in f[1:])
        elif f[0] == "I":
            w = dict(zip(FIELDS, (int(v) for v in f[1:])))
            w["kind"] = out["kinds"][w["kind"]]
            w["level"] = out["levels"][w["lv"]]
            out["items"].append(w)
    return out


# the launch order of the levels: a level runs after every level of the
# groups named here (level 1b runs beside levels 2 and 3; 2h beside 2)
GROUP = {"LV1": "A", "LV1_C1": "A", "LV1B": "B1", "LV1B_C1": "B1", "LV2": "P", "LV2H": "H",
         "LV2H_C1": "H", "LV3": "E", "LV4A": "F", "LV4A_ODD": "F", "LV4B": "F", "LV4B_C1": "F",
         "LV4B_C2": "F"}
BEFORE = {"A": set(), "B1": {"A"}, "H": {"A"}, "P": {"A"}, "E": {"A", "H", "P"},
          "F": {"A", "B1", "H", "P", "E"}}


def accesses(w, p, outs):
    """[(mode, start, end)] of the bytes the item's body reads ("r") or
    writes ("w")."""
    F, C = p["F"], p["C"]
    kd = w["kind"]
    acc = []
    if kd.startswith("S"):
        e = w["O"] * w["n"] * w["I"]
        acc += [("r", w["src"], e * F), ("w", w["dst"], e * F)]
    elif kd.startswith("H1"):
        e = w["O"] * w["n"] * w["I"]
        acc += [("r", w["src"], e * (C if kd.startswith("H1C") else F)), ("w", w["dst"], e * C)]
    elif kd.startswith("RT"):
        acc += [("r", w["src"], w["O"] * w["L"] * F), ("w", w["r"], w["O"] * C)]
    elif kd.startswith("PT"):
        acc += [("r", w["src"], w["vgrid"] * w["n2"] * (F if kd == "PT_IN" else C)),
                ("w", w["r"], w["vgrid"] * C)]
    elif kd.startswith("E2"):
        e = w["n"] * w["n2"]
        acc += [("r", w["src"], e * (F if kd == "E2_IN" else C)), ("r", w["t"], w["n"] * C),
                ("w", w["dst"], e * (C if kd == "E2_CAR" else F))]
    elif kd.startswith("BK") or kd.startswith("RX"):
        t = outs.get(w["dst"])
        if t is None:
            return None
        N = t["N"]
        acc += [("r", w["src"], N * F), ("r", w["t"], N // w["L"] * C), ("w", w["dst"], N * F)]
    else:
        raise AssertionError("unknown kind %s" % kd)
    return [(m, a, a + b) for m, a, b in acc]


def _merge(iv):
    out = []
    for a, b in sorted(iv):
        if out and a <= out[-1][1]:
            out[-1][1] = max(out[-1][1], b)
        else:
            out.append([a, b])
    return out


def _covered(merged, starts, a, b):
    import bisect
    i = bisect.bisect_right(starts, a) - 1
    return i >= 0 and merged[i][0] <= a and b <= merged[i][1]


def violations(p):
    """Every broken rule of the plan, as text (empty: the plan is sound)."""
    import bisect
    bad = []
    F = p["F"]
    if p["sized"] != p["carved"]:
        bad.append("workspace sized %d bytes, carved %d" % (p["sized"], p["carved"]))
    ws = (p["base"], p["base"] + p["carved"])
    acc_t = [t for t in p["tensors"] if t["accepted"]]
    outs = {t["out"]: t for t in acc_t}
    regions = sorted([(t["inp"], t["inp"] + t["N"] * F, "in", t["id"]) for t in acc_t] +
                     [(t["out"], t["out"] + t["N"] * F, "out", t["id"]) for t in acc_t] +
                     [(ws[0], ws[1], "ws", -1)])
    rstarts = [r[0] for r in regions]

    def region(a, b):
        i = bisect.bisect_right(rstarts, a) - 1
        if i >= 0 and regions[i][0] <= a and b <= regions[i][1]:
            return regions[i]
        return None

    writes = {}            # (start, end, level, kind, src) -> item (pieces of one pass share one)
    reads = []
    pieces = {}
    for w in p["items"]:
        if w["count"] <= 0 or w["vbase"] < 0 or w["vbase"] + w["count"] > w["vgrid"]:
            bad.append("%s %s: pieces [%d, +%d) of a grid of %d" % (w["level"], w["kind"], w["vbase"],
                                                                   w["count"], w["vgrid"]))
        key = (w["level"], w["kind"], w["src"], w["dst"], w["r"], w["O"], w["n"], w["I"], w["Lc"], w["vgrid"])
        pieces.setdefault(key, []).append((w["vbase"], w["count"]))
        if w["kind"].startswith(("S4", "BK")):
            if w["src"] % 16 or w["dst"] % 16:
                bad.append("%s %s: rows not 16-byte aligned" % (w["level"], w["kind"]))
        if w["kind"].startswith("S4") and w["I"] % 4:
            bad.append("%s S4: I = %d not a multiple of 4" % (w["level"], w["I"]))
        if w["kind"].startswith("RX") and w["dst"] in outs and \
                w["O"] * w["n2"] * w["L"] != outs[w["dst"]]["N"]:
            bad.append("%s %s: O n2 L = %d x %d x %d, tensor of %d" % (w["level"], w["kind"], w["O"], w["n2"],
                                                                      w["L"], outs[w["dst"]]["N"]))
        acc = accesses(w, p, outs)
        if acc is None:
            bad.append("%s %s: final pass into no accepted output" % (w["level"], w["kind"]))
            continue
        for m, a, b in acc:
            rg = region(a, b)
            if rg is None:
                bad.append("%s %s: %s [%#x, %#x) outside every tensor and the workspace"
                           % (w["level"], w["kind"], m, a, b))
                continue
            if m == "w":
                if rg[2] == "in":
                    bad.append("%s %s: writes input %d" % (w["level"], w["kind"], rg[3]))
                writes.setdefault((a, b, w["level"], w["kind"], w["src"]), w)
            else:
                if rg[2] == "out":
                    bad.append("%s %s: reads output %d" % (w["level"], w["kind"], rg[3]))
                if rg[2] == "ws":
                    reads.append((GROUP[w["level"]], a, b, w))
    # pieces of a pass: [0, vgrid) once, in order
    for key, ps in pieces.items():
        ps.sort()
        pos = 0
        for v0, c in ps:
            if v0 != pos:
                bad.append("%s %s: pieces leave a gap or overlap at virtual block %d" % (key[0], key[1], pos))
                break
            pos += c
        else:
            if pos != key[-1]:
                bad.append("%s %s: pieces cover %d of %d virtual blocks" % (key[0], key[1], pos, key[-1]))
    # writes of different passes are disjoint
    wl = sorted(writes)
    for x, y in zip(wl, wl[1:]):
        if y[0] < x[1]:
            bad.append("%s %s and %s %s write overlapping bytes [%#x, %#x)" % (x[2], x[3], y[2], y[3], y[0],
                                                                               min(x[1], y[1])))
    # every workspace read was written by a level that runs before the reader
    by_group = {}
    for a, b, lv, kd, _ in writes:
        by_group.setdefault(GROUP[lv], []).append((a, b))
    merged = {}
    for g, before in BEFORE.items():
        m = _merge([iv for h in before for iv in by_group.get(h, [])])
        merged[g] = (m, [iv[0] for iv in m])
    for g, a, b, w in reads:
        m, st = merged[g]
        if not _covered(m, st, a, b):
            bad.append("%s %s reads [%#x, %#x) before it is written" % (w["level"], w["kind"], a, b))
    # every accepted output written whole, by one pass
    for t in acc_t:
        ws_t = [(a, b) for a, b, lv, kd, _ in writes if t["out"] <= a < t["out"] + t["N"] * F]
        if ws_t != [(t["out"], t["out"] + t["N"] * F)]:
            bad.append("tensor %d %s: output written by %d passes, ranges %s"
                       % (t["id"], t["shape"], len(ws_t), ws_t[:3]))
    return bad


# shapes that reach every pass body and level: bulk-staged final passes
# (rows of 128 .. 1024, a multiple of 4 or not), k_rowx (short rows), the
# second strided pass (a final pass that does not take the window along n_2),
# boxes of 1, both register classes of the strided passes, the small d = 2
# path with and without the window sums H1, and shapes the level set refuses
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
    ((300, 513), (32, 7)),
    ((3, 70, 129), (2, 1, 5)),
    ((2, 100, 131), (2, 4, 8)),
    ((4, 33, 130), (3, 8, 130)),
    ((2, 90, 255), (2, 16, 3)),
    ((2, 40, 997), (2, 32, 500)),
    ((200, 3, 1024), (17, 3, 9)),
    ((40, 1024, 64), (32, 32, 32)),
    ((17, 19, 23), (3, 4, 5)),
    ((8, 9, 130), (2, 9, 3)),
    # refused: rows under 16, d = 1 and 4, n_2 over 1024, boxes over 32 along x1
    ((5, 6, 7), (2, 2, 2)),
    ((4096,), (7,)),
    ((5, 6, 7, 8), (2, 3, 4, 5)),
    ((4, 2000, 64), (2, 2, 2)),
    ((100, 10, 64), (40, 2, 2)),
]

TUNINGS = [dict(lc=lc, interleave=il, tpv=tpv, tall=tall)
           for lc in (0, 16, 128) for il in (0, 1) for tpv in (1, 2, 4) for tall in (0, 1)]


def _sound(p):
    bad = violations(p)
    assert not bad, "\n".join(bad[:20])


@pytest.mark.parametrize("skew", [0, 4, 8])
def test_edge_shapes_every_tuning(planner, skew):
    seen_levels, seen_kinds = set(), set()
    for tune in TUNINGS:
        p = plan(planner, EDGE, skew=skew, **tune)
        _sound(p)
        seen_levels |= {w["level"] for w in p["items"]}
        seen_kinds |= {w["kind"] for w in p["items"]}
        acc = {t["shape"] for t in p["tensors"] if t["accepted"]}
        assert (5, 6, 7) not in acc and (4096,) not in acc and (5, 6, 7, 8) not in acc
        assert (4, 2000, 64) not in acc and (100, 10, 64) not in acc
        assert (4, 16, 128) in acc and (64, 1024) in acc and (2, 40, 997) in acc
    # the edge batch reaches every level (16-byte aligned rows for the bulk
    # copies and the vector strided passes)
    if skew == 0:
        assert seen_levels == set(GROUP), sorted(set(GROUP) - seen_levels)
        for kd in ("S4_K4", "S4_K8", "S1_K4", "S1_K32", "RT_4", "RT_32", "PT_IN", "PT_CAR", "E2_IN",
                   "E2_CAR", "E2_CO", "BK_K1", "BK_K8", "BK_K32", "H1C_K32", "H1I_K32"):
            assert kd in seen_kinds, kd
    else:
        # outputs off the 16-byte boundary take no bulk copies (the vector
        # strided passes only between workspace buffers, checked above)
        assert not any(k.startswith("BK") for k in seen_kinds)


@pytest.mark.parametrize("count,seed,kw", [
    (64, 5, dict(side_lo=2, side_hi=100, k_lo=1, k_hi=32, cap=1 << 16)),
    (256, 9, dict(side_lo=16, side_hi=64, k_lo=1, k_hi=32, cap=1 << 16)),
    (512, 11, dict()),
])
def test_uneven_batches(planner, count, seed, kw):
    spec = synth.batched_shapes(count, seed=seed, **kw)
    for tune in (dict(), dict(interleave=0), dict(lc=16, tall=1, tpv=4)):
        p = plan(planner, spec, **tune)
        _sound(p)
        assert sum(t["accepted"] for t in p["tensors"]) >= count // 2


def test_checker_reports_planted_mistakes(planner):
    """Each mistake is planted in a copy of a sound plan; the checker names it."""
    import copy
    p = plan(planner, EDGE[:21])
    assert not violations(p)

    def planted(pred, change):
        q = copy.deepcopy(p)
        hits = [w for w in q["items"] if pred(w)]
        assert hits
        change(hits[0], q)
        return violations(q)

    F = p["F"]
    # a row-totals piece shifted by one row: overlaps its neighbour
    assert planted(lambda w: w["kind"].startswith("RT") and w["vgrid"] > 0,
                   lambda w, q: w.update(r=w["r"] + p["C"]))
    # a strided pass writing its input
    assert planted(lambda w: w["kind"].startswith("S1"), lambda w, q: w.update(dst=w["src"]))
    # the lower problem of a d = 3 tensor planned before its window sums
    assert planted(lambda w: w["kind"] == "E2_CAR" and w["src"] != w["t"],
                   lambda w, q: w.update(level="LV2H"))
    # a final pass reading a buffer of the level that runs beside it
    assert planted(lambda w: w["level"] == "LV1B", lambda w, q: w.update(level="LV4B"))
    # a missing piece of an interleaved strided pass
    assert planted(lambda w: w["kind"].startswith("S") and w["count"] < w["vgrid"],
                   lambda w, q: q["items"].remove(w))
    # a null source (a pass whose input was never planned)
    assert planted(lambda w: w["kind"].startswith("S"), lambda w, q: w.update(src=0))
    # one element too many in a d = 2 lower problem
    assert planted(lambda w: w["kind"] in ("E2_IN", "E2_CO"), lambda w, q: w.update(n2=w["n2"] + 1))
    # the workspace one byte short
    assert planted(lambda w: True, lambda w, q: q.update(carved=q["carved"] - 1))
    # a bulk-staged final pass on rows off the 16-byte boundary
    assert planted(lambda w: w["kind"].startswith("BK"), lambda w, q: w.update(src=w["src"] + F))
