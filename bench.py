#!/usr/bin/env python
"""Benchmark of the excluded-sum hot path on GB300.

One step = one strong excluded sum (box-complement) of a synthetic tensor
through the C ABI.  The default workload is the 256^3 fp32 tensor with
values uniform in [-1, 1), box k = (8, 8, 8), operator +.  Prints ONE JSON
line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle, timed on host cores

Timing: the step is captured once into a CUDA graph, instantiated by the
library so that the side branches keep their stream priority
(exsum_graph_instantiate); each launch of it is bracketed by CUDA events
on the stream it runs on, and between steps a
256 MiB buffer is written and read back to flush the 129 MB L2 (leaving no
dirty lines), outside the timed spans.
`value` sums the K step spans.  The per-kernel roofline comes from a second
capture of the same step with the library's launch trace on (event-record
nodes around every kernel node), replayed K more times inside the timed
region and read back after each replay.  `e2e` calls the C ABI directly
(no graph) with pinned host input and output buffers, three lanes in flight.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "excluded-sum Gelem/s"
UNIT = "Gelem/s"
DEFAULT_WORKLOAD = "d3_256cube_f32_add_k8"
FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0

BYTES = {"i32": 4, "i64": 8, "f32": 4, "bf16": 2}
OUT_BYTES = {"i32": 4, "i64": 8, "f32": 4, "bf16": 4}


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default=DEFAULT_WORKLOAD)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the compact batched and served figures of the default line")
    p.add_argument("--mode", choices=["single", "batched", "served", "comparators"], default="single",
                   help="single: the default step; batched: 512 uneven tensors as one graph "
                        "launch vs plain per-tensor launches; served: a Poisson request stream "
                        "at three offered loads (p50/p99) vs one-at-a-time plain launches; "
                        "comparators: SAT/SATC, BDBSC and corners against box-complement over d, "
                        "and operator applications per element with a slowed operator")
    p.add_argument("--requests", type=int, default=20000)
    p.add_argument("--profile-once", action="store_true",
                   help="run the workload's excluded sum twice without graphs or timing "
                        "(a small, self-ending command for ncu) and exit; with --mode batched, "
                        "launch the 512-tensor batch's level schedule (tuning from "
                        "EXSUM_LEVEL_TUNE) twice")
    return p.parse_args(argv)


# ---- multi-rank plumbing (also exercised by the CPU tests with gloo) -------------------------

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(
        os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(value, world, device=None):
    """Max of a float over all ranks (identity when world == 1)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(elems_per_rank, world, max_seconds):
    """Units processed by all ranks divided by the slowest rank's time."""
    return elems_per_rank * world / max_seconds


# ---- helpers ---------------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        loaded = [v for v in sm if smax and v >= 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def source_digest():
    """Digest of the sources that define the kernels and their launch plans
    (kernel headers, the pass planner, the per-dtype instantiations); the
    C ABI, batch, server and allocation-free entry points are left out."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2106_00124_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if not (name.endswith(".cuh") or name.startswith("dispatch_")):
            continue
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    sources are unchanged since it was taken; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            tab = json.load(f)
        ent = tab.get(workload, {}).get(kernel)
        if ent and ent.get("source_digest") == source_digest():
            return float(ent["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def pass_bytes(kernel, level, elems, dtype):
    """Algorithmic (compulsory) bytes of one launch: every element the pass
    must read once plus every element it must write once."""
    if level == 0:
        rd = OUT_BYTES[dtype]
        wr = OUT_BYTES[dtype]
    else:
        car = 8 if dtype in ("f32", "bf16") else BYTES[dtype]
        rd = wr = car
    if kernel.startswith("bdbs_along_dim"):
        return elems * (rd + wr)
    if kernel in ("dim1_prefix_suffix_contrib", "row_prefix_suffix_contrib"):
        return elems * (rd + wr)
    if kernel == "segment_reduce":
        return elems * rd
    return elems * rd


# ---- our arm -----------------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    import paper_2106_00124_gb300 as ex
    from paper_2106_00124_gb300 import synth

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev_index = torch.cuda.current_device()
    device = torch.device("cuda", dev_index)

    dev, vals, spec = synth.workload_input(args.workload)
    shape, k, dtype, op = spec["shape"], spec["k"], spec["dtype"], spec["op"]
    N = int(np.prod(shape))
    d = len(shape)
    code, opc = ex.DTYPES[dtype], ex.OPS[op]
    x = (torch.from_numpy(np.ascontiguousarray(dev).view(np.int16)).view(torch.bfloat16)
         if dtype == "bf16" else torch.from_numpy(np.ascontiguousarray(dev))).to(device)
    out_t = {"i32": torch.int32, "i64": torch.int64}.get(dtype, torch.float32)
    out = torch.empty(shape, dtype=out_t, device=device)
    wsb, st = ex.exsum_workspace_bytes(d, shape, k, opc, code, 1)
    assert st == 0
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=device)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=device)
    flush64 = flush.view(torch.int64)

    def flush_l2():
        # Write 256 MiB (evicts the tensors from the 129 MB L2), then read it
        # back, so that the dirty lines of the write are written back here,
        # outside the timed span, and the step starts from a clean cold L2.
        flush.fill_(1)
        flush64.max()

    stream = torch.cuda.current_stream(device)
    sp = stream.cuda_stream

    def step(stream_ptr):
        rc = ex.exsum_excluded_ws(x.data_ptr(), out.data_ptr(), d, shape, k, opc, code,
                                  ws.data_ptr(), wsb, stream_ptr)
        if rc != 0:
            raise ex.ExsumError(rc, "exsum_excluded_ws")

    for _ in range(max(1, min(args.warmup, 3))):
        flush_l2()
        step(sp)
    torch.cuda.synchronize()

    # The step is captured once into a CUDA graph (all of its launches).  A
    # second capture of the same step carries the launch trace: each kernel
    # node is bracketed by event-record nodes, read back after every replay.
    # Capture on a stream that has run the step once outside capture: the
    # library creates the side stream of a caller stream on its first
    # uncaptured call, and forks onto it under capture from then on.
    cap_stream = torch.cuda.Stream(device)
    cap_stream.wait_stream(stream)
    with torch.cuda.stream(cap_stream):
        step(cap_stream.cuda_stream)
    cap_stream.synchronize()

    # The graph is instantiated by the library (exsum_graph_instantiate), which
    # keeps the per-node stream priorities of the side branches.
    def capture(traced):
        g = torch.cuda.CUDAGraph(keep_graph=True)
        ex.exsum_trace_collect(clear=True)
        ex.exsum_trace_enable(traced)
        l0 = ex.exsum_launch_count()
        with torch.cuda.graph(g, stream=cap_stream):
            step(cap_stream.cuda_stream)
        ex.exsum_trace_enable(False)
        return g, ex.exsum_graph_instantiate(g.raw_cuda_graph()), ex.exsum_launch_count() - l0

    graph, gexec, launches_per_step = capture(False)
    tgraph, tgexec, _ = capture(True)
    sh = stream.cuda_stream
    for _ in range(args.warmup):
        flush_l2()
        ex.exsum_graph_launch(gexec, sh)
    torch.cuda.synchronize()

    # ---- timed region -----------------------------------------------------------------------
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = ClockSampler(dev_index)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush_l2()
        evs[i][0].record(stream)
        ex.exsum_graph_launch(gexec, sh)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    # Per-kernel durations: the traced graph over the same number of steps.
    trace = []  # (position of the launch in the step, kernel, level, elements, ms)
    for i in range(args.steps):
        flush_l2()
        ex.exsum_graph_launch(tgexec, sh)
        torch.cuda.synchronize()
        trace.extend((j,) + rec for j, rec in enumerate(ex.exsum_trace_collect(cap=256, clear=False)))
    # L2-warm figure: the same graph back to back with no flush in between
    # (the 256^3 tensors and intermediates partly stay in the 129 MB L2).
    warm_steps = max(3, min(args.steps, 200))
    wa, wb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        ex.exsum_graph_launch(gexec, sh)
    wa.record(stream)
    for _ in range(warm_steps):
        ex.exsum_graph_launch(gexec, sh)
    wb.record(stream)
    torch.cuda.synchronize()
    warm_ms = wa.elapsed_time(wb) / warm_steps
    launches = launches_per_step * args.steps
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ex.exsum_trace_collect(clear=True)
    ex.exsum_graph_exec_destroy(gexec)
    ex.exsum_graph_exec_destroy(tgexec)
    del graph, tgraph
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_s = sum(step_ms) / 1e3
    max_s = max_over_ranks(total_s, world, device)
    value = whole_job_rate(N, world, max_s / args.steps) / 1e9
    ms_per_step = max_s * 1e3 / args.steps

    # ---- per-kernel roofline from the trace ---------------------------------------------------
    peak, peak_kind = measured_peaks()
    groups = {}
    for pos, name, level, elems, ms in trace:
        g = groups.setdefault((pos, name, level, elems), [0, 0.0])
        g[0] += 1
        g[1] += ms
    passes = []
    for (pos, name, level, elems), (cnt, tot) in groups.items():
        mean_ms = tot / cnt
        b = pass_bytes(name, level, elems, dtype)
        passes.append({"pos": pos, "kernel": name, "level": level, "elems": elems, "launches": cnt,
                       "mean_us": round(mean_ms * 1e3, 3), "share": 0.0,
                       "algo_bytes": b, "achieved_gbs": round(b / (mean_ms * 1e-3) / 1e9, 1),
                       "frac": round(b / (mean_ms * 1e-3) / 1e9 / peak, 4)})
    total_kernel_ms = sum(p["mean_us"] * p["launches"] for p in passes) or 1.0
    for p_ in passes:
        p_["share"] = round(p_["mean_us"] * p_["launches"] / total_kernel_ms, 4)
    passes.sort(key=lambda p_: -p_["share"])
    dom = passes[0] if passes else None
    roofline = None
    if dom:
        achieved = dom["achieved_gbs"]
        roofline = {"bound": "hbm", "kernel": dom["kernel"], "level": dom["level"],
                    "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                    "frac": round(achieved / peak, 4),
                    "traffic": profiled_traffic(dom["kernel"], args.workload),
                    "algo_bytes_per_launch": dom["algo_bytes"]}
    one_rw = N * (BYTES[dtype] + OUT_BYTES[dtype])

    # ---- end to end through the public API with host buffers ----------------------------------
    # Every step copies its input from pinned host memory, runs the excluded
    # sum through the C ABI and copies the result back to pinned host memory.
    # Consecutive steps rotate over three lanes (stream + device buffers +
    # workspace each), so one step's copies overlap the other steps' copies
    # and work, as a caller streaming independent tensors would run them.
    # The host link bounds this (both copy directions at once share it).
    e2e = None
    if not args.no_e2e:
        lanes = 3
        host_in = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        host_in.copy_(x.cpu())
        lane = []
        for _ in range(lanes):
            lane.append({"s": torch.cuda.Stream(device), "x": torch.empty_like(x),
                         "o": torch.empty_like(out),
                         "w": torch.empty(max(wsb, 256), dtype=torch.uint8, device=device),
                         "h": torch.empty(out.shape, dtype=out.dtype, pin_memory=True)})
        e2e_steps = max(4, min(args.steps, 200))

        def e2e_step(i):
            L = lane[i % lanes]
            with torch.cuda.stream(L["s"]):
                L["x"].copy_(host_in, non_blocking=True)
                rc = ex.exsum_excluded_ws(L["x"].data_ptr(), L["o"].data_ptr(), d, shape, k, opc,
                                          code, L["w"].data_ptr(), wsb, L["s"].cuda_stream)
                if rc != 0:
                    raise ex.ExsumError(rc, "exsum_excluded_ws")
                L["h"].copy_(L["o"], non_blocking=True)

        for i in range(2 * lanes):
            e2e_step(i)
        torch.cuda.synchronize()
        t_a, t_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_a.record(stream)
        for L in lane:
            L["s"].wait_stream(stream)
        for i in range(e2e_steps):
            e2e_step(i)
        for L in lane:
            stream.wait_stream(L["s"])
        t_b.record(stream)
        torch.cuda.synchronize()
        e_s = t_a.elapsed_time(t_b) / 1e3 / e2e_steps
        e_s = max_over_ranks(e_s, world, device)
        same = all(torch.equal(L["h"], lane[0]["h"]) for L in lane)
        e2e = {"value": round(whole_job_rate(N, world, e_s) / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": x.numel() * x.element_size(),
               "d2h_bytes_per_step": out.numel() * out.element_size(), "steps": e2e_steps,
               "lanes": lanes, "ms_per_step": round(e_s * 1e3, 4), "lanes_agree": same}
        out.copy_(lane[0]["o"])

    # ---- CPU oracle baseline (rank 0, N = 1 only) ------------------------------------------------
    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, ref = cpu_baseline(vals, spec, budget_s=12.0)
        if ref is not None:
            accuracy = accuracy_vs_oracle(out.cpu().numpy(), ref, dtype, op)
        try:
            cpu["all_cores"] = cpu_all_cores(vals, spec, budget_s=6.0)
        except Exception as e:  # no OpenMP-capable compiler on this host
            cpu["all_cores"] = {"unavailable": str(e)[:200]}

    # ---- compact batched, served and comparator figures (rank 0, N = 1) -----------------------------------
    batched = served = comparators = None
    if rank == 0 and world == 1 and not args.no_extras:
        try:
            batched = batched_bench(64, steps=10, warmup=2, plain_steps=2)
        except Exception as e:
            batched = {"error": str(e)[:300]}
        try:
            served = served_bench(1500)
        except Exception as e:
            served = {"error": str(e)[:300]}
        try:
            comparators = comparators_bench(compact=True)
        except Exception as e:
            comparators = {"error": str(e)[:300]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic (seeded Philox, uniform; shapes of the paper's workloads)",
            "config": workload_config(args.workload, shape, k, op, world),
            "roofline": roofline,
            "one_read_one_write": {"bytes": one_rw, "achieved_gbs":
                                   round(one_rw / (ms_per_step * 1e-3) / 1e9, 1),
                                   "frac": round(one_rw / (ms_per_step * 1e-3) / 1e9 / peak, 4)},
            "passes": passes,
            "lowest_level0_pass": (min((p_ for p_ in passes if p_["level"] == 0),
                                       key=lambda p_: p_["frac"], default=None) or {}).get("kernel"),
            "l2_warm": {"value": round(whole_job_rate(N, world, warm_ms * 1e-3) / 1e9, 3),
                        "ms_per_step": round(warm_ms, 5), "steps": warm_steps,
                        "note": "same graph back to back, no L2 flush between steps"},
            "e2e": e2e, "gpu_launches": launches, "clocks": clk, "cpu_baseline": cpu,
            "batched": batched, "served": served, "comparators": comparators,
            "accuracy": accuracy,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def accuracy_vs_oracle(got, ref, dtype, op):
    """Error of the GPU result against the oracle's (fp64 / int64) result."""
    import numpy as np
    if dtype in ("i32", "i64") or op == "max":
        want = ref
        if dtype == "i32":
            want = np.where(ref == np.iinfo(np.int64).min, np.iinfo(np.int32).min,
                            ref).astype(np.int32) if op == "max" else ref.astype(np.int32)
        elif dtype == "i64":
            want = ref.astype(np.int64)
        else:
            want = ref.astype(np.float32)
        return {"exact": bool(np.array_equal(got, want)),
                "mismatches": int(np.count_nonzero(got != want))}
    g = got.astype(np.float64).ravel()
    r = ref.astype(np.float64).ravel()
    rms = float(np.sqrt(np.mean(r * r)))
    diff = np.abs(g - r)
    floored = float(np.max(diff / np.maximum(np.abs(r), rms)))
    nz = np.abs(r) > 0
    return {"vs": "fp64 oracle", "max_rel_floored": floored,
            "max_rel_unfloored": float(np.max(diff[nz] / np.abs(r[nz]))) if nz.any() else 0.0,
            "normwise": float(np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300)),
            "tolerance": 1e-5, "within": floored <= 1e-5}


def cpu_baseline(vals, spec, budget_s):
    """The CPU oracle's box-complement timed on this host, on whole tensors
    of the workload when one run fits the budget, else on leading slabs.
    Returns (record, oracle result of the whole tensor or None)."""
    import numpy as np
    from oracle import oracle
    shape, k, op = spec["shape"], spec["k"], spec["op"]
    sample = np.ascontiguousarray(vals[:1]) if len(shape) > 1 else np.ascontiguousarray(
        vals[: 1 << 16])
    t0 = time.perf_counter()
    oracle.box_complement(sample, [min(kk, nn) for kk, nn in zip(k, sample.shape)], op)
    per_elem = (time.perf_counter() - t0) / sample.size
    N = int(np.prod(shape))
    if per_elem * N <= budget_s:
        runs = max(1, int(budget_s // (per_elem * N)))
        t0 = time.perf_counter()
        for _ in range(runs):
            ref = oracle.box_complement(vals, k, op)
        dt = time.perf_counter() - t0
        return ({"value": round(runs * N / dt / 1e9, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
                 "sample": "%d run(s) of the whole %s tensor, single-threaded C oracle "
                           "(box-complement)" % (runs, "x".join(map(str, shape)))}, ref)
    rows = max(1, int(budget_s / (per_elem * (N // shape[0]))))
    rows = min(rows, shape[0])
    slab = np.ascontiguousarray(vals[:rows])
    kk = [min(a, b) for a, b in zip(k, slab.shape)]
    t0 = time.perf_counter()
    oracle.box_complement(slab, kk, op)
    dt = time.perf_counter() - t0
    return ({"value": round(slab.size / dt / 1e9, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
             "sample": "leading %d of %d slabs along dim 1, single-threaded C oracle" % (
                 rows, shape[0])}, None)


def cpu_all_cores(vals, spec, budget_s):
    """The same box-complement oracle with its independent rows spread over
    all host cores (OpenMP variant, bit-identical results), on the whole
    tensor."""
    from oracle import oracle
    shape, k, op = spec["shape"], spec["k"], spec["op"]
    N = 1
    for s_ in shape:
        N *= s_
    t0 = time.perf_counter()
    oracle.box_complement_omp(vals, k, op)
    first = time.perf_counter() - t0
    runs = max(1, min(20, int(budget_s // max(first, 1e-6))))
    t0 = time.perf_counter()
    for _ in range(runs):
        oracle.box_complement_omp(vals, k, op)
    dt = time.perf_counter() - t0
    return {"value": round(runs * N / dt / 1e9, 5), "unit": UNIT, "cores": oracle.omp_threads(),
            "kind": "oracle_openmp", "nproc": os.cpu_count(),
            "sample": "%d run(s) of the whole %s tensor, OpenMP oracle over rows" % (
                runs, "x".join(map(str, shape)))}


# ---- reference arm: the CPU oracle -------------------------------------------------------------

def workload_config(workload, shape, k, op, world):
    """The `config` of a single-workload line: the workload, how the timed
    steps treat the L2, and how ranks split the work.  Both arms print the
    same object, so that their lines describe one configuration."""
    return {"workload": workload, "shape": list(shape), "k": list(k), "op": op,
            "l2": "flushed between steps (256 MiB write + read back, outside the timed spans)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args):
    import numpy as np
    from oracle import oracle
    from paper_2106_00124_gb300 import synth

    rank, world, _ = dist_env()
    if rank != 0:
        return
    oracle.build()
    dev, vals, spec = synth.workload_input(args.workload)
    shape, k, op = spec["shape"], spec["k"], spec["op"]
    # Each step runs the oracle on the leading slab of the tensor along dim 1,
    # sized so the whole run stays near two minutes of CPU time.
    probe = np.ascontiguousarray(vals[:1]) if len(shape) > 1 else np.ascontiguousarray(vals[:4096])
    t0 = time.perf_counter()
    oracle.box_complement(probe, [min(a, b) for a, b in zip(k, probe.shape)], op)
    per_elem = (time.perf_counter() - t0) / probe.size
    budget_per_step = 120.0 / max(1, args.steps + args.warmup)
    if len(shape) > 1:
        plane = int(np.prod(shape[1:]))
        rows = int(max(1, min(shape[0], budget_per_step / (per_elem * plane))))
        sample = np.ascontiguousarray(vals[:rows])
        desc = "leading %d of %d slabs along dim 1 per step" % (rows, shape[0])
    else:
        n = int(max(k[0], min(shape[0], budget_per_step / per_elem)))
        sample = np.ascontiguousarray(vals[:n])
        desc = "leading %d of %d elements per step" % (n, shape[0])
    kk = [min(a, b) for a, b in zip(k, sample.shape)]
    for _ in range(args.warmup):
        oracle.box_complement(sample, kk, op)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.box_complement(sample, kk, op)
    dt = time.perf_counter() - t0
    value = sample.size * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": spec["dtype"], "data": "synthetic",
        "config": workload_config(args.workload, shape, k, op, world),
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_profile_once(args):
    """Two plain calls of the workload's excluded sum, for profilers; the L2
    is flushed (256 MiB written, then read back) before each call, as
    between the bench's timed steps."""
    import numpy as np
    import torch

    import paper_2106_00124_gb300 as ex
    from paper_2106_00124_gb300 import synth
    torch.cuda.set_device(0)
    dev, _, spec = synth.workload_input(args.workload)
    x = (torch.from_numpy(np.ascontiguousarray(dev).view(np.int16)).view(torch.bfloat16)
         if spec["dtype"] == "bf16" else torch.from_numpy(np.ascontiguousarray(dev))).cuda()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        flush.fill_(1)
        flush.view(torch.int64).max()
        ex.excluded(x, spec["k"], spec["op"])
    torch.cuda.synchronize()
    print(json.dumps({"profile_once": args.workload, "launches": ex.exsum_launch_count()}))


def _seeded_device_tensors(shapes, seed, dtype):
    """Seeded synthetic tensors generated on the device (uniform [-1, 1) fp32,
    or integers in [-1000, 1000] for int64)."""
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    out = []
    for shape in shapes:
        if dtype == "f32":
            out.append(torch.rand(shape, generator=gen, device="cuda") * 2 - 1)
        else:
            out.append(torch.randint(-1000, 1001, shape, generator=gen, device="cuda",
                                     dtype=torch.int64))
    return out


def batched_bench(count, seed=11, steps=20, warmup=3, plain_steps=3):
    """`count` uneven tensors: d in {2, 3}, sides uniform in [32, 512] (at
    most 2^24 elements), k_i uniform in [2, 32], fp32 uniform [-1, 1), +;
    one planned, graph-captured batch against plain per-tensor launches on
    one stream.  Returns the record."""
    import numpy as np
    import torch

    import paper_2106_00124_gb300 as ex
    from paper_2106_00124_gb300 import synth
    spec = synth.batched_shapes(count, seed=seed)
    xs = _seeded_device_tensors([s_ for s_, _ in spec], seed, "f32")
    outs = [torch.empty_like(x) for x in xs]
    descs = [ex.make_desc(x.data_ptr(), o.data_ptr(), sh, k, ex.OP_ADD, ex.F32)
             for x, o, (sh, k) in zip(xs, outs, spec)]
    total = sum(int(np.prod(sh)) for sh, _ in spec)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    rc, plan = ex.exsum_batch_create(descs, lanes=0, stream=stream.cuda_stream)
    tune_s = time.perf_counter() - t0
    assert rc == 0, ex.strerror(rc)
    _, lanes, order, wsb, kernels = ex.exsum_batch_info(plan)
    _, mode, nlevel, lc, inter, tpv, tall, persist = ex.exsum_batch_schedule(plan)
    for _ in range(max(1, warmup)):
        ex.exsum_batch_launch(plan, stream.cuda_stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        ex.exsum_batch_launch(plan, stream.cuda_stream)
    b.record(stream)
    torch.cuda.synchronize()
    batch_ms = a.elapsed_time(b) / steps
    # plain per-tensor launches on one stream (no graph, no concurrency)
    need = max(ex.exsum_workspace_bytes(len(sh), sh, k, ex.OP_ADD, ex.F32, 1)[0] for sh, k in spec)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    sp = stream.cuda_stream

    def plain():
        for x, o, (sh, k) in zip(xs, outs, spec):
            ex.exsum_excluded_ws(x.data_ptr(), o.data_ptr(), len(sh), sh, k, ex.OP_ADD, ex.F32,
                                 ws.data_ptr(), need, sp)
    plain()
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs[:8]]
    a.record(stream)
    for _ in range(plain_steps):
        plain()
    b.record(stream)
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(b) / plain_steps
    ex.exsum_batch_launch(plan, sp)
    torch.cuda.synchronize()
    # the plain launches' results (checked against the oracle by the tests)
    # against the plan's: equal bits on lanes, within the fp32 bound on levels
    rel = 0.0
    for r_, o in zip(ref, outs[:8]):
        r64, o64 = r_.double(), o.double()
        scale = torch.clamp(r64.abs(), min=float(torch.sqrt(torch.mean(r64 * r64))))
        rel = max(rel, float(((o64 - r64).abs() / scale).max()))
    same = all(torch.equal(r_, o) for r_, o in zip(ref, outs[:8]))
    ex.exsum_batch_destroy(plan)
    return {
        "metric": "batched excluded-sum Gelem/s", "unit": "Gelem/s",
        "value": round(total / (batch_ms * 1e-3) / 1e9, 3),
        "plain_value": round(total / (plain_ms * 1e-3) / 1e9, 3),
        "speedup_vs_plain": round(plain_ms / batch_ms, 3), "ms_per_batch": round(batch_ms, 3),
        "plain_ms_per_batch": round(plain_ms, 3), "tensors": len(spec), "elements": total,
        "schedule": {"mode": ["lanes", "levels"][mode], "level_tensors": nlevel,
                     "lanes": lanes, "order": ["lpt", "round_robin"][order],
                     "level_tune": {"lc": lc, "interleave": inter, "tiles_per_vb": tpv, "tall": tall,
                                    "persist": persist},
                     "kernels_per_launch": kernels, "workspace_bytes": wsb,
                     "autotune_s": round(tune_s, 2)},
        "identical_to_plain": same, "max_rel_diff_vs_plain": rel,
        "dtype": "f32", "data": "synthetic (seeded, on device)",
        "config": {"workload": "batched_%d_uneven_d2d3_f32_add" % count,
                   "sides": [32, 512], "k": [2, 32], "cap": 1 << 24},
        "plain": "the same tensors, one exsum_excluded_ws call each on one stream"}


def run_batched_profile_once(count=512, seed=11):
    """The batched workload's level schedule, planned without autotuning
    (EXSUM_LEVEL_TUNE gives the tuning) and launched twice, for profilers."""
    import torch

    import paper_2106_00124_gb300 as ex
    from paper_2106_00124_gb300 import synth
    torch.cuda.set_device(0)
    spec = synth.batched_shapes(count, seed=seed)
    xs = _seeded_device_tensors([s_ for s_, _ in spec], seed, "f32")
    outs = [torch.empty_like(x) for x in xs]
    descs = [ex.make_desc(x.data_ptr(), o.data_ptr(), sh, k, ex.OP_ADD, ex.F32)
             for x, o, (sh, k) in zip(xs, outs, spec)]
    sp = torch.cuda.current_stream().cuda_stream
    rc, plan = ex.exsum_batch_create(descs, lanes=ex.BATCH_LEVELS, stream=sp)
    assert rc == 0, ex.strerror(rc)
    for _ in range(2):
        assert ex.exsum_batch_launch(plan, sp) == 0
    torch.cuda.synchronize()
    sched = ex.exsum_batch_schedule(plan)
    ex.exsum_batch_destroy(plan)
    print(json.dumps({"profile_once": "batched_%d" % count, "schedule": list(sched[1:])}))


def run_batched(args):
    """The 512-tensor batched workload."""
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(batched_bench(512, steps=max(3, min(args.steps, 20)), warmup=args.warmup)),
          flush=True)


def served_bench(nreq, slots=8, seed=12):
    """A Poisson stream of `nreq` excluded-sum requests per offered load
    (shapes and boxes as in the batched workload, 90% fp32 +, 10% int64 max)
    served with continuous batching at 0.5, 0.8 and 1.0 of the saturated
    rate, against plain launches: the same arrivals, each request one
    exsum_excluded call on one stream as it arrives.  Returns the record."""
    import numpy as np
    import torch

    import paper_2106_00124_gb300 as ex
    from paper_2106_00124_gb300 import synth
    f_spec = synth.batched_shapes(48, seed=seed)
    i_spec = synth.batched_shapes(8, seed=seed + 1)
    fx = _seeded_device_tensors([s_ for s_, _ in f_spec], seed, "f32")
    ix = _seeded_device_tensors([s_ for s_, _ in i_spec], seed + 1, "i64")
    fo = [torch.empty_like(x) for x in fx]
    io = [torch.empty_like(x) for x in ix]
    rng = np.random.default_rng(seed + 2)
    kinds = rng.random(nreq) < 0.1
    picks = [int(rng.integers(0, len(i_spec) if kd else len(f_spec))) for kd in kinds]
    descs, sizes, calls = [], [], []
    for kd, j in zip(kinds, picks):
        if kd:
            sh, k = i_spec[j]
            args_ = (ix[j].data_ptr(), io[j].data_ptr(), len(sh), sh, k, ex.OP_MAX, ex.I64)
        else:
            sh, k = f_spec[j]
            args_ = (fx[j].data_ptr(), fo[j].data_ptr(), len(sh), sh, k, ex.OP_ADD, ex.F32)
        descs.append(ex.make_desc(args_[0], args_[1], sh, k, args_[5], args_[6]))
        calls.append(args_)
        sizes.append(int(np.prod(sh)))
    budget = 40 << 30

    def stats(lat, first, last, n):
        span = (last - first) / 1e9
        return {"p50_ms": round(float(np.percentile(lat, 50)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "throughput_req_s": round(n / span, 1),
                "gelem_s": round(sum(sizes[:n]) / span / 1e9, 3)}

    def arrivals_for(rate, n, start):
        if rate is None:
            return np.full(n, start, dtype=np.int64)
        return (start + np.cumsum(rng.exponential(1e9 / rate, size=n))).astype(np.int64)

    def serve(rate, n):
        srv = ex.exsum_server_create(budget, slots)
        assert srv
        arr = arrivals_for(rate, n, ex.exsum_server_now_ns() + 200_000_000)
        tickets = []
        for i in range(n):
            rc, t = ex.exsum_server_submit_at(srv, descs[i], 0, int(arr[i]))
            assert rc == 0
            tickets.append(t)
        for t in tickets:
            rc = ex.exsum_server_wait(srv, t, 60 * 10 ** 9)
            if rc != 0:
                raise RuntimeError("served request %d: %s" % (t, ex.strerror(rc)))
        lat, first, last = [], None, 0
        for t in tickets:
            _, sub, st_, done = ex.exsum_server_ticket_times(srv, t)
            lat.append((done - sub) / 1e6)
            first = sub if first is None else min(first, sub)
            last = max(last, done)
        ex.exsum_server_destroy(srv)
        return stats(lat, first, last, n)

    def plain(rate, n):
        # one stream, one exsum_excluded call per request at its arrival
        # time; completion times from events, mapped onto the host clock by
        # a reference event recorded right before the first arrival
        stream = torch.cuda.Stream()
        sp = stream.cuda_stream
        for c in calls[:8]:   # the stream's workspace and side streams exist before timing
            ex.exsum_excluded(c[0], c[1], c[2], c[3], c[4], c[5], c[6], sp)
        stream.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        ref = torch.cuda.Event(enable_timing=True)
        ref.record(stream)
        stream.synchronize()
        t_ref = ex.exsum_server_now_ns()
        arr = arrivals_for(rate, n, t_ref + 50_000_000)
        for i in range(n):
            while ex.exsum_server_now_ns() < arr[i]:
                pass
            c = calls[i]
            rc = ex.exsum_excluded(c[0], c[1], c[2], c[3], c[4], c[5], c[6], sp)
            assert rc == 0, ex.strerror(rc)
            evs[i].record(stream)
        stream.synchronize()
        done = [t_ref + int(ref.elapsed_time(e) * 1e6) for e in evs]
        lat = [(d_ - a_) / 1e6 for d_, a_ in zip(done, arr)]
        return stats(lat, int(arr[0]), max(done), n)

    sat = serve(None, nreq)          # saturated: everything arrives at once
    sat_rate = sat["throughput_req_s"]
    loads = {}
    for f in (0.5, 0.8, 1.0):
        loads[str(f)] = {"offered_req_s": round(f * sat_rate, 1),
                         "served": serve(f * sat_rate, nreq),
                         "plain": plain(f * sat_rate, nreq)}
    return {
        "metric": "served excluded-sum p50/p99 latency and throughput", "unit": "ms / req/s",
        "requests_per_load": nreq, "slots": slots, "budget_bytes": budget,
        "saturated": sat, "loads": loads, "dtype": "f32 (+ int64 max)",
        "data": "synthetic (seeded, on device)",
        "config": {"workload": "served_poisson_uneven_d2d3_f32add_i64max",
                   "plain": "the same arrivals, one exsum_excluded call each on one stream"}}


def _event_ms(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def comparators_bench(compact=False, reps=5):
    """The paper's comparison methods on this GPU (int64 +, seeded uniform
    [-1000, 1000], k = 8 per dimension, about 2^24 elements per d; d = 1
    uses k = 64): box-complement (strong excluded sum), BDBSC (weak),
    SAT with inclusion-exclusion (weak) and corners (strong, d = 2, 3), in
    Gelem/s; then the operator cost: the slowed int64 + at several extra
    costs on a 128^3 tensor (k = 4), each method's slope of time against
    the extra cost over the calibration kernel's slope per application:
    operator applications per element, weighted by how serial each method's
    chains of applications are.  Returns the record."""
    import numpy as np
    import torch

    import paper_2106_00124_gb300 as ex
    torch.cuda.set_device(0)
    sweep = [(3, 256)] if compact else [(1, 1 << 24), (2, 4096), (3, 256), (4, 64), (5, 28), (6, 16)]
    rows = []
    g = torch.Generator(device="cuda")
    for d, side in sweep:
        sh = [side] * d
        k = [64] if d == 1 else [8] * d
        N = int(np.prod(sh))
        g.manual_seed(1000 + d)
        x = torch.randint(-1000, 1001, sh, dtype=torch.int64, device="cuda", generator=g)
        o = torch.empty_like(x)
        r = {"d": d, "shape": sh, "k": k}
        for name, fn in (("box_complement", lambda: ex.excluded(x, k, "add", out=o)),
                         ("bdbsc", lambda: ex.excluded_weak(x, k, out=o)),
                         ("satc", lambda: ex.sat(x, k, excluded=True, out=o)),
                         ("corners", (lambda: ex.corners(x, k, "add", out=o)) if d in (2, 3) else None)):
            if fn is None:
                continue
            ms = _event_ms(fn, reps)
            r[name] = {"ms": round(ms, 4), "gelem_s": round(N / (ms * 1e-3) / 1e9, 2)}
        rows.append(r)
        del x, o
    # operator cost
    sh, k = [128, 128, 128], [4, 4, 4]
    N = int(np.prod(sh))
    g.manual_seed(77)
    x = torch.randint(-1000, 1001, sh, dtype=torch.int64, device="cuda", generator=g)
    o = torch.empty_like(x)
    sp = torch.cuda.current_stream().cuda_stream
    extras = [0, 64, 256] if compact else [0, 32, 64, 128, 256]
    methods = {"calibration": ex.SLOW_CALIBRATE, "box_complement": ex.SLOW_BOX_COMPLEMENT,
               "bdbs": ex.SLOW_BDBS, "corners": ex.SLOW_CORNERS}
    times = {m: [] for m in methods}
    try:
        for e in extras:
            assert ex.exsum_slow_extra(e) == 0
            for m, code in methods.items():
                def run(code=code):
                    rc = ex.exsum_slow_run(x.data_ptr(), o.data_ptr(), 3, sh, k, code, sp)
                    assert rc == 0, ex.strerror(rc)
                times[m].append(_event_ms(run, 2))
    finally:
        ex.exsum_slow_extra(0)
    slope = {m: float(np.polyfit(extras, t, 1)[0]) for m, t in times.items()}
    per_app = slope["calibration"] / ex.SLOW_CALIBRATE_REPS
    ops = {m: round(slope[m] / per_app, 2) for m in methods if m != "calibration"}
    return {"metric": "comparators: Gelem/s per method and d; operator applications per element",
            "dtype": "i64", "op": "add", "data": "synthetic (seeded, on device)", "sweep": rows,
            "operator_cost": {"shape": sh, "k": k, "extra_costs": extras,
                              "ms": {m: [round(t, 4) for t in v] for m, v in times.items()},
                              "effective_applications_per_element": ops,
                              "note": "time slope per unit of operator cost over that of one fully parallel "
                                      "application per element: operator applications per element, weighted "
                                      "by how serial their chains are (a thread walking a line pays latency)"}}


def run_comparators(args):
    print(json.dumps(comparators_bench()), flush=True)


def run_served(args):
    """The served workload at its full request count."""
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(served_bench(args.requests)), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.mode == "batched":
        if args.profile_once:
            run_batched_profile_once()
        else:
            run_batched(args)
        return
    if args.mode == "served":
        run_served(args)
        return
    if args.mode == "comparators":
        run_comparators(args)
        return
    if args.profile_once:
        run_profile_once(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
