"""GB300 (sm_103a) CUDA library for multidimensional included and excluded sums.

Xu, Fraser, Leiserson, "Multidimensional Included and Excluded Sums"
(SIAM ACDA 2021): BDBS for included sums (Sec. 3) and box-complement for
strong excluded sums (Sec. 4-5), as hand-written CUDA behind a small C ABI
(``include/exsum.h``).

This module is a thin ctypes binding: the functions named ``exsum_*`` take
the same arguments as the C entry points (device pointers as integers, host
sequences for shape and box, a cudaStream_t as an integer) and return the C
status code.  ``included`` / ``excluded`` are conveniences over torch CUDA
tensors that allocate the output and raise ``ExsumError`` on failure.  All
arithmetic runs in the CUDA library; there is no CPU fallback, and calling
anything without the built library raises.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libexsum.so")

OP_ADD, OP_MAX = 0, 1
I32, I64, F32, BF16 = 0, 1, 2, 3
EXSUM_OK, EXSUM_EINVAL, EXSUM_ENOMEM, EXSUM_EUNSUPPORTED, EXSUM_ECUDA, EXSUM_ETIMEDOUT, EXSUM_EBUSY = (
    0, -1, -2, -3, -4, -5, -6)
MAX_DIMS = 8

OPS = {"add": OP_ADD, "max": OP_MAX}
DTYPES = {"i32": I32, "i64": I64, "f32": F32, "bf16": BF16}


class ExsumError(RuntimeError):
    """A non-zero status from the C library."""

    def __init__(self, status, what=""):
        self.status = status
        msg = "%s: %s (status %d)" % (what or "exsum", strerror(status), status)
        if status == EXSUM_ECUDA:
            msg += ", cudaError %d" % _load().exsum_last_cuda_error()
        super().__init__(msg)


_lib = None


class exsum_desc(ctypes.Structure):
    """C struct exsum_desc: one tensor of a batch or one served request."""
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("d", ctypes.c_int),
                ("op", ctypes.c_int), ("dtype", ctypes.c_int),
                ("shape", ctypes.c_int64 * MAX_DIMS), ("k", ctypes.c_int64 * MAX_DIMS)]


def make_desc(in_ptr, out_ptr, shape, k, op, dtype):
    """An exsum_desc for device (or, for served host requests, host) pointers."""
    dsc = exsum_desc()
    dsc.in_ = in_ptr
    dsc.out = out_ptr
    dsc.d = len(shape)
    dsc.op = int(op)
    dsc.dtype = int(dtype)
    for i, (n, kk) in enumerate(zip(shape, k)):
        dsc.shape[i] = int(n)
        dsc.k[i] = int(kk)
    return dsc


SERVE_HOST = 1
BATCH_LEVELS = -1

_P = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_SIG = {
    "exsum_version": ([], ctypes.c_int),
    "exsum_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "exsum_last_cuda_error": ([], ctypes.c_int),
    "exsum_out_dtype": ([ctypes.c_int], ctypes.c_int),
    "exsum_dtype_size": ([ctypes.c_int], ctypes.c_size_t),
    "exsum_workspace_bytes": ([ctypes.c_int, _I64P, _I64P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_int)], ctypes.c_size_t),
    "exsum_included": ([_P, _P, ctypes.c_int, _I64P, _I64P, ctypes.c_int, ctypes.c_int, _P],
                       ctypes.c_int),
    "exsum_excluded": ([_P, _P, ctypes.c_int, _I64P, _I64P, ctypes.c_int, ctypes.c_int, _P],
                       ctypes.c_int),
    "exsum_included_ws": ([_P, _P, ctypes.c_int, _I64P, _I64P, ctypes.c_int, ctypes.c_int, _P,
                           ctypes.c_size_t, _P], ctypes.c_int),
    "exsum_excluded_ws": ([_P, _P, ctypes.c_int, _I64P, _I64P, ctypes.c_int, ctypes.c_int, _P,
                           ctypes.c_size_t, _P], ctypes.c_int),
    "exsum_release_cached_workspace": ([], ctypes.c_int),
    "exsum_excluded_noalloc": ([_P, _P, ctypes.c_int, _I64P, _I64P, ctypes.c_int, ctypes.c_int, _P],
                               ctypes.c_int),
    "exsum_trace_enable": ([ctypes.c_int], None),
    "exsum_trace_collect": ([ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_float),
                             ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "exsum_kernel_name": ([ctypes.c_int], ctypes.c_char_p),
    "exsum_launch_count": ([], ctypes.c_int64),
    "exsum_side_streams_created": ([], ctypes.c_int64),
    "exsum_excluded_weak": ([_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                             ctypes.POINTER(ctypes.c_int64), ctypes.c_int, _P], ctypes.c_int),
    "exsum_graph_instantiate": ([_P, ctypes.POINTER(_P)], ctypes.c_int),
    "exsum_graph_launch": ([_P, _P], ctypes.c_int),
    "exsum_graph_exec_destroy": ([_P], ctypes.c_int),
    "exsum_batch_create": ([ctypes.POINTER(exsum_desc), ctypes.c_int, ctypes.c_int, _P,
                            ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "exsum_batch_launch": ([_P, _P], ctypes.c_int),
    "exsum_batch_info": ([_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int64)],
                         ctypes.c_int),
    "exsum_sat": ([_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                   ctypes.c_int, ctypes.c_int, _P], ctypes.c_int),
    "exsum_corners": ([_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                       ctypes.c_int, ctypes.c_int, _P], ctypes.c_int),
    "exsum_corner_region": ([ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "exsum_device_timeouts": ([], ctypes.c_uint),
    "exsum_slow_extra": ([ctypes.c_int], ctypes.c_int),
    "exsum_slow_run": ([_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                        ctypes.c_int, _P], ctypes.c_int),
    "exsum_batch_schedule": ([_P] + [ctypes.POINTER(ctypes.c_int)] * 7, ctypes.c_int),
    "exsum_batch_destroy": ([_P], None),
    "exsum_server_create": ([ctypes.c_size_t, ctypes.c_int], _P),
    "exsum_server_submit": ([_P, ctypes.POINTER(exsum_desc), ctypes.c_int,
                             ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "exsum_server_submit_at": ([_P, ctypes.POINTER(exsum_desc), ctypes.c_int, ctypes.c_int64,
                                ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "exsum_server_now_ns": ([], ctypes.c_int64),
    "exsum_server_wait": ([_P, ctypes.c_uint64, ctypes.c_int64], ctypes.c_int),
    "exsum_server_ticket_times": ([_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
                                  ctypes.c_int),
    "exsum_server_release": ([_P, ctypes.c_uint64], ctypes.c_int),
    "exsum_server_completed": ([_P], ctypes.c_int64),
    "exsum_server_fail_next": ([_P, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "exsum_server_destroy": ([_P], None),
}


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "the CUDA library %s is not built; run `python -m paper_2106_00124_gb300.build` "
                "(or __graft_entry__.build()) on a machine with nvcc" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIG.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def declared_symbols():
    """Names of the C entry points this binding expects the library to export."""
    return sorted(_SIG)


def _arr(seq):
    return (ctypes.c_int64 * len(seq))(*[int(v) for v in seq])


# ---- C-ABI mirrors: argument marshalling only -------------------------------------------------

def exsum_version():
    return _load().exsum_version()


def strerror(status):
    return _load().exsum_strerror(int(status)).decode()


exsum_strerror = strerror


def exsum_last_cuda_error():
    return _load().exsum_last_cuda_error()


def exsum_out_dtype(dtype):
    return _load().exsum_out_dtype(int(dtype))


def exsum_dtype_size(dtype):
    return _load().exsum_dtype_size(int(dtype))


def exsum_workspace_bytes(d, shape, k, op, dtype, excluded):
    """Returns (bytes, status)."""
    st = ctypes.c_int(0)
    b = _load().exsum_workspace_bytes(int(d), _arr(shape), _arr(k), int(op), int(dtype),
                                      int(bool(excluded)), ctypes.byref(st))
    return int(b), st.value


def exsum_included(in_ptr, out_ptr, d, shape, k, op, dtype, stream=0):
    return _load().exsum_included(in_ptr, out_ptr, int(d), _arr(shape), _arr(k), int(op),
                                  int(dtype), stream or None)


def exsum_excluded(in_ptr, out_ptr, d, shape, k, op, dtype, stream=0):
    return _load().exsum_excluded(in_ptr, out_ptr, int(d), _arr(shape), _arr(k), int(op),
                                  int(dtype), stream or None)


def exsum_excluded_weak(in_ptr, out_ptr, d, shape, k, dtype, stream=0):
    return _load().exsum_excluded_weak(in_ptr, out_ptr, int(d), _arr(shape), _arr(k), int(dtype),
                                       stream or None)


def exsum_included_ws(in_ptr, out_ptr, d, shape, k, op, dtype, ws_ptr, ws_bytes, stream=0):
    return _load().exsum_included_ws(in_ptr, out_ptr, int(d), _arr(shape), _arr(k), int(op),
                                     int(dtype), ws_ptr, int(ws_bytes), stream or None)


def exsum_excluded_ws(in_ptr, out_ptr, d, shape, k, op, dtype, ws_ptr, ws_bytes, stream=0):
    return _load().exsum_excluded_ws(in_ptr, out_ptr, int(d), _arr(shape), _arr(k), int(op),
                                     int(dtype), ws_ptr, int(ws_bytes), stream or None)


# Size of the static scratch buffer behind exsum_excluded_noalloc (bytes).
NOALLOC_SCRATCH_BYTES = 64 << 20


def exsum_excluded_noalloc(in_ptr, out_ptr, d, shape, k, op, dtype, stream=0):
    """Excluded sums on the library's static scratch buffer: no allocation.
    For callers that cannot allocate device memory at call time."""
    return _load().exsum_excluded_noalloc(in_ptr, out_ptr, int(d), _arr(shape), _arr(k), int(op),
                                          int(dtype), stream or None)


def exsum_release_cached_workspace():
    return _load().exsum_release_cached_workspace()


def exsum_trace_enable(on):
    _load().exsum_trace_enable(int(bool(on)))


def exsum_trace_collect(cap=4096, clear=True):
    """Returns a list of (kernel_name, level, elements, ms); clears the trace if asked."""
    tags = (ctypes.c_int * cap)()
    levels = (ctypes.c_int * cap)()
    elems = (ctypes.c_int64 * cap)()
    ms = (ctypes.c_float * cap)()
    n = _load().exsum_trace_collect(tags, levels, elems, ms, cap, int(bool(clear)))
    if n < 0:
        raise ExsumError(n, "exsum_trace_collect")
    return [(exsum_kernel_name(tags[i]), levels[i], elems[i], ms[i]) for i in range(min(n, cap))]


def exsum_kernel_name(tag):
    return _load().exsum_kernel_name(int(tag)).decode()


def exsum_launch_count():
    return int(_load().exsum_launch_count())


def exsum_side_streams_created():
    return int(_load().exsum_side_streams_created())


def exsum_graph_instantiate(graph):
    """Instantiates a captured cudaGraph_t (an integer handle, e.g.
    torch.cuda.CUDAGraph(keep_graph=True).raw_cuda_graph()) with per-node
    priorities honoured; returns the cudaGraphExec_t handle."""
    ex = _P()
    rc = _load().exsum_graph_instantiate(_P(int(graph)), ctypes.byref(ex))
    if rc != EXSUM_OK:
        raise ExsumError(rc, "exsum_graph_instantiate")
    return int(ex.value)


def exsum_graph_launch(exec_, stream=0):
    rc = _load().exsum_graph_launch(_P(int(exec_)), _P(int(stream)))
    if rc != EXSUM_OK:
        raise ExsumError(rc, "exsum_graph_launch")


def exsum_graph_exec_destroy(exec_):
    rc = _load().exsum_graph_exec_destroy(_P(int(exec_)))
    if rc != EXSUM_OK:
        raise ExsumError(rc, "exsum_graph_exec_destroy")


def exsum_batch_create(descs, lanes=0, stream=0):
    """Plans a batch (a sequence of exsum_desc); returns (status, plan handle)."""
    arr = (exsum_desc * len(descs))(*descs)
    plan = ctypes.c_void_p(0)
    rc = _load().exsum_batch_create(arr, len(descs), int(lanes), stream or None, ctypes.byref(plan))
    return rc, plan.value


def exsum_batch_launch(plan, stream=0):
    return _load().exsum_batch_launch(plan, stream or None)


def exsum_batch_info(plan):
    """(status, lanes, order, workspace_bytes, kernels_per_launch)."""
    lanes, order, ws, ker = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t(), ctypes.c_int64()
    rc = _load().exsum_batch_info(plan, ctypes.byref(lanes), ctypes.byref(order), ctypes.byref(ws),
                                  ctypes.byref(ker))
    return rc, lanes.value, order.value, ws.value, ker.value


def exsum_sat(in_ptr, out_ptr, d, shape, k, excluded, dtype, stream=0):
    return _load().exsum_sat(in_ptr, out_ptr, d, _arr(shape), _arr(k), int(excluded), dtype, stream or None)


def exsum_corners(in_ptr, out_ptr, d, shape, k, op, dtype, stream=0):
    return _load().exsum_corners(in_ptr, out_ptr, d, _arr(shape), _arr(k), op, dtype, stream or None)


def exsum_device_timeouts():
    """Blocks of the bulk final pass that gave up waiting for a copy (never expected)."""
    return int(_load().exsum_device_timeouts())


def exsum_corner_region(d, corner, dim):
    return _load().exsum_corner_region(d, corner, dim)


SLOW_BOX_COMPLEMENT, SLOW_BDBS, SLOW_CORNERS, SLOW_CALIBRATE = 0, 1, 2, 3
SLOW_CALIBRATE_REPS = 16


def exsum_slow_extra(extra):
    return _load().exsum_slow_extra(int(extra))


def exsum_slow_run(in_ptr, out_ptr, d, shape, k, method, stream=0):
    return _load().exsum_slow_run(in_ptr, out_ptr, d, _arr(shape), _arr(k), int(method), stream or None)


def exsum_batch_schedule(plan):
    """(status, mode, level_tensors, lc, interleave, tiles_per_vb, tall, persist); mode 0 lanes, 1 levels."""
    v = [ctypes.c_int() for _ in range(7)]
    rc = _load().exsum_batch_schedule(plan, *[ctypes.byref(x) for x in v])
    return (rc,) + tuple(x.value for x in v)


def exsum_batch_destroy(plan):
    _load().exsum_batch_destroy(plan)


def exsum_server_create(mem_budget_bytes, max_slots):
    """Returns a server handle, or None."""
    return _load().exsum_server_create(int(mem_budget_bytes), int(max_slots))


def exsum_server_submit(server, desc, flags=0):
    """Returns (status, ticket)."""
    t = ctypes.c_uint64(0)
    rc = _load().exsum_server_submit(server, ctypes.byref(desc), int(flags), ctypes.byref(t))
    return rc, t.value


def exsum_server_submit_at(server, desc, flags, arrival_ns):
    """Returns (status, ticket); the request is not admitted before arrival_ns."""
    t = ctypes.c_uint64(0)
    rc = _load().exsum_server_submit_at(server, ctypes.byref(desc), int(flags), int(arrival_ns),
                                        ctypes.byref(t))
    return rc, t.value


def exsum_server_now_ns():
    return int(_load().exsum_server_now_ns())


def exsum_server_wait(server, ticket, timeout_ns):
    return _load().exsum_server_wait(server, int(ticket), int(timeout_ns))


def exsum_server_ticket_times(server, ticket):
    """Returns (status, submit_ns, start_ns, done_ns)."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = _load().exsum_server_ticket_times(server, int(ticket), ctypes.byref(a), ctypes.byref(b),
                                           ctypes.byref(c))
    return rc, a.value, b.value, c.value


def exsum_server_release(server, ticket):
    return _load().exsum_server_release(server, int(ticket))


def exsum_server_completed(server):
    return int(_load().exsum_server_completed(server))


def exsum_server_fail_next(server, count, status):
    """Host-side fault injection: the next `count` admitted requests end with `status`."""
    return _load().exsum_server_fail_next(server, int(count), int(status))


def exsum_server_destroy(server):
    _load().exsum_server_destroy(server)


# ---- torch conveniences ------------------------------------------------------------------------

def torch_dtype_code(t):
    """exsum dtype code of a torch tensor (int32, int64, float32, bfloat16)."""
    import torch
    table = {torch.int32: I32, torch.int64: I64, torch.float32: F32, torch.bfloat16: BF16}
    if t.dtype not in table:
        raise ExsumError(EXSUM_EINVAL, "unsupported tensor dtype %s" % t.dtype)
    return table[t.dtype]


def _out_like(x, dtype):
    import torch
    out_dtype = {I32: torch.int32, I64: torch.int64, F32: torch.float32, BF16: torch.float32}[dtype]
    return torch.empty(x.shape, dtype=out_dtype, device=x.device)


def _torch_call(fn, x, k, op, out, what):
    import torch
    if not x.is_cuda or not x.is_contiguous():
        raise ExsumError(EXSUM_EINVAL, what + ": input must be a contiguous CUDA tensor")
    dt = torch_dtype_code(x)
    if out is None:
        out = _out_like(x, dt)
    stream = torch.cuda.current_stream(x.device).cuda_stream
    with torch.cuda.device(x.device):
        rc = fn(x.data_ptr(), out.data_ptr(), x.dim(), list(x.shape), list(k), OPS[op], dt, stream)
    if rc != EXSUM_OK:
        raise ExsumError(rc, what)
    return out


def included(x, k, op="add", out=None):
    """Included sums of a contiguous CUDA tensor (bf16 -> fp32 output)."""
    return _torch_call(exsum_included, x, k, op, out, "exsum_included")


def excluded(x, k, op="add", out=None):
    """Strong excluded sums of a contiguous CUDA tensor (bf16 -> fp32 output)."""
    return _torch_call(exsum_excluded, x, k, op, out, "exsum_excluded")


def excluded_weak(x, k, out=None):
    """Weak excluded sums (total minus included) of a contiguous int32/int64
    CUDA tensor, operator +."""
    return _torch_call(lambda i, o, d, sh, kk, op, dt, st: exsum_excluded_weak(i, o, d, sh, kk, dt, st),
                       x, k, "add", out, "exsum_excluded_weak")


def sat(x, k, excluded=True, out=None):
    """Box sums of an integer CUDA tensor through a summed-area table (the
    paper's SAT / SATC comparator): the weak excluded sum, or the included
    sum with excluded=False."""
    def fn(i, o, d, sh, kk, op, dt, st):
        return exsum_sat(i, o, d, sh, kk, excluded, dt, st)
    return _torch_call(fn, x, k, "add", out, "exsum_sat")


def corners(x, k, op="add", out=None):
    """Strong excluded sums of a d = 2 or 3 CUDA tensor by the corners
    algorithm (the paper's comparator, App. A)."""
    return _torch_call(exsum_corners, x, k, op, out, "exsum_corners")
