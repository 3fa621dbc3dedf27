"""CPU oracle for included and excluded sums -- TEST INFRASTRUCTURE ONLY.

Python front end to ``exsum_oracle.c``, a plain single-threaded C
restatement of the definitions and algorithms of Xu, Fraser and Leiserson,
"Multidimensional Included and Excluded Sums" (SIAM ACDA 2021).  Only the
test suite, the smoke check and the CPU-baseline leg of the benchmark may
import this module; the CUDA library never does.

Every function takes a numpy array holding the tensor (row-major, last
dimension contiguous), the box size ``k`` and an operator name (``"add"`` or
``"max"``).  Integer arrays are widened to int64 and floating-point arrays to
float64 exactly before the call; integer ``+`` wraps modulo 2**64, so the low
32 bits of a result are the wrapping int32 result.  bfloat16 inputs are passed
as their float32 values.

Parity status: the definition (``*_brute``, ``*_at``), BDBS, box-complement,
corners (d = 2, 3), SAT and BDBSC are each pinned by the ``-m "not gpu"``
tests (closed forms, invariants, special cases, brute force).
"""

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "exsum_oracle.c")
_LIB = os.path.join(_HERE, "libexsum_oracle.so")

_MON = {("int", "add"): 0, ("int", "max"): 1, ("float", "add"): 2, ("float", "max"): 3}

_lib = None
_SRC_OMP = os.path.join(_HERE, "exsum_oracle_omp.c")
_LIB_OMP = os.path.join(_HERE, "libexsum_oracle_omp.so")
_lib_omp = None


def build(force=False):
    """Compiles the oracle shared library with gcc (plain C99, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build_omp(force=False):
    """Compiles the OpenMP variant of the box-complement oracle (the same
    steps with independent rows spread over the host cores); without an
    OpenMP-capable compiler it is built single-threaded."""
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC_OMP):
        tmp = _LIB_OMP + ".tmp%d" % os.getpid()
        base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC_OMP, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def _load_omp():
    global _lib_omp
    if _lib_omp is None:
        build_omp()
        lib = ctypes.CDLL(_LIB_OMP)
        p, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
        lib.orcp_box_complement.argtypes = [p, p, ctypes.c_int, i64p, i64p, ctypes.c_int]
        lib.orcp_box_complement.restype = ctypes.c_int
        lib.orcp_threads.argtypes = []
        lib.orcp_threads.restype = ctypes.c_int
        _lib_omp = lib
    return _lib_omp


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        p, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
        for name in ("orc_included_brute", "orc_excluded_brute", "orc_bdbs",
                     "orc_box_complement", "orc_corners"):
            fn = getattr(lib, name)
            fn.argtypes = [p, p, ctypes.c_int, i64p, i64p, ctypes.c_int]
            fn.restype = ctypes.c_int
        for name in ("orc_included_at", "orc_excluded_at"):
            fn = getattr(lib, name)
            fn.argtypes = [p, ctypes.c_int, i64p, i64p, ctypes.c_int, i64p, p]
            fn.restype = ctypes.c_int
        for name in ("orc_sat_included", "orc_bdbsc"):
            fn = getattr(lib, name)
            fn.argtypes = [p, p, ctypes.c_int, i64p, i64p]
            fn.restype = ctypes.c_int
        lib.orc_reset_ops.argtypes = []
        lib.orc_reset_ops.restype = None
        lib.orc_get_ops.argtypes = []
        lib.orc_get_ops.restype = ctypes.c_uint64
        lib.orc_corner_threshold_hi.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint]
        lib.orc_corner_threshold_hi.restype = ctypes.c_int
        _lib = lib
    return _lib


def _kind(a):
    return "int" if np.issubdtype(a.dtype, np.integer) else "float"


def _widen(a):
    if _kind(a) == "int":
        return np.ascontiguousarray(a, dtype=np.int64)
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(seq):
    arr = (ctypes.c_int64 * len(seq))(*[int(v) for v in seq])
    return arr


def _call_full(name, a, k, op):
    lib = _load()
    w = _widen(a)
    out = np.empty_like(w)
    mon = _MON[(_kind(a), op)]
    rc = getattr(lib, name)(w.ctypes.data, out.ctypes.data, w.ndim, _i64(w.shape), _i64(k), mon)
    if rc != 0:
        raise ValueError("%s failed with status %d" % (name, rc))
    return out


def included_brute(a, k, op):
    """Included sums straight from the definition (Sec. 2)."""
    return _call_full("orc_included_brute", a, k, op)


def excluded_brute(a, k, op):
    """Excluded sums straight from the definition (Sec. 2); O(N^2)."""
    return _call_full("orc_excluded_brute", a, k, op)


def bdbs(a, k, op):
    """Included sums by BDBS (Sec. 3)."""
    return _call_full("orc_bdbs", a, k, op)


def box_complement(a, k, op):
    """Excluded sums by the box-complement algorithm (Sec. 5)."""
    return _call_full("orc_box_complement", a, k, op)


def box_complement_omp(a, k, op):
    """box_complement with independent rows on all host cores (OpenMP);
    the same steps and operand order, so the same bits."""
    lib = _load_omp()
    w = _widen(a)
    out = np.empty_like(w)
    mon = _MON[(_kind(a), op)]
    rc = lib.orcp_box_complement(w.ctypes.data, out.ctypes.data, w.ndim, _i64(w.shape), _i64(k), mon)
    if rc != 0:
        raise ValueError("orcp_box_complement failed with status %d" % rc)
    return out


def omp_threads():
    """Host threads the OpenMP oracle uses (1 if built without OpenMP)."""
    return int(_load_omp().orcp_threads())


def corners(a, k, op):
    """Excluded sums by the corners algorithm (App. A); d = 2 or 3."""
    return _call_full("orc_corners", a, k, op)


def _call_at(name, a, k, op, x):
    lib = _load()
    w = _widen(a)
    res = np.zeros(1, dtype=w.dtype)
    mon = _MON[(_kind(a), op)]
    rc = getattr(lib, name)(w.ctypes.data, w.ndim, _i64(w.shape), _i64(k), mon, _i64(x),
                            res.ctypes.data)
    if rc != 0:
        raise ValueError("%s failed with status %d" % (name, rc))
    return res[0]


def included_at(a, k, op, x):
    """The included sum at one coordinate x, from the definition."""
    return _call_at("orc_included_at", a, k, op, x)


def excluded_at(a, k, op, x):
    """The excluded sum at one coordinate x, from the definition."""
    return _call_at("orc_excluded_at", a, k, op, x)


def sat_included(a, k):
    """Included sums by the summed-area table (Sec. 1); integer + only."""
    lib = _load()
    w = np.ascontiguousarray(a, dtype=np.int64)
    out = np.empty_like(w)
    rc = lib.orc_sat_included(w.ctypes.data, out.ctypes.data, w.ndim, _i64(w.shape), _i64(k))
    if rc != 0:
        raise ValueError("orc_sat_included failed with status %d" % rc)
    return out


def bdbsc(a, k):
    """Weak excluded sums by BDBS complement (Sec. 1); integer + only."""
    lib = _load()
    w = np.ascontiguousarray(a, dtype=np.int64)
    out = np.empty_like(w)
    rc = lib.orc_bdbsc(w.ctypes.data, out.ctypes.data, w.ndim, _i64(w.shape), _i64(k))
    if rc != 0:
        raise ValueError("orc_bdbsc failed with status %d" % rc)
    return out


def reset_ops():
    """Resets the counter of operator applications."""
    _load().orc_reset_ops()


def get_ops():
    """Number of operator applications since the last reset."""
    return int(_load().orc_get_ops())


def corner_threshold_hi(d, dim, mask):
    """1 if region ``mask`` of the corners partition uses x+k in ``dim``."""
    return int(_load().orc_corner_threshold_hi(d, dim, mask))


def identity(kind, op):
    """The identity element e of the oracle's monoid for ``kind`` in {int, float}."""
    if op == "add":
        return np.int64(0) if kind == "int" else np.float64(0.0)
    return np.int64(np.iinfo(np.int64).min) if kind == "int" else np.float64(-np.inf)
