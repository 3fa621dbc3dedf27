"""Seeded synthetic inputs and named workloads.

This module only draws numbers and names shapes; it performs none of the
included/excluded-sum arithmetic.  Both the CUDA path's tests and the CPU
oracle's tests take their inputs from here, so the two sides see identical
bits.  Generation uses numpy's counter-based Philox generator keyed by the
seed, which gives the same stream on x86 and Arm hosts.

The paper evaluates on synthetic tensors only (3-D with N = 88^3 and k = 4,
and a dimension sweep with N in [2^21, 2^27] and k_i = 8; Sec. 6); the
workloads below have the same structure: dense row-major tensors of uniform
random values, cubic or hypercubic shapes, equal box sides per dimension.
"""

import numpy as np

DTYPES = ("i32", "i64", "f32", "bf16")
OPS = ("add", "max")


def _rng(seed):
    return np.random.Generator(np.random.Philox(key=int(seed) & ((1 << 64) - 1)))


def uniform_int(shape, lo, hi, seed, dtype=np.int64):
    """Integers uniform on the closed range [lo, hi]."""
    return _rng(seed).integers(lo, hi, size=shape, endpoint=True, dtype=np.int64).astype(dtype)


def uniform_f32(shape, seed, lo=-1.0, hi=1.0):
    """float32 values uniform on [lo, hi): 24-bit mantissa draws, exact in fp32."""
    u = _rng(seed).integers(0, 1 << 24, size=shape, dtype=np.int64)
    scale = (hi - lo) / float(1 << 24)
    return (lo + u.astype(np.float64) * scale).astype(np.float32)


def f32_to_bf16_bits(x):
    """Rounds float32 values to bfloat16 (nearest, ties to even); returns uint16 bits."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounding = 0x7FFF + ((b >> 16) & 1)
    return ((b + rounding) >> 16).astype(np.uint16)


def bf16_bits_to_f32(bits):
    """Exact float32 values of bfloat16 bit patterns."""
    return (np.ascontiguousarray(bits, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def make_input(shape, dtype, seed, int_lo=-1000, int_hi=1000):
    """A tensor for the named dtype.

    Returns (device_array, values): ``device_array`` holds the bits the CUDA
    library reads (bf16 as uint16), ``values`` the same numbers in a numpy
    dtype the oracle accepts (int32/int64/float32).
    """
    if dtype == "i64":
        a = uniform_int(shape, int_lo, int_hi, seed, np.int64)
        return a, a
    if dtype == "i32":
        a = uniform_int(shape, int_lo, int_hi, seed, np.int32)
        return a, a
    if dtype == "f32":
        a = uniform_f32(shape, seed)
        return a, a
    if dtype == "bf16":
        bits = f32_to_bf16_bits(uniform_f32(shape, seed))
        return bits, bf16_bits_to_f32(bits)
    raise ValueError("unknown dtype %r" % (dtype,))


# Named workloads: (name, shape, k, dtype, op, value range for integers).
WORKLOADS = {
    # d = 2, 256 x 256 int64 in [-1000, 1000], k = (16, 16), +
    "d2_256x256_i64_add_k16": dict(shape=(256, 256), k=(16, 16), dtype="i64", op="add",
                                   int_range=(-1000, 1000), seed=1),
    # d = 3, 256^3 float32 uniform [-1, 1), k = (8, 8, 8), +
    "d3_256cube_f32_add_k8": dict(shape=(256, 256, 256), k=(8, 8, 8), dtype="f32", op="add",
                                  seed=2),
    # d = 3, 256^3 int32 uniform [0, 2^20), k = (8, 8, 8), max
    "d3_256cube_i32_max_k8": dict(shape=(256, 256, 256), k=(8, 8, 8), dtype="i32", op="max",
                                  int_range=(0, (1 << 20) - 1), seed=3),
    # dimension sweep at about 2^25 elements, float32 and bfloat16, +
    "d1_2p25_f32_add_k64": dict(shape=(1 << 25,), k=(64,), dtype="f32", op="add", seed=4),
    "d1_2p25_bf16_add_k64": dict(shape=(1 << 25,), k=(64,), dtype="bf16", op="add", seed=5),
    "d4_76p4_f32_add_k4": dict(shape=(76, 76, 76, 76), k=(4, 4, 4, 4), dtype="f32", op="add",
                               seed=6),
    "d4_76p4_bf16_add_k4": dict(shape=(76, 76, 76, 76), k=(4, 4, 4, 4), dtype="bf16", op="add",
                                seed=7),
    "d5_32p5_f32_add_k4": dict(shape=(32,) * 5, k=(4,) * 5, dtype="f32", op="add", seed=8),
    "d5_32p5_bf16_add_k4": dict(shape=(32,) * 5, k=(4,) * 5, dtype="bf16", op="add", seed=9),
    # 512^3 float32: larger than L2, for HBM-true per-pass figures
    "d3_512cube_f32_add_k8": dict(shape=(512, 512, 512), k=(8, 8, 8), dtype="f32", op="add",
                                  seed=10),
    # boxes over 32 along the strided dimensions (suffixes kept in the output)
    "d3_256cube_f32_add_k64": dict(shape=(256, 256, 256), k=(64, 64, 64), dtype="f32", op="add", seed=12),
    # rows longer than one warp scans: the row schedule's one-block-per-row final pass
    "d2_4096x2048_f32_add_k8": dict(shape=(4096, 2048), k=(8, 8), dtype="f32", op="add", seed=13),
    # rows whose length (301) is not a multiple of 4, larger than L2: the
    # realigned bulk final pass
    "d3_256x512x301_f32_add_k484": dict(shape=(256, 512, 301), k=(4, 8, 4), dtype="f32", op="add",
                                        seed=11),
}


def workload_input(name):
    """(device_array, values, spec) for a named workload."""
    spec = WORKLOADS[name]
    lo, hi = spec.get("int_range", (-1000, 1000))
    dev, vals = make_input(spec["shape"], spec["dtype"], spec["seed"], lo, hi)
    return dev, vals, spec


def batched_shapes(count, seed, side_lo=32, side_hi=512, k_lo=2, k_hi=32, cap=1 << 24):
    """Shapes and boxes for a batch of uneven tensors.

    d uniform in {2, 3}, every side uniform in [side_lo, side_hi], every k_i
    uniform in [k_lo, min(k_hi, n_i)]; a shape above ``cap`` elements is drawn
    again (rejection sampling).
    """
    rng = _rng(seed)
    out = []
    while len(out) < count:
        d = int(rng.integers(2, 4))
        shape = tuple(int(v) for v in rng.integers(side_lo, side_hi, size=d, endpoint=True))
        if int(np.prod(shape)) > cap:
            continue
        k = tuple(int(rng.integers(k_lo, min(k_hi, n), endpoint=True)) for n in shape)
        out.append((shape, k))
    return out
