// monoid.cuh -- element types and operators of the GPU path.
//
// The paper states every algorithm over a monoid (S, (+), e) (Sec. 1);
// box-complement also regroups operands across regions, so the operator must
// be commutative as well.  This library provides + and max:
//
//   dtype  op   input      accumulate             big intermediates  carries   output
//   I32    +    int32      int32, wraps mod 2^32  int32              int32     int32
//   I64    +    int64      int64, wraps mod 2^64  int64              int64     int64
//   F32    +    fp32       fp32 pair (hi, lo)     fp32 (hi+lo)       fp32 pair fp32
//   BF16   +    bf16 bits  fp32 pair (hi, lo)     fp32 (hi+lo)       fp32 pair fp32
//   *      max  as above   the input's value type, identity INT_MIN / -inf
//
// Each monoid has two accumulators: acc_t for long reductions (carries) and
// loc_t for short local scans over at most a few dozen elements (windows of
// BDBS, the in-segment part of the dimension-1 step).  They differ only for
// floating-point +, where loc_t is plain fp32: a short scan of values of
// similar size adds an error far below the compensated carries it is added
// to.
//
// Integer + and max are exact under any regrouping, so integer and max
// results are bit-exact.  Floating-point + carries its running sums as an
// unevaluated pair hi + lo (Knuth's TwoSum), so long reductions -- carries
// along dimension 1, column totals, the recursion's totals -- lose almost
// nothing to rounding; the short window sums of the big intermediate tensor
// are rounded to fp32 once each.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace exsum {

enum { OP_ADD = 0, OP_MAX = 1 };

// A compensated fp32 value: the exact value is hi + lo.
struct __align__(8) f2 {
    float hi, lo;
};

// Double-float addition: TwoSum of the high parts (Knuth), the low parts
// folded into the error term, then a FastTwoSum renormalisation.  Written
// with explicit round-to-nearest intrinsics so that the compiler cannot
// contract or regroup it.
__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bv = __fsub_rn(s, a.hi);
    const float av = __fsub_rn(s, bv);
    const float err = __fadd_rn(__fsub_rn(a.hi, av), __fsub_rn(b.hi, bv));
    const float lo = __fadd_rn(err, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, lo);
    f2 r;
    r.hi = hi;
    r.lo = __fsub_rn(lo, __fsub_rn(hi, s));
    return r;
}

__device__ __forceinline__ float bf16_bits_to_float(uint16_t b)
{
    return __uint_as_float(((uint32_t)b) << 16);
}

// --- integer + (wrapping) -----------------------------------------------------
template <class T, class U>
struct MonIntAdd {
    using in_t = T;
    using out_t = T;
    using acc_t = T;
    using car_t = T;
    using loc_t = T;
    static constexpr bool compensated = false;
    __device__ __forceinline__ static acc_t id() { return (T)0; }
    __device__ __forceinline__ static acc_t op(acc_t a, acc_t b) { return (T)((U)a + (U)b); }
    __device__ __forceinline__ static acc_t get(T v) { return v; }
    template <class S>
    __device__ __forceinline__ static S put(acc_t a) { return a; }
    __device__ __forceinline__ static loc_t lid() { return id(); }
    __device__ __forceinline__ static loc_t lop(loc_t a, loc_t b) { return op(a, b); }
    __device__ __forceinline__ static loc_t lget(T v) { return v; }
    __device__ __forceinline__ static acc_t widen(loc_t v) { return v; }
    template <class S>
    __device__ __forceinline__ static S lput(loc_t a) { return a; }
};

// --- integer max ---------------------------------------------------------------
template <class T, long long MINV>
struct MonIntMax {
    using in_t = T;
    using out_t = T;
    using acc_t = T;
    using car_t = T;
    using loc_t = T;
    static constexpr bool compensated = false;
    __device__ __forceinline__ static acc_t id() { return (T)MINV; }
    __device__ __forceinline__ static acc_t op(acc_t a, acc_t b) { return a > b ? a : b; }
    __device__ __forceinline__ static acc_t get(T v) { return v; }
    template <class S>
    __device__ __forceinline__ static S put(acc_t a) { return a; }
    __device__ __forceinline__ static loc_t lid() { return id(); }
    __device__ __forceinline__ static loc_t lop(loc_t a, loc_t b) { return op(a, b); }
    __device__ __forceinline__ static loc_t lget(T v) { return v; }
    __device__ __forceinline__ static acc_t widen(loc_t v) { return v; }
    template <class S>
    __device__ __forceinline__ static S lput(loc_t a) { return a; }
};

// --- floating-point + with compensated accumulation -----------------------------
template <class IN>
struct MonFloatAdd {
    using in_t = IN;        // float or uint16_t (bf16 bits)
    using out_t = float;
    using acc_t = f2;
    using car_t = f2;
    using loc_t = float;
    static constexpr bool compensated = true;
    __device__ __forceinline__ static acc_t id() { f2 z; z.hi = 0.f; z.lo = 0.f; return z; }
    __device__ __forceinline__ static acc_t op(acc_t a, acc_t b) { return f2_add(a, b); }
    // Local (short-range) arithmetic: plain fp32.
    __device__ __forceinline__ static loc_t lid() { return 0.f; }
    __device__ __forceinline__ static loc_t lop(loc_t a, loc_t b) { return __fadd_rn(a, b); }
    __device__ __forceinline__ static loc_t lget(float v) { return v; }
    __device__ __forceinline__ static loc_t lget(uint16_t v) { return bf16_bits_to_float(v); }
    __device__ __forceinline__ static loc_t lget(f2 v) { return __fadd_rn(v.hi, v.lo); }
    __device__ __forceinline__ static acc_t widen(loc_t v) { f2 r; r.hi = v; r.lo = 0.f; return r; }
    template <class S>
    __device__ __forceinline__ static S lput(loc_t a);
    __device__ __forceinline__ static acc_t get(float v) { f2 r; r.hi = v; r.lo = 0.f; return r; }
    __device__ __forceinline__ static acc_t get(uint16_t v) { return get(bf16_bits_to_float(v)); }
    __device__ __forceinline__ static acc_t get(f2 v) { return v; }
    template <class S>
    __device__ __forceinline__ static S put(acc_t a);
};
template <>
template <>
__device__ __forceinline__ float MonFloatAdd<float>::put<float>(f2 a) { return __fadd_rn(a.hi, a.lo); }
template <>
template <>
__device__ __forceinline__ float MonFloatAdd<float>::lput<float>(float a) { return a; }
template <>
template <>
__device__ __forceinline__ f2 MonFloatAdd<float>::lput<f2>(float a) { f2 r; r.hi = a; r.lo = 0.f; return r; }
template <>
template <>
__device__ __forceinline__ float MonFloatAdd<uint16_t>::lput<float>(float a) { return a; }
template <>
template <>
__device__ __forceinline__ f2 MonFloatAdd<uint16_t>::lput<f2>(float a) { f2 r; r.hi = a; r.lo = 0.f; return r; }
template <>
template <>
__device__ __forceinline__ f2 MonFloatAdd<float>::put<f2>(f2 a) { return a; }
template <>
template <>
__device__ __forceinline__ float MonFloatAdd<uint16_t>::put<float>(f2 a) { return __fadd_rn(a.hi, a.lo); }
template <>
template <>
__device__ __forceinline__ f2 MonFloatAdd<uint16_t>::put<f2>(f2 a) { return a; }

// --- floating-point max -----------------------------------------------------------
template <class IN>
struct MonFloatMax {
    using in_t = IN;
    using out_t = float;
    using acc_t = float;
    using car_t = float;
    using loc_t = float;
    static constexpr bool compensated = false;
    __device__ __forceinline__ static acc_t id() { return -__int_as_float(0x7f800000); }
    __device__ __forceinline__ static acc_t op(acc_t a, acc_t b) { return fmaxf(a, b); }
    __device__ __forceinline__ static acc_t get(float v) { return v; }
    __device__ __forceinline__ static acc_t get(uint16_t v) { return bf16_bits_to_float(v); }
    template <class S>
    __device__ __forceinline__ static S put(acc_t a) { return a; }
    __device__ __forceinline__ static loc_t lid() { return id(); }
    __device__ __forceinline__ static loc_t lop(loc_t a, loc_t b) { return op(a, b); }
    template <class V>
    __device__ __forceinline__ static loc_t lget(V v) { return get(v); }
    __device__ __forceinline__ static acc_t widen(loc_t v) { return v; }
    template <class S>
    __device__ __forceinline__ static S lput(loc_t a) { return a; }
};

using M_I32_ADD = MonIntAdd<int32_t, uint32_t>;
using M_I64_ADD = MonIntAdd<int64_t, uint64_t>;
using M_I32_MAX = MonIntMax<int32_t, (long long)INT32_MIN>;
using M_I64_MAX = MonIntMax<int64_t, (long long)INT64_MIN>;
using M_F32_ADD = MonFloatAdd<float>;
using M_F32_MAX = MonFloatMax<float>;
using M_BF16_ADD = MonFloatAdd<uint16_t>;
using M_BF16_MAX = MonFloatMax<uint16_t>;

// --- compensated local arithmetic ------------------------------------------------------
// The same monoid with the long (compensated) accumulator used for the short
// scans too.  Box-complement uses it for everything computed on carries: the
// carries' included sums and the lower-dimensional recursion, whose values
// are as large as the final sums.
template <class M>
struct MonComp {
    using in_t = typename M::in_t;
    using out_t = typename M::out_t;
    using acc_t = typename M::acc_t;
    using car_t = typename M::car_t;
    using loc_t = acc_t;
    static constexpr bool compensated = false;   // already the compensated form
    __device__ __forceinline__ static acc_t id() { return M::id(); }
    __device__ __forceinline__ static acc_t op(acc_t a, acc_t b) { return M::op(a, b); }
    template <class V>
    __device__ __forceinline__ static acc_t get(V v) { return M::get(v); }
    template <class S>
    __device__ __forceinline__ static S put(acc_t a) { return M::template put<S>(a); }
    __device__ __forceinline__ static loc_t lid() { return M::id(); }
    __device__ __forceinline__ static loc_t lop(loc_t a, loc_t b) { return M::op(a, b); }
    template <class V>
    __device__ __forceinline__ static loc_t lget(V v) { return M::get(v); }
    __device__ __forceinline__ static acc_t widen(loc_t v) { return v; }
    template <class S>
    __device__ __forceinline__ static S lput(loc_t a) { return M::template put<S>(a); }
};

// --- L2 eviction-priority hints ---------------------------------------------------------
// Passes hand their output to the next pass through global memory.  When the
// tensor fits in L2 (129 MB on GB300), writing such intermediates with the
// evict_last priority and reading inputs used once with evict_first lets the
// next pass find them in L2 instead of HBM.  Hints only: results do not
// depend on them.
__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}

template <class T>
__device__ __forceinline__ T ld_hint(const T *p, uint64_t pol)
{
    static_assert(sizeof(T) == 2 || sizeof(T) == 4 || sizeof(T) == 8, "element size");
    T v;
    if constexpr (sizeof(T) == 4) {
        uint32_t r;
        asm volatile("ld.global.L2::cache_hint.b32 %0, [%1], %2;\n" : "=r"(r) : "l"(p), "l"(pol));
        memcpy(&v, &r, 4);
    } else if constexpr (sizeof(T) == 8) {
        uint64_t r;
        asm volatile("ld.global.L2::cache_hint.b64 %0, [%1], %2;\n" : "=l"(r) : "l"(p), "l"(pol));
        memcpy(&v, &r, 8);
    } else {
        uint16_t r;
        asm volatile("ld.global.L2::cache_hint.b16 %0, [%1], %2;\n" : "=h"(r) : "l"(p), "l"(pol));
        memcpy(&v, &r, 2);
    }
    return v;
}

template <class T>
__device__ __forceinline__ void st_hint(T *p, T v, uint64_t pol)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "element size");
    if constexpr (sizeof(T) == 4) {
        uint32_t r;
        memcpy(&r, &v, 4);
        asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;\n" ::"l"(p), "r"(r), "l"(pol) : "memory");
    } else {
        uint64_t r;
        memcpy(&r, &v, 8);
        asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;\n" ::"l"(p), "l"(r), "l"(pol) : "memory");
    }
}

__device__ __forceinline__ uint4 ld_hint_v4(const void *p, uint64_t pol)
{
    uint4 r;
    asm volatile("ld.global.L2::cache_hint.v4.b32 {%0, %1, %2, %3}, [%4], %5;\n"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint2 ld_hint_v2(const void *p, uint64_t pol)
{
    uint2 r;
    asm volatile("ld.global.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;\n"
                 : "=r"(r.x), "=r"(r.y)
                 : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ void st_hint_v4(void *p, uint4 r, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;\n" ::"l"(p), "r"(r.x),
                 "r"(r.y), "r"(r.z), "r"(r.w), "l"(pol)
                 : "memory");
}

// --- programmatic dependent launch -------------------------------------------------------
// A kernel launched with programmatic stream serialization may start while
// the kernel before it on the stream is still running.  pdl_wait() returns
// once that kernel has completed and its memory is visible; every read of
// its results (and every write to memory it reads) comes after it.
// pdl_trigger() lets the next such kernel launch before this one ends.
// Both are no-ops for a kernel launched normally.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// --- warp shuffles of accumulator values ---------------------------------------------
__device__ __forceinline__ int32_t shfl_up(int32_t v, int dl) { return __shfl_up_sync(0xffffffffu, v, dl); }
__device__ __forceinline__ int64_t shfl_up(int64_t v, int dl)
{
    return (int64_t)__shfl_up_sync(0xffffffffu, (long long)v, dl);
}
__device__ __forceinline__ float shfl_up(float v, int dl) { return __shfl_up_sync(0xffffffffu, v, dl); }
__device__ __forceinline__ f2 shfl_up(f2 v, int dl)
{
    f2 r;
    r.hi = __shfl_up_sync(0xffffffffu, v.hi, dl);
    r.lo = __shfl_up_sync(0xffffffffu, v.lo, dl);
    return r;
}
__device__ __forceinline__ int32_t shfl_down(int32_t v, int dl)
{
    return __shfl_down_sync(0xffffffffu, v, dl);
}
__device__ __forceinline__ int64_t shfl_down(int64_t v, int dl)
{
    return (int64_t)__shfl_down_sync(0xffffffffu, (long long)v, dl);
}
__device__ __forceinline__ float shfl_down(float v, int dl) { return __shfl_down_sync(0xffffffffu, v, dl); }
__device__ __forceinline__ f2 shfl_down(f2 v, int dl)
{
    f2 r;
    r.hi = __shfl_down_sync(0xffffffffu, v.hi, dl);
    r.lo = __shfl_down_sync(0xffffffffu, v.lo, dl);
    return r;
}

// The value of lane `src`.
__device__ __forceinline__ int32_t shfl_idx(int32_t v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ int64_t shfl_idx(int64_t v, int src)
{
    return (int64_t)__shfl_sync(0xffffffffu, (long long)v, src);
}
__device__ __forceinline__ float shfl_idx(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ f2 shfl_idx(f2 v, int src)
{
    f2 r;
    r.hi = __shfl_sync(0xffffffffu, v.hi, src);
    r.lo = __shfl_sync(0xffffffffu, v.lo, src);
    return r;
}

// Segmented variants: lanes exchange only within aligned groups of `w` lanes.
__device__ __forceinline__ int32_t shfl_up_w(int32_t v, int dl, int w) { return __shfl_up_sync(0xffffffffu, v, dl, w); }
__device__ __forceinline__ int64_t shfl_up_w(int64_t v, int dl, int w)
{
    return (int64_t)__shfl_up_sync(0xffffffffu, (long long)v, dl, w);
}
__device__ __forceinline__ float shfl_up_w(float v, int dl, int w) { return __shfl_up_sync(0xffffffffu, v, dl, w); }
__device__ __forceinline__ f2 shfl_up_w(f2 v, int dl, int w)
{
    f2 r;
    r.hi = __shfl_up_sync(0xffffffffu, v.hi, dl, w);
    r.lo = __shfl_up_sync(0xffffffffu, v.lo, dl, w);
    return r;
}
__device__ __forceinline__ int32_t shfl_down_w(int32_t v, int dl, int w) { return __shfl_down_sync(0xffffffffu, v, dl, w); }
__device__ __forceinline__ int64_t shfl_down_w(int64_t v, int dl, int w)
{
    return (int64_t)__shfl_down_sync(0xffffffffu, (long long)v, dl, w);
}
__device__ __forceinline__ float shfl_down_w(float v, int dl, int w) { return __shfl_down_sync(0xffffffffu, v, dl, w); }
__device__ __forceinline__ f2 shfl_down_w(f2 v, int dl, int w)
{
    f2 r;
    r.hi = __shfl_down_sync(0xffffffffu, v.hi, dl, w);
    r.lo = __shfl_down_sync(0xffffffffu, v.lo, dl, w);
    return r;
}
__device__ __forceinline__ int32_t shfl_xor(int32_t v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ int64_t shfl_xor(int64_t v, int m)
{
    return (int64_t)__shfl_xor_sync(0xffffffffu, (long long)v, m);
}
__device__ __forceinline__ float shfl_xor(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ f2 shfl_xor(f2 v, int m)
{
    f2 r;
    r.hi = __shfl_xor_sync(0xffffffffu, v.hi, m);
    r.lo = __shfl_xor_sync(0xffffffffu, v.lo, m);
    return r;
}

}  // namespace exsum
