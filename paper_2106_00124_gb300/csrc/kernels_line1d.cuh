// kernels_line1d.cuh -- excluded sums of one long contiguous line (d = 1),
// with 16-byte loads and stores.
//
// For d = 1 the excluded sum is the exclusive prefix before x plus the
// suffix from x + k (Sec. 4 with one dimension; the prefix and suffix steps
// of Sec. 5).  The line is cut into segments of NT * V elements, one block
// each; thread t owns the strip of V consecutive outputs from s0 = segment
// start + t * V.  Its output x needs
//   the prefix of the line before x       = Q-part before the segment
//                                           (+) prefix of the segment's strips before t
//                                           (+) the strip's own elements before x,
//   the suffix of the line from x + k     = the same over the "target window",
//                                           the segment shifted by k, whose
//                                           strips line up with the outputs',
// so the exclusive prefix and the target-window suffix of an output sit in
// the same thread and register slot.  The carries Q (everything before the
// segment and everything past its target window) come from the segment
// totals (k_reduce_line, k_carry_line2), and the combination of a
// segment's warps, in compensated arithmetic; a strip (V elements) and a
// warp's strips (at most 32 V) are scanned in the local type.
#pragma once

#include "kernels_fold.cuh"
#include "kernels_rows.cuh"

namespace exsum {

// Exclusive prefix of `a` and exclusive suffix of `b` across the threads of
// a block, in a fixed order: inclusive scans within each warp (in the long,
// compensated accumulator when COMP, else in the local type), then the warp
// totals combined in the long accumulator, where partial sums grow large.
template <class M, int NT, bool COMP>
__device__ __forceinline__ void block_exscan_pair(typename M::loc_t a, typename M::loc_t b,
                                                  typename M::acc_t &pre, typename M::acc_t &suf)
{
    using Lt = typename M::loc_t;
    using A = typename M::acc_t;
    using W = typename std::conditional<COMP, A, Lt>::type;
    constexpr int NW = NT / 32;
    __shared__ A wp[NW], ws[NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto wop = [](W u, W v) -> W {
        if constexpr (COMP)
            return M::op(u, v);
        else
            return M::lop(u, v);
    };
    auto wid = []() -> W {
        if constexpr (COMP)
            return M::id();
        else
            return M::lid();
    };
    auto toA = [](W u) -> A {
        if constexpr (COMP)
            return u;
        else
            return M::widen(u);
    };
    W ia, ib;
    if constexpr (COMP) {
        ia = M::widen(a);
        ib = M::widen(b);
    } else {
        ia = a;
        ib = b;
    }
#pragma unroll
    for (int dl = 1; dl < 32; dl <<= 1) {
        const W o = shfl_up(ia, dl);
        const W q = shfl_down(ib, dl);
        if (lane >= dl) ia = wop(o, ia);
        if (lane + dl < 32) ib = wop(ib, q);
    }
    if (lane == 31) wp[warp] = toA(ia);
    if (lane == 0) ws[warp] = toA(ib);
    __syncthreads();
    A x = M::id(), y = M::id();
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        if (w < warp) x = M::op(x, wp[w]);
        if (w > warp) y = M::op(y, ws[w]);
    }
    W ea = shfl_up(ia, 1), eb = shfl_down(ib, 1);
    if (lane == 0) ea = wid();
    if (lane == 31) eb = wid();
    pre = M::op(x, toA(ea));
    suf = M::op(toA(eb), y);
    __syncthreads();
}

// V consecutive elements from p into the local type: 16-byte loads when
// `vec` (p 16-byte aligned for 4-byte inputs, 8-byte for bf16), else
// element loads; positions at or past `valid` hold the identity.
template <class M, class SIn, int V>
__device__ __forceinline__ void load_strip(const SIn *p, bool vec, int valid, typename M::loc_t *v, uint64_t pol)
{
    if (vec && valid >= V) {
#pragma unroll
        for (int i = 0; i < V / 4; ++i) load4<M>(p + 4 * i, true, 4, v + 4 * i, pol);
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) v[j] = j < valid ? M::lget(ld_hint(p + j, pol)) : M::lid();
    }
}

// Segment totals of the line: R[s] over the segment, Rt[s] over the segment
// from offset r on (the part a target window shifted by k covers).
template <class M, class SIn, int NT, int V>
__global__ void __launch_bounds__(NT)
k_reduce_line(const SIn *__restrict__ X, typename M::car_t *__restrict__ R,
              typename M::car_t *__restrict__ Rt, int64_t n1, int64_t r, int vec)
{
    using Lt = typename M::loc_t;
    using A = typename M::acc_t;
    using C = typename M::car_t;
    constexpr int NW = NT / 32;
    __shared__ A wh[NW], wt[NW];
    const int64_t base = (int64_t)blockIdx.x * (NT * V);
    const int64_t s0 = base + (int64_t)threadIdx.x * V;
    const uint64_t pol = l2_policy_evict_first();
    Lt v[V];
    const int64_t left = n1 - s0;
    load_strip<M, SIn, V>(X + (s0 < n1 ? s0 : 0), vec != 0, left <= 0 ? 0 : (left > V ? V : (int)left), v, pol);
    Lt head = M::lid(), tail = M::lid();
    const int64_t off = s0 - base;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        if (off + j < r)
            head = M::lop(head, v[j]);
        else
            tail = M::lop(tail, v[j]);
    }
    // strip sums (V elements) in the local type, everything wider compensated
    A hw = M::widen(head), tw = M::widen(tail);
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        hw = M::op(hw, shfl_xor(hw, m));
        tw = M::op(tw, shfl_xor(tw, m));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        wh[warp] = hw;
        wt[warp] = tw;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        A h = M::id(), t = M::id();
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            h = M::op(h, wh[w]);
            t = M::op(t, wt[w]);
        }
        R[blockIdx.x] = M::template put<C>(M::op(h, t));
        if (Rt) Rt[blockIdx.x] = M::template put<C>(t);
    }
}

// Carries of the S segments of one line, one block per NT segments:
//   Q[s] = (+)_{s' < s} R[s']  (+)  Rt[q] (+) (+)_{s' > q} R[s'],   q = s + qoff
// (everything before the segment and everything past its target window).
// Block b reduces, over all segment totals, those before its range
// (lo = NT b) and those past hi + qoff (hi = lo + NT), in a fixed order; then thread t
// (segment s = lo + t) takes the exclusive prefix of its range and the
// exclusive suffix of the shifted range [lo + qoff, hi + qoff):
//   Q[s] = pre(lo) (+) (+)_{lo <= s' < s} R[s']
//          (+) Rt[q] (+) (+)_{q < s' < hi + qoff} R[s'] (+) suf(hi + qoff),  q = s + qoff.
// Every block reads all S totals once (a few MB from L2 for millions of
// elements), and nothing depends on the order in which blocks run.
template <class M, int NT>
__global__ void __launch_bounds__(NT)
k_carry_line2(const typename M::car_t *__restrict__ R, const typename M::car_t *__restrict__ Rt,
              typename M::car_t *__restrict__ Q, int64_t S, int64_t qoff)
{
    using A = typename M::acc_t;
    using C = typename M::car_t;
    __shared__ A red[33];
    const int t = threadIdx.x;
    const int64_t lo = (int64_t)blockIdx.x * NT, hi = lo + NT < S ? lo + NT : S;
    const int64_t sh = hi + qoff;   // suffix part starts here
    A pa = M::id(), sa = M::id();
    for (int64_t b0 = 0; b0 < S; b0 += 8 * NT) {
        C v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t s = b0 + u * NT + t;
            v[u] = s < S ? R[s] : M::template put<C>(M::id());
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t s = b0 + u * NT + t;
            if (s < lo) pa = M::op(pa, M::get(v[u]));
            if (s >= sh && s < S) sa = M::op(sa, M::get(v[u]));
        }
    }
    pa = block_reduce<M>(pa, red);
    sa = block_reduce<M>(sa, red);
    const int64_t s = lo + t;
    const int64_t q = s + qoff;
    const A r = s < hi ? M::get(R[s]) : M::id();
    const A rq = q < sh && q < S ? M::get(R[q]) : M::id();
    A pre, unused1, unused2, suf;
    block_exscan_both<M, NT>(r, pre, unused1);
    block_exscan_both<M, NT>(rq, unused2, suf);
    if (s < hi) {
        A w = M::id();
        if (q < S) w = M::op(M::get(Rt[q]), M::op(suf, sa));
        Q[s] = M::template put<C>(M::op(M::op(pa, pre), w));
    }
}

// Outputs of one segment (see the file comment).  Q null: a single segment.
template <class M, class SIn, class SOut, int NT, int V>
__global__ void __launch_bounds__(NT)
k_exline_line(const SIn *__restrict__ H, const typename M::car_t *__restrict__ Q,
              SOut *__restrict__ out, int64_t n1, int64_t k1, int vec_in, int vec_tgt, int vec_out)
{
    using Lt = typename M::loc_t;
    using A = typename M::acc_t;
    const int64_t s0 = (int64_t)blockIdx.x * (NT * V) + (int64_t)threadIdx.x * V;
    const uint64_t pol_in = l2_policy_evict_first();
    const uint64_t pol_out = l2_policy_evict_first();
    Lt p[V], t[V];
    {
        const int64_t left = n1 - s0;
        load_strip<M, SIn, V>(H + (s0 < n1 ? s0 : 0), vec_in != 0, left <= 0 ? 0 : (left > V ? V : (int)left), p,
                              pol_in);
        const int64_t y0 = s0 + k1;
        const int64_t lt = n1 - y0;
        load_strip<M, SIn, V>(H + (y0 < n1 ? y0 : 0), vec_tgt != 0, lt <= 0 ? 0 : (lt > V ? V : (int)lt), t,
                              pol_in);
    }
    // exclusive prefix within the strip (in place) and its total
    Lt ptot = M::lid();
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const Lt x = p[j];
        p[j] = ptot;
        ptot = M::lop(ptot, x);
    }
    // inclusive suffix within the target strip (in place) and its total
#pragma unroll
    for (int j = V - 2; j >= 0; --j) t[j] = M::lop(t[j], t[j + 1]);
    const Lt stot = t[0];
    // scans across the strips: within a warp in the local type, across
    // warps in the long (compensated) accumulator -- the partial sums of a
    // segment can be far larger than the results they cancel to
    A bp, bs;
    block_exscan_pair<M, NT, true>(ptot, stot, bp, bs);
    A base = Q ? M::get(Q[blockIdx.x]) : M::id();
    base = M::op(base, M::op(bp, bs));
    SOut res[V];
#pragma unroll
    for (int j = 0; j < V; ++j) res[j] = finish<M, SOut>(base, M::lop(p[j], t[j]));
    const int64_t left = n1 - s0;
    if (vec_out && left >= V && sizeof(SOut) == 4) {
#pragma unroll
        for (int i = 0; i < V / 4; ++i) {
            uint4 w;
            memcpy(&w, res + 4 * i, 16);
            st_hint_v4(out + s0 + 4 * i, w, pol_out);
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j)
            if (j < left) st_hint(out + s0 + j, res[j], pol_out);
    }
}

}  // namespace exsum
