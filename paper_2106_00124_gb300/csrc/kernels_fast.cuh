// kernels_fast.cuh -- register-resident kernels for the common box sizes.
//
// BDBS-1D (Sec. 3) needs, for the block of k elements holding x, the suffix
// of that block from x and the prefix of the next block up to x+k-1.  Here a
// thread keeps both blocks in registers: arrays of compile-time length KMAX
// hold a block of runtime length k <= KMAX, padded with the identity e, so
// every register index is a compile-time constant (no local memory) and the
// padding contributes nothing (Sec. 3 footnote: padding with e).  One thread
// walks one line chunk; per element it performs one prefix step, one suffix
// step and one combine (Combine-Along-Row).
#pragma once

#include <type_traits>

#include "kernels_lines.cuh"

namespace exsum {

// Walks outputs [r0, rend) of one line.  ld(x) returns the element at line
// position x as loc_t (e beyond the data); st(x, v) stores output x.
template <class M, int KMAX, class LD, class ST>
__device__ __forceinline__ void bdbs_walk(int k, int r0, int rend, LD ld, ST st)
{
    using Lt = typename M::loc_t;
    Lt S[KMAX], v[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) v[j] = (j < k) ? ld(r0 + j) : M::lid();
    S[KMAX - 1] = v[KMAX - 1];
#pragma unroll
    for (int j = KMAX - 2; j >= 0; --j) S[j] = M::lop(v[j], S[j + 1]);
    for (int sb = r0; sb < rend; sb += k) {
        st(sb, S[0]);
        const int nb = sb + k;
#pragma unroll
        for (int j = 0; j < KMAX; ++j) v[j] = (j < k) ? ld(nb + j) : M::lid();
        Lt p = M::lid();
#pragma unroll
        for (int j = 0; j + 1 < KMAX; ++j) {
            p = M::lop(p, v[j]);
            if (j + 1 < k && sb + 1 + j < rend) st(sb + 1 + j, M::lop(S[j + 1], p));
        }
        S[KMAX - 1] = v[KMAX - 1];
#pragma unroll
        for (int j = KMAX - 2; j >= 0; --j) S[j] = M::lop(v[j], S[j + 1]);
    }
}

// ---------------------------------------------------------------------------
// BDBS-Along-Dim along a strided dimension (view [O, n, I], I > 1): one
// thread per (outer, chunk, inner) line chunk; consecutive threads take
// consecutive inner positions, so every load and store is coalesced.
// ---------------------------------------------------------------------------
template <class M, class SIn, class SOut, int KMAX>
__device__ __forceinline__ void k_inc_strided_body(const SIn *__restrict__ in, SOut *__restrict__ out, int64_t O, int n, int64_t I,
              int k, int Lc, int nchunks, int64_t vbid, int64_t vgrid)
{
    const int64_t total = O * nchunks * I;
    const int64_t gid = (int64_t)vbid * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const int64_t i = gid % I;
    const int64_t rest = gid / I;
    const int ch = (int)(rest % nchunks);
    const int64_t o = rest / nchunks;
    const SIn *src = in + o * n * I + i;
    SOut *dst = out + o * n * I + i;
    const int r0 = ch * Lc;
    const int rend = min(r0 + Lc, n);
    const uint64_t pol_in = l2_policy_evict_first();
    const uint64_t pol_out = l2_policy_evict_last();
    bdbs_walk<M, KMAX>(
        k, r0, rend,
        [&](int x) { return x < n ? M::lget(ld_hint(src + (int64_t)x * I, pol_in)) : M::lid(); },
        [&](int x, typename M::loc_t v) {
            st_hint(dst + (int64_t)x * I, M::template lput<SOut>(v), pol_out);
        });
}

template <class M, class SIn, class SOut, int KMAX>
__global__ void __launch_bounds__(128)
k_inc_strided(const SIn *__restrict__ in, SOut *__restrict__ out, int64_t O, int n, int64_t I,
              int k, int Lc, int nchunks)
{
    k_inc_strided_body<M, SIn, SOut, KMAX>(in, out, O, n, I, k, Lc, nchunks, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// BDBS-Along-Dim along a strided dimension for boxes too long to keep a
// block in registers (k > 32).  The same blocks of k lines and the same
// combination as bdbs_walk (so the same results), with the block's
// suffixes kept in the output itself: one thread per (outer, chunk, inner)
// line chunk of whole blocks; for each block it walks the block backwards,
// writing the suffixes S[x] to out[x], then the next block forwards,
// replacing out[x] by S[x] (+) (prefix of the next block up to x + k - 1).
// The second reads of a block and of its suffixes come from this thread's
// recent accesses (L1/L2).  Four loads in flight in each walk.
// ---------------------------------------------------------------------------
template <class M, class SIn, class SOut>
__global__ void __launch_bounds__(128)
k_inc_strided_big(const SIn *__restrict__ in, SOut *__restrict__ out, int64_t O, int n, int64_t I, int k, int Lc,
                  int nchunks)
{
    using Lt = typename M::loc_t;
    const int64_t total = O * nchunks * I;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const int64_t i = gid % I;
    const int64_t rest = gid / I;
    const int ch = (int)(rest % nchunks);
    const int64_t o = rest / nchunks;
    const SIn *src = in + o * n * I + i;
    SOut *dst = out + o * n * I + i;
    const int r0 = ch * Lc;
    const int rend = min(r0 + Lc, n);
    auto ld = [&](int x) { return M::lget(src[(int64_t)x * I]); };
    for (int sb = r0; sb < rend; sb += k) {
        const int be = min(sb + k, n);
        // suffixes of the block, backwards
        Lt s = M::lid();
        int x = be - 1;
        for (; x - 3 >= sb; x -= 4) {
            Lt v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = ld(x - u);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                s = M::lop(v[u], s);
                dst[(int64_t)(x - u) * I] = M::template lput<SOut>(s);
            }
        }
        for (; x >= sb; --x) {
            s = M::lop(ld(x), s);
            dst[(int64_t)x * I] = M::template lput<SOut>(s);
        }
        // out[sb] is the block's total; later outputs add the next block's prefix
        Lt p = M::lid();
        int xo = sb + 1;
        for (; xo + 3 < be; xo += 4) {
            Lt v[4], sv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int y = xo + u + k - 1;
                v[u] = y < n ? ld(y) : M::lid();
                sv[u] = M::lget(dst[(int64_t)(xo + u) * I]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                p = M::lop(p, v[u]);
                dst[(int64_t)(xo + u) * I] = M::template lput<SOut>(M::lop(sv[u], p));
            }
        }
        for (; xo < be; ++xo) {
            const int y = xo + k - 1;
            if (y < n) p = M::lop(p, ld(y));
            dst[(int64_t)xo * I] = M::template lput<SOut>(M::lop(M::lget(dst[(int64_t)xo * I]), p));
        }
    }
}

// ---------------------------------------------------------------------------
// Rows [ya, yb) of column c of a view [*, Mc], reduced with short fp32 runs
// (at most 32 rows) combined into the long accumulator.
// ---------------------------------------------------------------------------
template <class M, class SIn>
__device__ __forceinline__ typename M::acc_t reduce_rows(const SIn *__restrict__ col, int64_t Mc,
                                                         int64_t ya, int64_t yb)
{
    typename M::acc_t acc = M::id();
    for (int64_t y0 = ya; y0 < yb; y0 += 32) {
        typename M::loc_t l = M::lid();
#pragma unroll
        for (int b = 0; b < 32; b += 8) {
            typename M::loc_t v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int64_t y = y0 + b + j;
                v[j] = y < yb ? M::lget(col[y * Mc]) : M::lid();
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) l = M::lop(l, v[j]);
        }
        acc = M::op(acc, M::widen(l));
    }
    return acc;
}

// Segment reductions along dimension 1 of a view [n1, Mc]: R[s][c] over rows
// [s*L, s*L+L) and Rt[s][c] over the same rows from offset r on.
template <class M, class SIn>
__global__ void __launch_bounds__(256)
k_reduce_seg2(const SIn *__restrict__ X, typename M::car_t *__restrict__ R,
              typename M::car_t *__restrict__ Rt, int64_t n1, int64_t Mc, int64_t L, int64_t S,
              int64_t r)
{
    using C = typename M::car_t;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= S * Mc) return;
    const int64_t c = gid % Mc, s = gid / Mc;
    const int64_t y0 = s * L;
    const int64_t y1 = min(y0 + L, n1);
    const int64_t ys = min(y0 + r, y1);
    const SIn *col = X + c;
    const typename M::acc_t head = reduce_rows<M>(col, Mc, y0, ys);
    const typename M::acc_t tail = reduce_rows<M>(col, Mc, ys, y1);
    R[gid] = M::template put<C>(M::op(head, tail));
    if (Rt) Rt[gid] = M::template put<C>(tail);
}

// ---------------------------------------------------------------------------
// Dimension-1 step (strided, Mc > 1): as k_exline, with the in-segment
// prefix and suffix in the fast local accumulator and one long-accumulator
// combine with the carry per output.
// ---------------------------------------------------------------------------
template <class M, class SIn, class SOut, int L>
__global__ void __launch_bounds__(128)
k_exline2(const SIn *__restrict__ H, const typename M::car_t *__restrict__ Q, int64_t qs,
          const typename M::car_t *__restrict__ T, SOut *__restrict__ out, int64_t n1, int64_t Mc,
          int64_t k1, int64_t S)
{
    using Lt = typename M::loc_t;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= S * Mc) return;
    const int64_t c = gid % Mc, s = gid / Mc;
    const int64_t s0 = s * L;
    const SIn *hp = H + s0 * Mc + c;
    const SIn *tp = hp + k1 * Mc;
    SOut *op_ = out + s0 * Mc + c;
    const uint64_t pol_out = l2_policy_evict_first();   // final output: streamed out
    Lt P[L];
    Lt acc = M::lid();
    typename M::acc_t q = Q ? M::get(Q[s * qs + c]) : M::id();
    if (T) q = M::op(q, M::get(T[c]));
    Lt sacc = M::lid();
    if (s0 + L + k1 <= n1) {
        // Both windows' loads issued before any use: one memory latency per thread.
        Lt tv[L];
#pragma unroll
        for (int t = 0; t < L; ++t) {
            P[t] = M::lget(hp[t * Mc]);
            tv[t] = M::lget(tp[t * Mc]);
        }
#pragma unroll
        for (int t = 0; t < L; ++t) {
            const Lt v = P[t];
            P[t] = acc;
            acc = M::lop(acc, v);
        }
#pragma unroll
        for (int t = L - 1; t >= 0; --t) {
            sacc = M::lop(tv[t], sacc);
            st_hint(op_ + t * Mc, M::template put<SOut>(M::op(q, M::widen(M::lop(P[t], sacc)))), pol_out);
        }
    } else {
#pragma unroll
        for (int t = 0; t < L; ++t) {
            P[t] = acc;
            if (s0 + t < n1) acc = M::lop(acc, M::lget(hp[t * Mc]));
        }
#pragma unroll
        for (int t = L - 1; t >= 0; --t) {
            if (s0 + k1 + t < n1) sacc = M::lop(M::lget(tp[t * Mc]), sacc);
            if (s0 + t < n1)
                op_[t * Mc] = M::template put<SOut>(M::op(q, M::widen(M::lop(P[t], sacc))));
        }
    }
}

// ---------------------------------------------------------------------------
// Dimension-1 step for a single contiguous line (Mc = 1).  One block per
// segment of NT*V outputs; thread t owns outputs s0 + t*V .. s0 + t*V + V-1.
// It scans its V prefix-window elements and the V target-window elements
// (positions +k1) locally, and the block scans the per-thread totals, so the
// exclusive prefix and the target-window suffix of an output live in the
// same thread and register slot.
// ---------------------------------------------------------------------------
template <class M, class SIn, class SOut, int NT, int V>
__global__ void __launch_bounds__(NT)
k_exline_contig(const SIn *__restrict__ H, const typename M::car_t *__restrict__ Q,
                SOut *__restrict__ out, int64_t n1, int64_t k1)
{
    using Lt = typename M::loc_t;
    using A = typename M::acc_t;
    constexpr int L = NT * V;
    const int64_t s = blockIdx.x;
    const int64_t s0 = s * L + (int64_t)threadIdx.x * V;
    Lt pre[V], suf[V];
    Lt acc = M::lid();
#pragma unroll
    for (int j = 0; j < V; ++j) {
        pre[j] = acc;
        if (s0 + j < n1) acc = M::lop(acc, M::lget(H[s0 + j]));
    }
    const Lt ptot = acc;
    Lt sacc = M::lid();
#pragma unroll
    for (int j = V - 1; j >= 0; --j) {
        const int64_t y = s0 + k1 + j;
        if (y < n1) sacc = M::lop(M::lget(H[y]), sacc);
        suf[j] = sacc;
    }
    A bp, bs_unused, tp_unused, bsuf;
    block_exscan_both<M, NT>(M::widen(ptot), bp, bs_unused);
    block_exscan_both<M, NT>(M::widen(sacc), tp_unused, bsuf);
    A q = Q ? M::get(Q[s]) : M::id();
    q = M::op(q, M::op(bp, bsuf));
#pragma unroll
    for (int j = 0; j < V; ++j)
        if (s0 + j < n1) out[s0 + j] = M::template put<SOut>(M::op(q, M::widen(M::lop(pre[j], suf[j]))));
}

// ---------------------------------------------------------------------------
// Carries from the dimension-1 segment totals of the input (view [n1, Mc],
// segments of L rows): per segment s and column c
//   Qa[s][c] = (+)_{s' < s} R[s'][c]  (+)  Rt[q][c] (+) (+)_{s' > q} R[s'][c],
// q = s + qoff (the rows before the segment and the rows past its target
// window), and the column total G[c] = (+)_s R[s][c].  Box-complement then
// applies the included sums along dimensions 2..d to Qa; by linearity of the
// reduction over boxes this equals the carries of the included tensor.
// ---------------------------------------------------------------------------
template <class M>
__global__ void __launch_bounds__(256)
k_carry_qa(const typename M::car_t *__restrict__ R, const typename M::car_t *__restrict__ Rt,
           typename M::car_t *__restrict__ Qa, typename M::car_t *__restrict__ G, int64_t Mc,
           int64_t S, int64_t qoff)
{
    using A = typename M::acc_t;
    using C = typename M::car_t;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Mc) return;
    if (S <= 16) {
        // Few segments: every load issued up front, all arithmetic in registers.
        A r[16], rt[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            r[s] = s < S ? M::get(R[s * Mc + c]) : M::id();
            rt[s] = s < S ? M::get(Rt[s * Mc + c]) : M::id();
        }
        A sr[17];
        sr[16] = M::id();
#pragma unroll
        for (int s = 15; s >= 0; --s) sr[s] = M::op(r[s], sr[s + 1]);
        G[c] = M::template put<C>(sr[0]);
        if (!Qa) return;
        A pc = M::id();
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            if (s < S) {
                const int64_t q = s + qoff;
                A w = M::id();
                if (q < S) {
#pragma unroll
                    for (int qq = 0; qq < 16; ++qq)
                        if (qq == q) w = M::op(rt[qq], sr[qq + 1]);
                }
                Qa[s * Mc + c] = M::template put<C>(M::op(pc, w));
                pc = M::op(pc, r[s]);
            }
        }
        return;
    }
    // Backward: suffix totals SR[s] parked in Qa.
    A acc = M::id();
    for (int64_t s = S - 1; s >= 0; --s) {
        acc = M::op(M::get(R[s * Mc + c]), acc);
        if (Qa) Qa[s * Mc + c] = M::template put<C>(acc);
    }
    G[c] = M::template put<C>(acc);
    if (!Qa) return;
    A pc = M::id();
    for (int64_t s = 0; s < S; ++s) {
        const int64_t q = s + qoff;
        A w = M::id();
        if (q < S) {
            w = M::get(Rt[q * Mc + c]);
            if (q + 1 < S) w = M::op(w, M::get(Qa[(q + 1) * Mc + c]));
        }
        const A rs = M::get(R[s * Mc + c]);
        Qa[s * Mc + c] = M::template put<C>(M::op(pc, w));
        pc = M::op(pc, rs);
    }
}

// Segment reductions of a single contiguous line: one block per segment of
// NT*V elements; R[s] and the tail Rt[s] from offset r.
template <class M, class SIn, int NT, int V>
__global__ void __launch_bounds__(NT)
k_reduce_seg_contig(const SIn *__restrict__ X, typename M::car_t *__restrict__ R,
                    typename M::car_t *__restrict__ Rt, int64_t n1, int64_t r)
{
    using Lt = typename M::loc_t;
    using A = typename M::acc_t;
    using C = typename M::car_t;
    constexpr int L = NT * V;
    const int64_t s = blockIdx.x;
    const int64_t base = s * L;
    const int64_t s0 = base + (int64_t)threadIdx.x * V;
    Lt head = M::lid(), tail = M::lid();
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const int64_t y = s0 + j;
        if (y < n1) {
            const Lt v = M::lget(X[y]);
            if (y - base < r)
                head = M::lop(head, v);
            else
                tail = M::lop(tail, v);
        }
    }
    A hp, hs, tpre, tsuf;
    block_exscan_both<M, NT>(M::widen(head), hp, hs);
    block_exscan_both<M, NT>(M::widen(tail), tpre, tsuf);
    if (threadIdx.x == NT - 1) {
        const A h = M::op(hp, M::widen(head));
        const A t = M::op(tpre, M::widen(tail));
        R[s] = M::template put<C>(M::op(h, t));
        if (Rt) Rt[s] = M::template put<C>(t);
    }
}

}  // namespace exsum
