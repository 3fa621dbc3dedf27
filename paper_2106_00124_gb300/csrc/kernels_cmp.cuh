// kernels_cmp.cuh -- the paper's comparison methods on the GPU: the
// summed-area table with inclusion-exclusion (SAT / SATC, Sec. 1) and the
// corners algorithm (App. A).  They are baselines for the row schedule of
// box-complement, not part of it.
//
// Both are built from inclusive scans along one dimension of a view
// [O, n, I]: the prefix of x is the (+) of the line up to and including x,
// the suffix the (+) from x to the end.
//   SAT    = the prefix along every dimension in turn; the box sum at x is
//            then the alternating sum of the SAT at the box's 2^d corners
//            (an operator with an inverse: integer +, modulo 2^w), and the
//            weak excluded sum is the total minus the box sum.
//   corners: the 2^d tensors T_b (b in {prefix, suffix}^d: the (+) over the
//            orthant below or above y in every dimension), then for every x
//            the (+) of 2^d of their entries: the orthants, shifted to x or
//            to x + k dimension by dimension, tile the complement of the box
//            exactly (no inverse needed, so max works too).
#pragma once

#include "monoid.cuh"

namespace exsum {

// Inclusive prefix (SUF: suffix) of every line along the middle dimension of
// the view [O, n, I], I > 1: one thread per line (o, i), consecutive i on
// consecutive threads, so every access is coalesced.  Eight loads in flight.
// `in` and `out` may be the same array (each element is read, by the thread
// that writes it, before it is written), as in k_scan_rows.
template <class M, class SR, class SW, bool SUF>
__global__ void __launch_bounds__(256)
k_scan_lines(const SR *in, SW *out, int64_t O, int64_t n, int64_t I)
{
    using A = typename M::acc_t;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= O * I) return;
    const int64_t o = gid / I, i = gid - o * I;
    const SR *src = in + o * n * I + i;
    SW *dst = out + o * n * I + i;
    A acc = M::id();
    for (int64_t t0 = 0; t0 < n; t0 += 8) {
        SR v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t t = t0 + u;
            if (t < n) v[u] = src[(SUF ? n - 1 - t : t) * I];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t t = t0 + u;
            if (t < n) {
                acc = M::op(acc, M::get(v[u]));
                dst[(SUF ? n - 1 - t : t) * I] = M::template put<SW>(acc);
            }
        }
    }
}

// The same along the contiguous dimension (rows of L elements): one warp
// per row, chunks of 32 elements scanned across the lanes, each chunk
// carrying the total of the ones before it.
template <class M, class SR, class SW, bool SUF>
__global__ void __launch_bounds__(256)
k_scan_rows(const SR *in, SW *out, int64_t rows, int64_t L)
{
    using A = typename M::acc_t;
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= rows) return;   // whole warps
    const SR *src = in + row * L;
    SW *dst = out + row * L;
    A carry = M::id();
    for (int64_t c0 = 0; c0 < L; c0 += 32) {
        const int64_t t = c0 + lane;
        const int64_t x = SUF ? L - 1 - t : t;
        A v = t < L ? M::get(src[x]) : M::id();
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const A w = shfl_up(v, d);
            if (lane >= d) v = M::op(w, v);
        }
        v = M::op(carry, v);
        if (t < L) dst[x] = M::template put<SW>(v);
        carry = shfl_idx(v, 31);
    }
}

// Long lines in few of them: each line is cut into nseg segments of G
// elements, scanned independently (k_scan_seg: one thread per (line,
// segment) for I > 1, one warp for I == 1), then the carry of every segment
// -- the (+) of the totals of the segments before it (after it, for a
// suffix) -- is formed per line in segment order (k_seg_carry) and combined
// into the segment's elements (k_seg_apply).
template <class M, class SR, class SW, bool SUF>
__global__ void __launch_bounds__(256)
k_scan_seg(const SR *in, SW *out, int64_t O, int64_t n, int64_t I, int64_t G, int64_t nseg)
{
    using A = typename M::acc_t;
    if (I == 1) {
        const int lane = threadIdx.x & 31;
        const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        if (w >= O * nseg) return;   // whole warps
        const int64_t o = w / nseg, sg = w - o * nseg;
        const int64_t a = sg * G, len = min(G, n - a);
        const SR *src = in + o * n + a;
        SW *dst = out + o * n + a;
        A carry = M::id();
        for (int64_t c0 = 0; c0 < len; c0 += 32) {
            const int64_t t = c0 + lane;
            const int64_t x = SUF ? len - 1 - t : t;
            A v = t < len ? M::get(src[x]) : M::id();
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const A u = shfl_up(v, d);
                if (lane >= d) v = M::op(u, v);
            }
            v = M::op(carry, v);
            if (t < len) dst[x] = M::template put<SW>(v);
            carry = shfl_idx(v, 31);
        }
        return;
    }
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= O * nseg * I) return;
    const int64_t i = gid % I, r = gid / I, sg = r % nseg, o = r / nseg;
    const int64_t a = sg * G, len = min(G, n - a);
    const SR *src = in + (o * n + a) * I + i;
    SW *dst = out + (o * n + a) * I + i;
    A acc = M::id();
    for (int64_t t0 = 0; t0 < len; t0 += 8) {
        SR v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t t = t0 + u;
            if (t < len) v[u] = src[(SUF ? len - 1 - t : t) * I];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t t = t0 + u;
            if (t < len) {
                acc = M::op(acc, M::get(v[u]));
                dst[(SUF ? len - 1 - t : t) * I] = M::template put<SW>(acc);
            }
        }
    }
}

// Carries: Cy[(o * nseg + s) * I + i] = (+) of the totals of the segments
// before s (SUF: after s) of line (o, i); a segment's total is its scan at
// its last (SUF: first) element.  One warp per line: 32 segments at a time,
// scanned across the lanes, each group carrying the total of the ones
// before it.
template <class M, class SW, bool SUF>
__global__ void __launch_bounds__(256)
k_seg_carry(const SW *__restrict__ out, SW *__restrict__ Cy, int64_t O, int64_t n, int64_t I, int64_t G,
            int64_t nseg)
{
    using A = typename M::acc_t;
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= O * I) return;   // whole warps
    const int64_t o = w / I, i = w - o * I;
    A run = M::id();
    for (int64_t t0 = 0; t0 < nseg; t0 += 32) {
        const int64_t t = t0 + lane;
        const int64_t sg = SUF ? nseg - 1 - t : t;
        A v = M::id();
        if (t < nseg) {
            const int64_t a = sg * G, len = min(G, n - a);
            v = M::get(out[(o * n + (SUF ? a : a + len - 1)) * I + i]);
        }
        A inc = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const A u = shfl_up(inc, d);
            if (lane >= d) inc = M::op(u, inc);
        }
        A ex = shfl_up(inc, 1);
        if (lane == 0) ex = M::id();
        if (t < nseg) Cy[(o * nseg + sg) * I + i] = M::template put<SW>(M::op(run, ex));
        run = M::op(run, shfl_idx(inc, 31));
    }
}

template <class M, class SW, bool SUF>
__global__ void __launch_bounds__(256)
k_seg_apply(SW *__restrict__ out, const SW *__restrict__ Cy, int64_t O, int64_t n, int64_t I, int64_t G,
            int64_t nseg)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= O * n * I) return;
    const int64_t i = gid % I, r = gid / I, x = r % n, o = r / n;
    const int64_t sg = x / G;
    if (SUF ? sg == nseg - 1 : sg == 0) return;   // the carry is the identity
    out[gid] = M::template put<SW>(M::op(M::get(Cy[(o * nseg + sg) * I + i]), M::get(out[gid])));
}

// Shape, box and row-major strides of a tensor of at most 8 dimensions.
struct CmpDims {
    int d;
    int64_t n[8], k[8], st[8];
};

// SATC: the box sum at every x from the summed-area table S (integer +,
// wrapping), and with `weak` the total minus it.  For each of the 2^d
// corners c (bit i set: the upper end x_i + k_i - 1 clipped to n_i - 1,
// else x_i - 1) the term is S[c] with sign (-1)^(d - bits), and 0 where a
// lower end is -1.
template <class T, class U>
__global__ void __launch_bounds__(256)
k_satc(const T *__restrict__ S, T *__restrict__ out, CmpDims g, int64_t N, int weak)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= N) return;
    int64_t x[8];
    int64_t r = gid;
    for (int i = g.d - 1; i >= 0; --i) {
        x[i] = r % g.n[i];
        r /= g.n[i];
    }
    U box = 0;
    const int nc = 1 << g.d;
    for (int c = 0; c < nc; ++c) {
        int64_t off = 0;
        bool empty = false;
        int lows = 0;
        for (int i = 0; i < g.d; ++i) {
            int64_t y;
            if ((c >> i) & 1) {
                y = x[i] + g.k[i] - 1;
                if (y > g.n[i] - 1) y = g.n[i] - 1;
            } else {
                y = x[i] - 1;
                ++lows;
                if (y < 0) empty = true;
            }
            off += y * g.st[i];
        }
        if (empty) continue;
        const U v = (U)S[off];
        box = (lows & 1) ? box - v : box + v;
    }
    if (weak) {
        const U total = (U)S[N - 1];
        box = total - box;
    }
    out[gid] = (T)box;
}

// Corners: which orthant each of the 2^d corner tensors contributes, for
// d = 2 and 3.  Entry [c][i] for dimension i: 0 prefix below x_i (y < x_i),
// 1 prefix below x_i + k_i, 2 suffix from x_i (y >= x_i), 3 suffix from
// x_i + k_i.  d = 2: the pinwheel of App. A (four regions turning around
// the box); d = 3: eight regions found by an exhaustive search over the
// 3^3 cells (below / inside / above the box in every dimension) and checked
// to cover every cell but the box exactly once.
__host__ __device__ constexpr int corner_region(int d, int c, int i)
{
    constexpr int t2[4][2] = {{0, 1}, {1, 3}, {3, 2}, {2, 0}};
    constexpr int t3[8][3] = {{0, 0, 0}, {0, 1, 2}, {1, 2, 0}, {1, 3, 2},
                              {2, 0, 1}, {2, 1, 3}, {3, 2, 1}, {3, 3, 3}};
    return d == 2 ? t2[c][i] : t3[c][i];
}

// The corner tensors' index of corner c: bit i of the tensor index is set
// when dimension i is a suffix (regions 2 and 3).
__host__ __device__ constexpr int corner_tensor(int d, int c)
{
    int b = 0;
    for (int i = 0; i < d; ++i)
        if (corner_region(d, c, i) >= 2) b |= 1 << i;
    return b;
}

struct CornerTensors {
    const void *t[8];
};

// excluded[x] = (+) over the 2^D corners of T_b at the shifted corner point,
// e where a region is empty.  T_b[y] holds the (+) over the orthant of y
// that b names (prefix: indices <= y, suffix: >= y).
template <class M, class SC, class SOut, int D>
__global__ void __launch_bounds__(256)
k_corners(CornerTensors T, SOut *__restrict__ out, CmpDims g, int64_t N)
{
    using A = typename M::acc_t;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= N) return;
    int64_t x[D];
    int64_t r = gid;
#pragma unroll
    for (int i = D - 1; i >= 0; --i) {
        x[i] = r % g.n[i];
        r /= g.n[i];
    }
    A acc = M::id();
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        int64_t off = 0;
        bool empty = false;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            int64_t y;
            switch (corner_region(D, c, i)) {
            case 0: y = x[i] - 1; empty |= y < 0; break;                                   // y < x_i
            case 1: y = min(x[i] + g.k[i], g.n[i]) - 1; break;                              // y < x_i + k_i
            case 2: y = x[i]; break;                                                         // y >= x_i
            default: y = x[i] + g.k[i]; empty |= y >= g.n[i]; break;                        // y >= x_i + k_i
            }
            off += y * g.st[i];
        }
        if (!empty) acc = M::op(acc, M::get(static_cast<const SC *>(T.t[corner_tensor(D, c)])[off]));
    }
    out[gid] = M::template put<SOut>(acc);
}

}  // namespace exsum
