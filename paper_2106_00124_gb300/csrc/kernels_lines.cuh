// kernels_lines.cuh -- line kernels of the GPU path.
//
// Every pass of BDBS and box-complement works on "lines": the rows of a
// tensor along one dimension (Sec. 2, "a (tensor) row").  A tensor is seen
// as a 3-D view [O, n, I]: O outer positions, the dimension of length n
// being processed, and I inner positions (I = 1 when the dimension is the
// contiguous one).  Element x of line (o, i) sits at o*n*I + x*I + i.
//
// Kernels here:
//   k_inc_lines    BDBS-Along-Dim: the included sum of window k along each
//                  line, by the k-blocked prefix and suffix scans and the
//                  combine step of BDBS-1D (Sec. 3).
//   k_carry_*      Per-segment carries of the prefix/suffix along dim 1
//                  (the dimension-1 step itself is k_exline2 in
//                  kernels_fast.cuh).
#pragma once

#include "monoid.cuh"

namespace exsum {

// ---------------------------------------------------------------------------
// Block-wide exclusive prefix and exclusive suffix of one value per thread.
// Every thread of the block must call it.
// ---------------------------------------------------------------------------
template <class M, int NT>
__device__ __forceinline__ void block_exscan_both(typename M::acc_t v, typename M::acc_t &pre,
                                                  typename M::acc_t &suf)
{
    using A = typename M::acc_t;
    constexpr int NW = NT / 32;
    __shared__ A wtot[NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    A inc = v;
#pragma unroll
    for (int dl = 1; dl < 32; dl <<= 1) {
        A o = shfl_up(inc, dl);
        if (lane >= dl) inc = M::op(o, inc);
    }
    A sinc = v;
#pragma unroll
    for (int dl = 1; dl < 32; dl <<= 1) {
        A o = shfl_down(sinc, dl);
        if (lane + dl < 32) sinc = M::op(sinc, o);
    }
    if (lane == 31) wtot[warp] = inc;
    __syncthreads();
    A wpre = M::id(), wsuf = M::id();
    for (int w = 0; w < warp; ++w) wpre = M::op(wpre, wtot[w]);
    for (int w = NW - 1; w > warp; --w) wsuf = M::op(wtot[w], wsuf);
    A ex = shfl_up(inc, 1);
    if (lane == 0) ex = M::id();
    A sx = shfl_down(sinc, 1);
    if (lane == 31) sx = M::id();
    pre = M::op(wpre, ex);
    suf = M::op(sx, wsuf);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// BDBS-Along-Dim for one chunk of one line per thread.
//
// The thread produces outputs x in [r0, min(r0+Lc, n)) of its line and reads
// inputs up to x+k-1 (elements past n are the identity: the clipped box of
// Sec. 2 / the identity padding of the Sec. 3 footnote).  Blocks of length k
// start at r0.  For x in block b the window [x, x+k) is the suffix of block b
// from x (Range-Suffix-Row) followed by the prefix of block b+1 up to x+k-1
// (Range-Prefix-Row); a block start takes its whole block (Combine-Along-Row,
// Lemma "Correctness in 1D").  The suffix of the current block is held in k
// per-thread slots (shared memory, or global scratch for large k); the next
// block's prefix is a running register value, and its elements replace the
// consumed suffix slots as they stream in.
// ---------------------------------------------------------------------------
template <class M, class SIn, class SOut>
__global__ void __launch_bounds__(128)
k_inc_lines(const SIn *__restrict__ in, SOut *__restrict__ out, int64_t O, int64_t n, int64_t I,
            int64_t k, int64_t Lc, int64_t nchunks, typename M::acc_t *__restrict__ gslots)
{
    using A = typename M::acc_t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t total = O * nchunks * I;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const int64_t i = gid % I;
    const int64_t rest = gid / I;
    const int64_t ch = rest % nchunks;
    const int64_t o = rest / nchunks;
    const int64_t base = o * n * I + i;
    A *slot;
    int64_t ss;
    if (gslots) {
        slot = gslots + gid;
        ss = total;
    } else {
        slot = reinterpret_cast<A *>(smem_raw) + threadIdx.x;
        ss = blockDim.x;
    }
    const int64_t r0 = ch * Lc;
    const int64_t rend = (r0 + Lc < n) ? r0 + Lc : n;

    // Block 0: load, then suffix scan in place.
    for (int64_t j = 0; j < k; ++j) {
        const int64_t x = r0 + j;
        slot[j * ss] = x < n ? M::get(in[base + x * I]) : M::id();
    }
    for (int64_t j = k - 2; j >= 0; --j) slot[j * ss] = M::op(slot[j * ss], slot[(j + 1) * ss]);

    for (int64_t sb = r0; sb < rend; sb += k) {
        out[base + sb * I] = M::template put<SOut>(slot[0]);
        A p = M::id();
        const int64_t jmax = (rend - sb - 1 < k - 1) ? rend - sb - 1 : k - 1;  // outputs left in block
        const bool more = sb + k < rend;
#pragma unroll 4
        for (int64_t j = 0; j < k - 1; ++j) {
            if (j >= jmax && !more) break;
            const int64_t xn = sb + k + j;
            const A v = xn < n ? M::get(in[base + xn * I]) : M::id();
            p = M::op(p, v);
            if (j < jmax) out[base + (sb + 1 + j) * I] = M::template put<SOut>(M::op(slot[(j + 1) * ss], p));
            slot[j * ss] = v;
        }
        if (more) {
            const int64_t xl = sb + 2 * k - 1;
            slot[(k - 1) * ss] = xl < n ? M::get(in[base + xl * I]) : M::id();
            for (int64_t j = k - 2; j >= 0; --j) slot[j * ss] = M::op(slot[j * ss], slot[(j + 1) * ss]);
        }
    }
}

// ---------------------------------------------------------------------------
// Carries of the dimension-1 prefix/suffix, per segment s and column c:
//   Pc[s] = (+) of segments before s                       (exclusive prefix)
//   W[s]  = (+) of rows >= (s+1)*L + k1                     (suffix past the
//           target window of segment s); with q = s + qoff, qoff = 1 + k1/L,
//           r = k1 mod L, this is Rt[q] (+) (+)_{s' > q} R[s'].
//   Q[s]  = Pc[s] (+) W[s] (+) T[c]   (T: the lower-dimensional excluded sum
//           of the column totals, or the identity)
// ---------------------------------------------------------------------------
template <class M>
__global__ void __launch_bounds__(256)
k_carry_col(const typename M::car_t *__restrict__ R, const typename M::car_t *__restrict__ Rt,
            const typename M::car_t *__restrict__ T, typename M::car_t *__restrict__ Q, int64_t Mc,
            int64_t S, int64_t qoff)
{
    using A = typename M::acc_t;
    using C = typename M::car_t;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Mc) return;
    // Backward: suffix totals SR[s] = (+)_{s' >= s} R[s'], parked in Q.
    A acc = M::id();
    for (int64_t s = S - 1; s >= 0; --s) {
        acc = M::op(M::get(R[s * Mc + c]), acc);
        Q[s * Mc + c] = M::template put<C>(acc);
    }
    const A tc = T ? M::get(T[c]) : M::id();
    A pc = M::id();
    for (int64_t s = 0; s < S; ++s) {
        const int64_t q = s + qoff;
        A w = M::id();
        if (q < S) {
            w = M::get(Rt[q * Mc + c]);
            if (q + 1 < S) w = M::op(w, M::get(Q[(q + 1) * Mc + c]));  // SR[q+1], q+1 > s: not yet overwritten
        }
        const A rs = M::get(R[s * Mc + c]);
        Q[s * Mc + c] = M::template put<C>(M::op(M::op(pc, w), tc));
        pc = M::op(pc, rs);
    }
}

// Same carries with one block per column (many segments, few columns).
// SR is a scratch array of S*Mc carries.
template <class M, int NT>
__global__ void __launch_bounds__(NT)
k_carry_blk(const typename M::car_t *__restrict__ R, const typename M::car_t *__restrict__ Rt,
            const typename M::car_t *__restrict__ T, typename M::car_t *__restrict__ Q,
            typename M::car_t *__restrict__ SR, int64_t Mc, int64_t S, int64_t qoff,
            typename M::car_t *__restrict__ G)
{
    using A = typename M::acc_t;
    using C = typename M::car_t;
    const int64_t c = blockIdx.x;
    const int64_t per = (S + NT - 1) / NT;
    const int64_t sb = threadIdx.x * per;
    const int64_t se = (sb + per < S) ? sb + per : S;
    A tot = M::id();
    for (int64_t s = sb; s < se; ++s) tot = M::op(tot, M::get(R[s * Mc + c]));
    A pre, suf;
    block_exscan_both<M, NT>(tot, pre, suf);
    if (G && threadIdx.x == NT - 1) G[c] = M::template put<C>(M::op(pre, tot));
    A acc = suf;
    for (int64_t s = se - 1; s >= sb; --s) {
        acc = M::op(M::get(R[s * Mc + c]), acc);
        SR[s * Mc + c] = M::template put<C>(acc);
    }
    __syncthreads();
    const A tc = T ? M::get(T[c]) : M::id();
    A pc = pre;
    for (int64_t s = sb; s < se; ++s) {
        const int64_t q = s + qoff;
        A w = M::id();
        if (q < S) {
            w = M::get(Rt[q * Mc + c]);
            if (q + 1 < S) w = M::op(w, M::get(SR[(q + 1) * Mc + c]));
        }
        Q[s * Mc + c] = M::template put<C>(M::op(M::op(pc, w), tc));
        pc = M::op(pc, M::get(R[s * Mc + c]));
    }
}

// ---------------------------------------------------------------------------
// BDBS along the contiguous dimension for long boxes (k > 32): one warp per
// segment of G elements of a row (G a multiple of k, so segments hold whole
// blocks), in chunks of 32 consecutive elements, one per lane.
//   Backwards over the segment: the suffix of every element within its block
//   of k (a segmented warp scan: lanes whose elements lie in the same block
//   combine; the block continuing from the chunk before is carried in), into
//   out.
//   Forwards over the elements y the segment's windows reach in the next
//   blocks: the prefix of y within its block, the same way, and
//   out[y - k + 1] = S (+) prefix -- except where y - k + 1 starts a block
//   (its window is the whole block: the suffix alone).
//   Windows cut by the row's end take the prefix of the last element.
// Input read twice and out read once besides its two writes, all coalesced.
// ---------------------------------------------------------------------------
template <class M, class SIn, class SOut>
__global__ void __launch_bounds__(256)
k_inc_rows_big(const SIn *__restrict__ in, SOut *__restrict__ out, int64_t rows, int64_t L, int64_t k, int64_t G,
               int64_t nseg)
{
    using Lt = typename M::loc_t;
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= rows * nseg) return;   // whole warps
    const int64_t row = w / nseg, sg = w - row * nseg;
    const SIn *src = in + row * L;
    SOut *dst = out + row * L;
    const int64_t a = sg * G, e = min(a + G, L);
    // segmented inclusive scan across the lanes in lane order; blk: block of the lane's element
    auto seg_scan = [&](Lt v, int64_t blk) -> Lt {
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Lt u = shfl_up(v, d);
            const int64_t bu = shfl_up(blk, d);
            if (lane >= d && bu == blk) v = M::lop(u, v);
        }
        return v;
    };
    // backwards: suffixes within blocks, four chunks per round (their loads
    // in flight together)
    Lt carry = M::lid();
    int64_t carry_blk = -1;
    // (block indices: one division per chunk; k > 32, so a chunk meets at
    // most two blocks)
    for (int64_t r0 = 0; r0 < e - a; r0 += 128) {
        Lt v[4];
        int64_t xs[4], blks[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t xh = e - 1 - r0 - 32 * u;   // the chunk's first (highest) element
            const int64_t bh = xh / k, oh = xh - bh * k;
            const int64_t x = xh - lane;
            const bool ok = x >= a;
            xs[u] = x;
            blks[u] = ok ? (lane <= oh ? bh : bh - 1) : -2 - lane;
            v[u] = ok ? M::lget(src[x]) : M::lid();
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            Lt t = seg_scan(v[u], blks[u]);
            if (blks[u] == carry_blk) t = M::lop(t, carry);
            if (xs[u] >= a) dst[xs[u]] = M::template lput<SOut>(t);
            carry = shfl_idx(t, 31);
            carry_blk = shfl_idx(blks[u], 31);
        }
    }
    __syncwarp();
    // forwards: prefixes of the next blocks, combined
    const int64_t y0 = a + k, y1 = min(a + G + k - 1, L);
    carry = M::lid();
    carry_blk = -1;
    Lt last = M::lid();   // prefix of the row's last element, once reached
    for (int64_t r0 = y0; r0 < y1; r0 += 128) {
        Lt v[4], sv[4];
        int64_t blks[4], yms[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t t0 = r0 + 32 * u;
            const int64_t b0 = t0 / k, o0 = t0 - b0 * k;
            const int64_t y = t0 + lane;
            const bool ok = y < y1;
            const bool wrap = o0 + lane >= k;
            blks[u] = ok ? (wrap ? b0 + 1 : b0) : -2 - lane;
            yms[u] = wrap ? o0 + lane - k : o0 + lane;   // y mod k
            v[u] = ok ? M::lget(src[y]) : M::lid();
            sv[u] = (ok && yms[u] != k - 1) ? M::lget(dst[y - k + 1]) : M::lid();
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t y = r0 + 32 * u + lane;
            Lt t = seg_scan(v[u], blks[u]);
            if (blks[u] == carry_blk) t = M::lop(t, carry);
            if (y < y1 && yms[u] != k - 1) dst[y - k + 1] = M::template lput<SOut>(M::lop(sv[u], t));
            if (y == L - 1) last = t;
            carry = shfl_idx(t, 31);
            carry_blk = shfl_idx(blks[u], 31);
        }
    }
    // the lane that held y = L - 1 shares its prefix
    unsigned has = __ballot_sync(0xffffffffu, y1 == L && (L - 1 - y0) >= 0 && ((L - 1 - y0) & 31) == lane &&
                                                  L - 1 >= y0);
    if (has) last = shfl_idx(last, __ffs(has) - 1);
    __syncwarp();
    // windows cut by the row's end
    for (int64_t x = max(a, L - k + 1) + lane; x < e; x += 32) {
        if (x % k == 0) continue;   // a block start: the suffix alone
        if ((x / k + 1) * k < L && has) dst[x] = M::template lput<SOut>(M::lop(M::lget(dst[x]), last));
    }
}

}  // namespace exsum
