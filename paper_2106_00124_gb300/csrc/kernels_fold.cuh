// kernels_fold.cuh -- the row totals folded into the first strided pass, and
// the two-dimensional lower problem of the row schedule in two short kernels.
//
// For d = 3 the row schedule needs R[x1, x2] = (+)_{x3} X[x1, x2, x3] (the
// dimension reduction along the last dimension, Sec. 4) and the excluded
// sum T of R with box (k1, k2).  Reading X once more just for R costs a
// third of the tensor's traffic.  Instead the strided BDBS pass along
// dimension 1, which reads all of X anyway, also leaves partial row totals
// (one per 128 consecutive elements of a row), and
//   k_plane_totals  combines them into R and the plane totals
//                   R2[x1] = (+)_{x2} R[x1, x2],
//   k_exc2d         forms T[x1, x2] = T2[x1] (+) (+)_{y2 < x2} H1[x1, y2]
//                                     (+) (+)_{y2 >= x2 + k2} H1[x1, y2]
//                   with T2 the one-dimensional excluded sum of R2 (box k1)
//                   and H1 the window of k1 planes of R -- the row schedule
//                   once more, one block per x1 (Sec. 4, Theorem "Recursive
//                   Box-complement", the last dimension peeled).
// The same two kernels are a whole excluded sum of a small d = 2 tensor
// (read as R, written as T, in the compensated accumulator throughout).
// Every reduction runs in a fixed order, so results do not depend on timing.
#pragma once

#include "kernels_flat.cuh"

namespace exsum {

// ---------------------------------------------------------------------------
// BDBS-Along-Dim along dimension 1 (view [n, I], I % 128 == 0, 16-byte
// aligned rows, 4-byte local type) as k_inc_strided4, with row totals: the
// 32 lanes of a warp hold 128 consecutive inner positions, which lie in one
// row of length L (L % 128 == 0).  Every input row of the thread's chunk
// (Lc <= 32 rows) is reduced over its 4 columns as it is loaded, the 32
// lanes' values go to shared memory, and lane l adds up row r0 + l in lane
// order: Rp[(x1 * (I / L) + row) * H + h] = (+) of the 128 inputs, H = L / 128.
// ---------------------------------------------------------------------------
template <class M, class SIn, class SOut, int KMAX>
__global__ void __launch_bounds__(128)
k_inc_strided4_rt(const SIn *__restrict__ in, SOut *__restrict__ out, int n, int64_t I, int k, int Lc,
                  int nchunks, int L, typename M::loc_t *__restrict__ Rp)
{
    using Lt = typename M::loc_t;
    static_assert(sizeof(Lt) == 4, "4-byte local type");
    __shared__ Lt rp[4][32][33];
    const int64_t I4 = I >> 2;
    const int64_t total = nchunks * I4;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    pdl_trigger();   // the plane totals may launch (they wait for this grid)
    if (gid >= total) return;   // whole warps: total is a multiple of 32
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i4 = gid % I4;
    const int ch = (int)(gid / I4);
    const SIn *src = in + 4 * i4;
    SOut *dst = out + 4 * i4;
    const int r0 = ch * Lc;
    const int rend = min(r0 + Lc, n);
    const uint64_t pol_in = l2_policy_evict_first();
    const uint64_t pol_out = l2_policy_evict_last();
    Lt(*acc)[33] = rp[warp];
    auto note = [&](int x, const Lt *v) {
        if (x < rend) acc[x - r0][lane] = M::lop(M::lop(v[0], v[1]), M::lop(v[2], v[3]));
    };
    // (row totals are noted after all loads of a block are issued: a shared
    // store between the loads would hold each load back until the previous
    // one returns)
    Lt S[KMAX][4], v[KMAX][4];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        if (j < k && r0 + j < n) {
            load4<M>(src + (int64_t)(r0 + j) * I, true, 4, v[j], pol_in);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) v[j][c] = M::lid();
        }
    }
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
        if (j < k) note(r0 + j, v[j]);
#pragma unroll
    for (int c = 0; c < 4; ++c) S[KMAX - 1][c] = v[KMAX - 1][c];
#pragma unroll
    for (int j = KMAX - 2; j >= 0; --j)
#pragma unroll
        for (int c = 0; c < 4; ++c) S[j][c] = M::lop(v[j][c], S[j + 1][c]);
    for (int sb = r0; sb < rend; sb += k) {
        store4<M>(dst + (int64_t)sb * I, true, 4, S[0], pol_out);
        const int nb = sb + k;
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            if (j < k && nb + j < n) {
                load4<M>(src + (int64_t)(nb + j) * I, true, 4, v[j], pol_in);
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) v[j][c] = M::lid();
            }
        }
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
            if (j < k) note(nb + j, v[j]);
        Lt p[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) p[c] = v[0][c];
#pragma unroll
        for (int j = 0; j + 1 < KMAX; ++j) {
            Lt w[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (j > 0) p[c] = M::lop(p[c], v[j][c]);
                w[c] = M::lop(S[j + 1][c], p[c]);
            }
            if (j + 1 < k && sb + 1 + j < rend) store4<M>(dst + (int64_t)(sb + 1 + j) * I, true, 4, w, pol_out);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) S[KMAX - 1][c] = v[KMAX - 1][c];
#pragma unroll
        for (int j = KMAX - 2; j >= 0; --j)
#pragma unroll
            for (int c = 0; c < 4; ++c) S[j][c] = M::lop(v[j][c], S[j + 1][c]);
    }
    __syncwarp();
    const int x = r0 + lane;
    if (x < rend) {
        // pairwise (tree) combination of the 32 lanes' values, in a fixed
        // order: rounding grows with the tree depth, not the count
        Lt w[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) w[c] = acc[lane][c];
#pragma unroll
        for (int h = 16; h >= 1; h >>= 1)
#pragma unroll
            for (int c = 0; c < h; ++c) w[c] = M::lop(w[c], w[c + h]);
        const Lt t = w[0];
        const int64_t p0 = 4 * (i4 - lane);   // first inner position of the warp
        const int64_t rows_per_x1 = I / L;
        const int H = L >> 7;
        Rp[((int64_t)x * rows_per_x1 + p0 / L) * H + (int)((p0 % L) >> 7)] = t;
    }
}

// Block-wide combine of one value per thread, in a fixed order (butterfly
// within warps, then warp 0 over the warp results); the result is returned
// to every thread.  `red` holds at least blockDim.x / 32 values.
template <class M>
__device__ __forceinline__ typename M::acc_t block_reduce(typename M::acc_t v, typename M::acc_t *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v = M::op(v, shfl_xor(v, m));
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? red[lane] : M::id();
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) v = M::op(v, shfl_xor(v, m));
        if (lane == 0) red[32] = v;
    }
    __syncthreads();
    return red[32];
}

// ---------------------------------------------------------------------------
// Plane totals: block x1 combines the H partial row totals of each row x2
// (R[x1, x2], written unless R is null) and their total over x2 (R2[x1]).
// ---------------------------------------------------------------------------
template <class M, class SP>
__device__ __forceinline__ void k_plane_totals_body(const SP *__restrict__ P, int H, typename M::car_t *__restrict__ R,
               typename M::car_t *__restrict__ R2, int n2, int64_t vbid, int64_t vgrid)
{
    using A = typename M::acc_t;
    using C = typename M::car_t;
    __shared__ A red[33];
    const int64_t x1 = vbid;
    pdl_trigger();
    pdl_wait();   // P comes from the kernel before
    A tot = M::id();
    for (int x2 = threadIdx.x; x2 < n2; x2 += blockDim.x) {
        const SP *p = P + (x1 * n2 + x2) * H;
        // H <= 8: all loads issued before the first use
        SP v[8];
#pragma unroll
        for (int h = 0; h < 8; ++h)
            if (h < H) v[h] = p[h];
        A r = M::get(v[0]);
#pragma unroll
        for (int h = 1; h < 8; ++h)
            if (h < H) r = M::op(r, M::get(v[h]));
        if (R) R[x1 * n2 + x2] = M::template put<C>(r);
        tot = M::op(tot, r);
    }
    tot = block_reduce<M>(tot, red);
    if (threadIdx.x == 0) R2[x1] = M::template put<C>(tot);
}

template <class M, class SP>
__global__ void __launch_bounds__(256)
k_plane_totals(const SP *__restrict__ P, int H, typename M::car_t *__restrict__ R,
               typename M::car_t *__restrict__ R2, int n2)
{
    k_plane_totals_body<M, SP>(P, H, R, R2, n2, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// Excluded sums of the n1 x n2 tensor R with box (k1, k2), given its plane
// totals R2 (one block per x1, k1 <= 64, n2 <= 4096; dynamic shared memory
// 2 * n2 accumulators):
//   T2  = (+)_{y < x1} R2[y] (+) (+)_{y >= x1 + k1} R2[y]
//   H1  = (+)_{i < k1, x1 + i < n1} R[x1 + i, .]         (window of planes)
//   T[x1, x2] = T2 (+) exclusive prefix of H1 before x2 (+) suffix of H1 from x2 + k2
// The scans along x2: each thread scans a contiguous segment, the segment
// totals are scanned across the block (warp shuffles, then the warp totals),
// in both directions.
// ---------------------------------------------------------------------------
// r_ready: R does not come from the kernel before (it is the input itself),
// so the window of planes is read before waiting for that kernel (R2).
template <class M, class SR = typename M::car_t, class ST = typename M::car_t>
__device__ __forceinline__ void k_exc2d_body(const SR *__restrict__ R, const typename M::car_t *__restrict__ R2, ST *__restrict__ T, int n1,
        int n2, int k1, int k2, int64_t vbid, int64_t vgrid, int r_ready = 0)
{
    using A = typename M::acc_t;
    using C = typename M::car_t;
    extern __shared__ __align__(16) unsigned char e2_smem[];
    A *hv = reinterpret_cast<A *>(e2_smem);   // H1, then its exclusive prefixes
    A *sf = hv + n2;                            // inclusive suffixes of H1
    __shared__ A red[33];
    __shared__ A wpre[32], wsuf[32];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int x1 = vbid;
    pdl_trigger();
    if (!r_ready) pdl_wait();   // R and R2 come from the kernel before
    // window of k1 planes
    const int kw = min(k1, n1 - x1);
    for (int x2 = tid; x2 < n2; x2 += nt) {
        const SR *col = R + (int64_t)x1 * n2 + x2;
        A h = M::get(col[0]);
        // eight loads in flight per round
        for (int i0 = 1; i0 < kw; i0 += 8) {
            SR v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i0 + i < kw) v[i] = col[(int64_t)(i0 + i) * n2];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i0 + i < kw) h = M::op(h, M::get(v[i]));
        }
        hv[x2] = h;
    }
    if (r_ready) pdl_wait();   // R2 comes from the kernel before
    // the one-dimensional part
    A t2 = M::id();
    for (int y0 = 0; y0 < n1; y0 += 4 * nt) {
        C v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int y = y0 + u * nt + tid;
            v[u] = y < n1 ? R2[y] : M::template put<C>(M::id());
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int y = y0 + u * nt + tid;
            if (y < n1 && (y < x1 || y >= x1 + k1)) t2 = M::op(t2, M::get(v[u]));
        }
    }
    t2 = block_reduce<M>(t2, red);
    __syncthreads();
    // scans along x2: thread segment [s0, s1)
    const int seg = (n2 + nt - 1) / nt;
    const int s0 = min(tid * seg, n2), s1 = min(s0 + seg, n2);
    A st = M::id();
    for (int x = s0; x < s1; ++x) st = M::op(st, hv[x]);
    // exclusive prefix and exclusive suffix of the segment totals
    A pi = st, si = st;
#pragma unroll
    for (int dl = 1; dl < 32; dl <<= 1) {
        const A u = shfl_up(pi, dl);
        const A w = shfl_down(si, dl);
        if (lane >= dl) pi = M::op(u, pi);
        if (lane + dl < 32) si = M::op(si, w);
    }
    if (lane == 31) wpre[warp] = pi;
    if (lane == 0) wsuf[warp] = si;
    __syncthreads();
    A pw = M::id(), sw = M::id();
    for (int w = 0; w < warp; ++w) pw = M::op(pw, wpre[w]);
    for (int w = nw - 1; w > warp; --w) sw = M::op(wsuf[w], sw);
    A pe = shfl_up(pi, 1), se = shfl_down(si, 1);
    if (lane == 0) pe = M::id();
    if (lane == 31) se = M::id();
    pe = M::op(pw, pe);
    se = M::op(se, sw);
    // suffixes (backwards) and exclusive prefixes (forwards, in place)
    A run = se;
    for (int x = s1 - 1; x >= s0; --x) {
        run = M::op(hv[x], run);
        sf[x] = run;
    }
    run = pe;
    for (int x = s0; x < s1; ++x) {
        const A h = hv[x];
        hv[x] = run;
        run = M::op(run, h);
    }
    __syncthreads();
    for (int x2 = tid; x2 < n2; x2 += nt) {
        const A s = x2 + k2 < n2 ? sf[x2 + k2] : M::id();
        T[(int64_t)x1 * n2 + x2] = M::template put<ST>(M::op(t2, M::op(hv[x2], s)));
    }
}

// ---------------------------------------------------------------------------
// The same excluded sums, one WARP per plane x1 (blockDim / 32 planes per
// block, no block barrier), for n2 small enough that each warp keeps H1 and
// its suffixes in shared memory (dynamic: 2 * n2 accumulators per warp):
//   T2 over the plane totals (lanes stride over y, then a reduction tree
//   whose result lane 0 broadcasts: a fixed order);
//   backwards over chunks of 32 columns: H1 (k1 plane loads per column,
//   coalesced across the lanes) and its inclusive suffixes (warp scan of the
//   chunk, then the carry from the chunk after it);
//   forwards: the exclusive prefixes the same way, and every output
//   T2 (+) prefix before x2 (+) suffix from x2 + k2.
// ---------------------------------------------------------------------------
template <class M>
__device__ __forceinline__ typename M::acc_t warp_sum0(typename M::acc_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const typename M::acc_t w = shfl_down(v, d);
        if (lane + d < 32) v = M::op(v, w);
    }
    return shfl_idx(v, 0);
}

// kwin: planes of R combined into H1 -- k1, or 1 when R already holds the
// window sums along x1 (H1 itself, from a strided BDBS pass).
template <class M, class SR = typename M::car_t, class ST = typename M::car_t>
__device__ __forceinline__ void k_exc2d_w_body(const SR *__restrict__ R, const typename M::car_t *__restrict__ R2,
                                               ST *__restrict__ T, int n1, int n2, int k1, int k2, int64_t vbid,
                                               int64_t vgrid, int kwin)
{
    using A = typename M::acc_t;
    extern __shared__ __align__(16) unsigned char e2w_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    A *hv = reinterpret_cast<A *>(e2w_smem) + (int64_t)warp * 2 * n2;
    A *sf = hv + n2;
    pdl_trigger();
    pdl_wait();   // R and R2 come from the kernel before
    const int64_t x1l = vbid * nw + warp;
    if (x1l >= n1) return;   // a whole warp; nothing below waits for the block
    const int x1 = (int)x1l;
    A t2 = M::id();
    for (int y = lane; y < n1; y += 32)
        if (y < x1 || y >= x1 + k1) t2 = M::op(t2, M::get(R2[y]));
    t2 = warp_sum0<M>(t2);
    const int kw = min(kwin, n1 - x1);
    const SR *row = R + (int64_t)x1 * n2;
    const int nc = (n2 + 31) >> 5;
    A carry = M::id();
    for (int c = nc - 1; c >= 0; --c) {
        const int x2 = (c << 5) + lane;
        A h = M::id();
        if (x2 < n2) {
            const SR *col = row + x2;
            h = M::get(col[0]);
            for (int i0 = 1; i0 < kw; i0 += 8) {
                SR v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (i0 + i < kw) v[i] = col[(int64_t)(i0 + i) * n2];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (i0 + i < kw) h = M::op(h, M::get(v[i]));
            }
            hv[x2] = h;
        }
        A s = h;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const A w = shfl_down(s, d);
            if (lane + d < 32) s = M::op(s, w);
        }
        s = M::op(s, carry);
        if (x2 < n2) sf[x2] = s;
        carry = shfl_idx(s, 0);
    }
    __syncwarp();
    A run = M::id();
    for (int c = 0; c < nc; ++c) {
        const int x2 = (c << 5) + lane;
        const A h = x2 < n2 ? hv[x2] : M::id();
        A p = h;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const A w = shfl_up(p, d);
            if (lane >= d) p = M::op(w, p);
        }
        A ex = shfl_up(p, 1);
        if (lane == 0) ex = M::id();
        ex = M::op(run, ex);
        run = M::op(run, shfl_idx(p, 31));
        if (x2 < n2) {
            const A sx = x2 + k2 < n2 ? sf[x2 + k2] : M::id();
            T[(int64_t)x1 * n2 + x2] = M::template put<ST>(M::op(t2, M::op(ex, sx)));
        }
    }
}

template <class M, class SR = typename M::car_t, class ST = typename M::car_t>
__global__ void __launch_bounds__(256)
k_exc2d_w(const SR *__restrict__ R, const typename M::car_t *__restrict__ R2, ST *__restrict__ T, int n1, int n2,
          int k1, int k2)
{
    k_exc2d_w_body<M, SR, ST>(R, R2, T, n1, n2, k1, k2, blockIdx.x, gridDim.x, k1);
}

// Warps per block of k_exc2d_w for rows of n2 accumulators of `acc` bytes:
// 2 n2 accumulators per warp in at most 64 KB, at most 8 warps.
__host__ __device__ inline int exc2d_w_warps(int n2, int acc)
{
    int w = 8;
    while (w > 1 && (size_t)2 * n2 * acc * w > 64 * 1024) w >>= 1;
    return w;
}

template <class M, class SR = typename M::car_t, class ST = typename M::car_t>
__global__ void __launch_bounds__(256)
k_exc2d(const SR *__restrict__ R, const typename M::car_t *__restrict__ R2, ST *__restrict__ T, int n1,
        int n2, int k1, int k2, int r_ready = 0)
{
    k_exc2d_body<M, SR, ST>(R, R2, T, n1, n2, k1, k2, blockIdx.x, gridDim.x, r_ready);
}

}  // namespace exsum
