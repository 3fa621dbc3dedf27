// kernels_flat.cuh -- BDBS-Along-Dim passes with 16-byte global accesses:
// the contiguous dimension (k_inc_flat) and four adjacent inner positions of
// a strided dimension per thread (k_inc_strided4).
#pragma once

#include <string.h>

#include <type_traits>

#include "kernels_fast.cuh"

namespace exsum {

// Four consecutive elements starting at p (16-byte-aligned vector access when
// `vec`, else scalar), converted to the local accumulator type.
template <class M, class SIn>
__device__ __forceinline__ void load4(const SIn *p, bool vec, int valid, typename M::loc_t v[4],
                                      uint64_t pol)
{
    if (vec) {
        SIn t[4];
        if constexpr (sizeof(SIn) * 4 == 16) {
            const uint4 r = ld_hint_v4(p, pol);
            memcpy(t, &r, 16);
        } else if constexpr (sizeof(SIn) * 4 == 8) {
            const uint2 r = ld_hint_v2(p, pol);
            memcpy(t, &r, 8);
        } else {
            const uint4 r0 = ld_hint_v4(p, pol);
            const uint4 r1 = ld_hint_v4(reinterpret_cast<const uint4 *>(p) + 1, pol);
            memcpy(t, &r0, 16);
            memcpy(t + 2, &r1, 16);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = M::lget(t[i]);
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = i < valid ? M::lget(ld_hint(p + i, pol)) : M::lid();
    }
}

template <class M, class SOut>
__device__ __forceinline__ void store4(SOut *p, bool vec, int valid, const typename M::loc_t v[4],
                                       uint64_t pol)
{
    SOut t[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = M::template lput<SOut>(v[i]);
    if (vec) {
        if constexpr (sizeof(SOut) * 4 == 16) {
            uint4 r;
            memcpy(&r, t, 16);
            st_hint_v4(p, r, pol);
        } else {
            uint4 r0, r1;
            memcpy(&r0, t, 16);
            memcpy(&r1, t + 2, 16);
            st_hint_v4(p, r0, pol);
            st_hint_v4(reinterpret_cast<uint4 *>(p) + 1, r1, pol);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (i < valid) st_hint(p + i, t[i], pol);
    }
}

// ---------------------------------------------------------------------------
// BDBS-Along-Dim along a strided dimension (view [O, n, I], I % 4 == 0,
// 16-byte aligned rows): as k_inc_strided, but each thread walks four
// adjacent inner positions at once with 16-byte (8-byte for bf16) loads and
// stores -- the register BDBS walk of bdbs_walk on four columns.
// ---------------------------------------------------------------------------
template <class M, class SIn, class SOut, int KMAX>
__device__ __forceinline__ void k_inc_strided4_body(const SIn *__restrict__ in, SOut *__restrict__ out, int64_t O, int n, int64_t I,
               int k, int Lc, int nchunks, int64_t vbid, int64_t vgrid)
{
    using Lt = typename M::loc_t;
    const int64_t I4 = I >> 2;
    const int64_t total = O * nchunks * I4;
    const int64_t gid = (int64_t)vbid * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const int64_t i4 = gid % I4;
    const int64_t rest = gid / I4;
    const int ch = (int)(rest % nchunks);
    const int64_t o = rest / nchunks;
    const SIn *src = in + o * n * I + 4 * i4;
    SOut *dst = out + o * n * I + 4 * i4;
    const int r0 = ch * Lc;
    const int rend = min(r0 + Lc, n);
    const uint64_t pol_in = l2_policy_evict_first();
    const uint64_t pol_out = l2_policy_evict_last();
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
        Lt p[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) p[c] = M::lid();
#pragma unroll
        for (int j = 0; j + 1 < KMAX; ++j) {
            Lt w[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                p[c] = M::lop(p[c], v[j][c]);
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
}

template <class M, class SIn, class SOut, int KMAX>
__global__ void __launch_bounds__(128)
k_inc_strided4(const SIn *__restrict__ in, SOut *__restrict__ out, int64_t O, int n, int64_t I,
               int k, int Lc, int nchunks)
{
    k_inc_strided4_body<M, SIn, SOut, KMAX>(in, out, O, n, I, k, Lc, nchunks, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// BDBS-Along-Dim along the contiguous dimension, on the flattened tensor.
//
// A warp owns a chunk of 128 consecutive elements of one "plane" (M1
// consecutive elements; planes hold whole rows of length n); lane l owns
// elements 4l .. 4l+3 of the chunk and the warp also stages the 32 elements
// after it (the halo: k-1 <= 31 more are needed).  Each output x sums its
// window s[x .. x+k) with the window cut at the end of its row, i.e. over
// j < min(k, n - pos(x)), which is the clipped box of Sec. 2; the sum is
// unrolled to KMAX >= k with per-term predicates (register-only, no dynamic
// indexing).  For the small k this pass uses, this costs KMAX operations per
// element, against three for a sequential BDBS-1D walk, but every load and
// store is a coalesced 16-byte access and no thread walks a row serially.
//
// The warps of a block walk the 32 planes of one dimension-1 segment
// (4 planes each) at the same chunk position.  With Rsum != nullptr each lane
// also adds its 4 input elements over those planes -- the whole segment into
// Rsum[s][c], the planes from offset r_tail on into Rtail[s][c] -- the
// segment totals the box-complement carries need.
// ---------------------------------------------------------------------------
template <class M, class SIn, class SOut, int KMAX>
__global__ void __launch_bounds__(256)
k_inc_flat(const SIn *__restrict__ in, SOut *__restrict__ out, int64_t N, int64_t n1, int64_t M1,
           int64_t n, int k, int64_t nq, typename M::car_t *__restrict__ Rsum,
           typename M::car_t *__restrict__ Rtail, int r_tail)
{
    using Lt = typename M::loc_t;
    using C = typename M::car_t;
    constexpr int SEG = 32, WARPS = 8, CH = 128, HALO = 32;
    __shared__ __align__(16) Lt buf[WARPS][CH + HALO];
    __shared__ Lt red_h[WARPS][CH], red_t[WARPS][CH];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t q = blockIdx.x % nq;          // chunk position in the plane
    const int64_t s = blockIdx.x / nq;          // dimension-1 segment
    const int64_t c0 = q * CH;                  // first column of the chunk
    const bool sums = Rsum != nullptr;
    Lt hs[4], ts[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) hs[i] = ts[i] = M::lid();
    // row position of this lane's first column (the same in every plane)
    const int64_t col = c0 + 4 * lane;
    const int pos0 = (int)(col % n);
    Lt *sb = buf[warp];
    const uint64_t pol_in = l2_policy_evict_first();   // the input is read once
    const uint64_t pol_out = l2_policy_evict_last();   // the next pass reads the output
    // Plane-invariant lane geometry: every plane but a partial last one (only
    // without segment totals, when planes pack whole rows) has the same extent.
    const int64_t full_c = M1 - c0;                      // chunk elements that exist
    const int valid_full = (int)max((int64_t)0, min((int64_t)4, full_c - 4 * lane));
    const bool halo_full = CH + lane < full_c;
    const bool aligned_stride = ((M1 * (int64_t)sizeof(SIn)) & 15) == 0 &&
                                ((M1 * (int64_t)sizeof(SOut)) & 15) == 0;
    const bool fast = (k == KMAX) && (pos0 + 3 + KMAX <= n);
    const SIn *src = in + (s * SEG + warp) * M1 + c0 + 4 * lane;
    SOut *dst = out + (s * SEG + warp) * M1 + c0 + 4 * lane;
    const int64_t step = (int64_t)WARPS * M1;
    const bool vin0 = aligned_stride && ((((uintptr_t)src) & (4 * sizeof(SIn) - 1)) == 0);
    const bool vout0 = aligned_stride && ((((uintptr_t)dst) & (4 * sizeof(SOut) - 1)) == 0);
    for (int u = warp; u < SEG; u += WARPS, src += step, dst += step) {
        const int64_t x1 = s * SEG + u;
        if (x1 >= n1) break;
        int valid = valid_full;
        bool halo = halo_full;
        if (x1 == n1 - 1) {
            // a partial last plane: clip the chunk at the end of the tensor
            const int64_t lim_c = min(full_c, N - (x1 * M1 + c0));
            valid = (int)max((int64_t)0, min((int64_t)4, lim_c - 4 * lane));
            halo = CH + lane < lim_c;
        }
        // stage the chunk and its halo (e past the plane or the tensor)
        Lt v[4];
        load4<M>(src, vin0 && valid == 4, valid, v, pol_in);
        // 16-byte (or 2 x 16-byte) shared stores: no bank conflicts
        if constexpr (sizeof(Lt) == 4) {
            float4 w;
            memcpy(&w, v, 16);
            *reinterpret_cast<float4 *>(sb + 4 * lane) = w;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) sb[4 * lane + i] = v[i];
        }
        // halo element CH + lane of the chunk (src points at element 4 * lane)
        sb[CH + lane] = halo ? M::lget(ld_hint(src + (CH - 3 * lane), pol_in)) : M::lid();
        __syncwarp();
        if (sums) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (u < r_tail)
                    hs[i] = M::lop(hs[i], v[i]);
                else
                    ts[i] = M::lop(ts[i], v[i]);
            }
        }
        // The lane's strip: its own 4 values, then KMAX-1 values of the lanes
        // after it (read as 16-byte vectors from 16-byte-aligned offsets).
        Lt st[4 + KMAX + 3];
#pragma unroll
        for (int i = 0; i < 4; ++i) st[i] = v[i];
        if constexpr (sizeof(Lt) == 4) {
#pragma unroll
            for (int j = 4; j < 4 + KMAX; j += 4) {
                if (4 * lane + j < CH + HALO) {
                    const float4 w = *reinterpret_cast<const float4 *>(sb + 4 * lane + j);
                    memcpy(st + j, &w, 16);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) st[j + i] = M::lid();
                }
            }
        } else {
#pragma unroll
            for (int j = 4; j < 4 + KMAX; ++j) st[j] = (4 * lane + j < CH + HALO) ? sb[4 * lane + j] : M::lid();
        }
        __syncwarp();
        Lt o[4];
        if (fast) {
            // All four windows are whole (no row end inside them): they share
            // st[3 .. KMAX-1]; windows i and i+1 differ by one element at each
            // end, so the four sums take about KMAX + 7 operations.
            Lt m = st[3];
#pragma unroll
            for (int j = 4; j < KMAX; ++j) m = M::lop(m, st[j]);
            const Lt a = M::lop(st[1], st[2]);
            const Lt b = M::lop(st[KMAX], st[KMAX + 1]);
            o[0] = M::lop(M::lop(st[0], a), m);
            o[1] = M::lop(M::lop(a, m), st[KMAX]);
            o[2] = M::lop(M::lop(st[2], m), b);
            o[3] = M::lop(M::lop(m, b), st[KMAX + 2]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int p = pos0 + i;
                while (p >= n) p -= (int)n;
                const int lim = min(k, (int)n - p);
                Lt acc = st[i];
#pragma unroll
                for (int j = 1; j < KMAX; ++j)
                    if (j < lim) acc = M::lop(acc, st[i + j]);
                o[i] = acc;
            }
        }
        if (valid > 0) store4<M>(dst, vout0 && valid == 4, valid, o, pol_out);
    }
    if (sums) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            red_h[warp][4 * lane + i] = hs[i];
            red_t[warp][4 * lane + i] = ts[i];
        }
        __syncthreads();
        if (threadIdx.x < CH) {
            const int64_t c = c0 + threadIdx.x;
            if (c < M1) {
                Lt h = M::lid(), t = M::lid();
#pragma unroll
                for (int w = 0; w < WARPS; ++w) {
                    h = M::lop(h, red_h[w][threadIdx.x]);
                    t = M::lop(t, red_t[w][threadIdx.x]);
                }
                Rsum[s * M1 + c] = M::template put<C>(M::op(M::widen(h), M::widen(t)));
                Rtail[s * M1 + c] = M::template put<C>(M::widen(t));
            }
        }
    }
}

}  // namespace exsum
