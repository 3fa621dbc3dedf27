// kernels_rows.cuh -- box-complement with the last (contiguous) dimension
// peeled first.
//
// For x = (x', x_d), x' = (x_1 .. x_{d-1}), the points outside the box of x
// split into two disjoint sets (Sec. 4, the regions of the excluded-sum
// components): those whose first d-1 coordinates already leave the box of
// x', and those inside it in x' that leave it along dimension d only.  So
//
//   out[x] = T[x'] (+) ( (+)_{y_d < x_d} H[x', y_d] ) (+) ( (+)_{y_d >= x_d + k_d} H[x', y_d] )
//
// with R[x'] = (+)_{y_d} X[x', y_d] (the row totals), T = excluded sum of R
// with box k_1 .. k_{d-1} (the same problem one dimension lower), and
// H = BDBS of X along dimensions 1 .. d-1.  The two kernels here are the row
// totals and the final pass: the window along dimension d-1 (optional), then
// the exclusive prefix and the shifted suffix of every row, plus T.
#pragma once

#include <type_traits>

#include "kernels_flat.cuh"

namespace exsum {

// Padded shared-memory row index: one spare slot per 32 elements, so that
// lanes reading strips of 2^j consecutive elements hit distinct banks.
__device__ __forceinline__ int rpad(int e) { return e + (e >> 5); }

// Swizzled tile index: the 16-byte chunks of a row are permuted within
// aligned groups of 8 chunks (chunk q -> q ^ ((q >> 3) & 7)), so that both a
// warp reading one column element per lane and lanes reading 16-byte
// vectors at a stride of 2 or 4 chunks hit distinct banks.  Rows are padded
// to whole groups.
template <class Lt>
__device__ __forceinline__ int tswz(int e)
{
    constexpr int CE = 16 / (int)sizeof(Lt);
    const int q = e / CE;
    return (q ^ ((q >> 3) & 7)) * CE + (e - q * CE);
}

__device__ __forceinline__ void cp_async16_hint(void *sdst, const void *gsrc, uint64_t pol)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(sdst);
    const size_t g = __cvta_generic_to_global(gsrc);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(s), "l"(g),
                 "l"(pol));
}

// The long part t and the local part y of an output, rounded to the output
// type.  For fp32 + (t a compensated pair) the low part is added to y first:
// two roundings instead of a full pair addition.
template <class M, class SOut>
__device__ __forceinline__ SOut finish(const typename M::acc_t &t, typename M::loc_t y)
{
    if constexpr (std::is_same<typename M::loc_t, float>::value &&
                  std::is_same<typename M::acc_t, f2>::value && std::is_same<SOut, float>::value)
        return __fadd_rn(t.hi, __fadd_rn(t.lo, y));
    else
        return M::template put<SOut>(M::op(t, M::widen(y)));
}

// ---------------------------------------------------------------------------
// Row totals R[r] = (+)_{c < L} X[r * L + c] (the dimension reduction along
// dimension d).  LPR (a power of two) lanes share a row: each adds its
// 4-element vectors in the local accumulator, then the lanes combine by a
// butterfly; the total is widened to the carry type.  Warps stride over the
// rows (a grid of a few blocks per SM).
// ---------------------------------------------------------------------------
template <class M, class SIn, int LPR>
__device__ __forceinline__ void k_row_totals_body(const SIn *__restrict__ X, typename M::car_t *__restrict__ R, int64_t rows, int L, int64_t vbid, int64_t vgrid)
{
    using Lt = typename M::loc_t;
    constexpr int RPW = 32 / LPR;
    constexpr int RU = 4;  // row groups in flight per warp
    const int lane = threadIdx.x & 31;
    const int sub = lane & (LPR - 1);
    const int64_t warp = ((int64_t)vbid * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)vgrid * blockDim.x) >> 5;
    const uint64_t pol = l2_policy_evict_last();  // the first pass reads X too
    constexpr size_t VALIGN = sizeof(SIn) * 4 >= 16 ? 16 : sizeof(SIn) * 4;
    const bool vec = (L % 4 == 0) && ((((uintptr_t)X) & (VALIGN - 1)) == 0);
    constexpr int SPAN = 4 * LPR;  // elements one pass over the lanes covers
    for (int64_t rb = warp * (RPW * RU); rb < rows; rb += nwarps * (RPW * RU)) {
        Lt acc[RU];
        const SIn *src[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            int64_t r = rb + u * RPW + lane / LPR;
            if (r >= rows) r = rows - 1;  // a valid row; its total is not stored
            acc[u] = M::lid();
            src[u] = X + r * (int64_t)L + 4 * sub;
        }
        int c = 4 * sub;
        // two vectors of every row per iteration, all loads issued first
        for (; c + SPAN < L; c += 2 * SPAN) {
            const bool f0 = vec, f1 = vec && c + SPAN + 4 <= L;
            const int v1 = min(4, L - c - SPAN);
            Lt w[RU][8];
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                load4<M>(src[u], f0, 4, w[u], pol);
                load4<M>(src[u] + SPAN, f1, v1, w[u] + 4, pol);
                src[u] += 2 * SPAN;
            }
#pragma unroll
            for (int u = 0; u < RU; ++u)
                acc[u] = M::lop(acc[u], M::lop(M::lop(M::lop(w[u][0], w[u][1]), M::lop(w[u][2], w[u][3])),
                                               M::lop(M::lop(w[u][4], w[u][5]), M::lop(w[u][6], w[u][7]))));
        }
        if (c < L) {
            const bool f0 = vec && c + 4 <= L;
            const int v0 = min(4, L - c);
            Lt w[RU][4];
#pragma unroll
            for (int u = 0; u < RU; ++u) load4<M>(src[u], f0, v0, w[u], pol);
#pragma unroll
            for (int u = 0; u < RU; ++u)
                acc[u] = M::lop(acc[u], M::lop(M::lop(w[u][0], w[u][1]), M::lop(w[u][2], w[u][3])));
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
#pragma unroll
            for (int m = LPR >> 1; m > 0; m >>= 1) acc[u] = M::lop(acc[u], shfl_xor(acc[u], m));
            const int64_t r = rb + u * RPW + lane / LPR;
            if (sub == 0 && r < rows) R[r] = M::template put<typename M::car_t>(M::widen(acc[u]));
        }
    }
}

template <class M, class SIn, int LPR>
__global__ void __launch_bounds__(256)
k_row_totals(const SIn *__restrict__ X, typename M::car_t *__restrict__ R, int64_t rows, int L)
{
    k_row_totals_body<M, SIn, LPR>(X, R, rows, L, blockIdx.x, gridDim.x);
}

// Suffix-buffer index: 4 spare slots per 32 elements, so that 16-byte
// accesses by lanes at a stride of 4, 8 or 16 elements hit distinct banks
// and 4-aligned groups stay contiguous.
__device__ __forceinline__ int spad(int e) { return e + 4 * (e >> 5); }

// In-place window sums down one shared-memory column: row r of `col` (rows
// LS apart) becomes the sum of rows r .. r+k-1, for r < nout, by the BDBS
// walk (blocks of k rows: suffixes of the current block plus prefixes of
// the next).  Rows up to nout + 2k - 2 must be readable, past the data
// holding the identity; a block is read before any of its rows is written.
template <class M, int KMAX>
__device__ __forceinline__ void smem_walk(typename M::loc_t *col, int LS, int k, int nout)
{
    using Lt = typename M::loc_t;
    Lt S[KMAX], v[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) v[j] = (j < k) ? col[j * LS] : M::lid();
    S[KMAX - 1] = v[KMAX - 1];
#pragma unroll
    for (int j = KMAX - 2; j >= 0; --j) S[j] = M::lop(v[j], S[j + 1]);
    Lt *p = col;
    for (int sb = 0; sb < nout; sb += k, p += k * LS) {
        p[0] = S[0];
        const Lt *q = p + k * LS;
        if (k == KMAX) {
#pragma unroll
            for (int j = 0; j < KMAX; ++j) v[j] = q[j * LS];
        } else {
#pragma unroll
            for (int j = 0; j < KMAX; ++j) v[j] = (j < k) ? q[j * LS] : M::lid();
        }
        Lt acc = M::lid();
        if (k == KMAX && sb + KMAX <= nout) {
#pragma unroll
            for (int j = 0; j + 1 < KMAX; ++j) {
                acc = M::lop(acc, v[j]);
                p[(j + 1) * LS] = M::lop(S[j + 1], acc);
            }
        } else {
#pragma unroll
            for (int j = 0; j + 1 < KMAX; ++j) {
                acc = M::lop(acc, v[j]);
                if (j + 1 < k && sb + 1 + j < nout) p[(j + 1) * LS] = M::lop(S[j + 1], acc);
            }
        }
        S[KMAX - 1] = v[KMAX - 1];
#pragma unroll
        for (int j = KMAX - 2; j >= 0; --j) S[j] = M::lop(v[j], S[j + 1]);
    }
}

// ---------------------------------------------------------------------------
// Final pass over the view [O, n2, L] of its input (n2 = n_{d-1}, L = n_d).
//
// A block takes GO consecutive slices o and a tile of TR consecutive rows x2
// of each, with all L columns, in a swizzled shared tile of RSA rows of LS
// elements per slice.  Staging: when the input has the local element type
// and 16-byte rows, the block copies rows x2 in [a, a + RS) with 16-byte
// asynchronous copies and sets the rows after them to the identity; with
// KMAX > 1 every thread then walks one column in place (smem_walk), leaving
// the window sums of width k2 along n2 in the first TR rows.  Otherwise the
// register BDBS walk (or a plain copy for KMAX == 1) reads global memory.
// Columns L .. round_up(L, EPL) - 1 of the tile hold the identity.
//
// Phase 2: `lpr` lanes take one row, lane s the strip of EPL elements from
// s * EPL.  A segmented scan of the strip totals gives each lane the
// exclusive prefix before its strip and the suffix after it; the inclusive
// suffixes go to a per-row shared buffer so that a lane can read the suffix
// at x_d + k3, which another lane owns (16-byte accesses when k3 and L are
// multiples of 4 and the element is 4 bytes; slot L holds the identity for
// the scalar reads).  Each output is T[row] (+) prefix (+) suffix.
// ---------------------------------------------------------------------------
template <class M, class SIn, class SOut, int KMAX, int EPL>
__device__ __forceinline__ void k_rowx_body(const SIn *__restrict__ in, const typename M::car_t *__restrict__ T,
       const typename M::car_t *__restrict__ R1, int k1, SOut *__restrict__ out, int64_t O, int n2,
       int L, int k2, int k3, int TR, int GO, int ntile, int RS, int RSA, int LS, int lpr, int64_t vbid, int64_t vgrid)
{
    using Lt = typename M::loc_t;
    using A = typename M::acc_t;
    constexpr int CE = 16 / (int)sizeof(Lt);
    extern __shared__ __align__(128) unsigned char rowx_smem[];
    Lt *tile = reinterpret_cast<Lt *>(rowx_smem);
    const int L32 = (L + 31) & ~31;
    const int LPs = L32 + 4 * (L32 >> 5) + 4;
    const int rpw = 32 / lpr;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t og = vbid / ntile;
    const int a = (int)(vbid - og * ntile) * TR;
    const int64_t o0 = og * GO;
    const int ng = (int)min((int64_t)GO, O - o0);  // slices in this block
    const int rend = min(a + TR, n2);
    const int nout = rend - a;
    const int nst = min(RS, n2 - a);  // rows staged per slice
    const uint64_t pol_in = l2_policy_evict_first();
    const uint64_t pol_out = l2_policy_evict_first();
    Lt *sbuf = tile + (int64_t)GO * RSA * LS;
    using C = typename M::car_t;
    C *Tt = reinterpret_cast<C *>(
        rowx_smem + (((int64_t)GO * RSA * LS + (int64_t)(blockDim.x >> 5) * rpw * LPs) * sizeof(Lt) + 15) / 16 * 16);

    // identity: strip padding of the output rows, slot L of every suffix row
    const int LE = (L + EPL - 1) / EPL * EPL;
    if (LE > L) {
        const int padw = LE - L;
        for (int i = threadIdx.x; i < ng * TR * padw; i += blockDim.x) {
            const int rr = i / padw;
            const int g = rr / TR;
            tile[((int64_t)g * RSA + (rr - g * TR)) * LS + tswz<Lt>(L + (i - rr * padw))] = M::lid();
        }
    }
    for (int i = threadIdx.x; i < (int)(blockDim.x >> 5) * rpw; i += blockDim.x)
        sbuf[(int64_t)i * LPs + spad(L)] = M::lid();

    bool staged = false;
    if constexpr (std::is_same<SIn, Lt>::value) {
        staged = (L % CE == 0) && ((((uintptr_t)in) & 15) == 0);
        if (staged) {
            // thread -> (chunk tq, first row tr0); rows advance by rpp
            const int cpr = L / CE;
            const int rpp = (int)blockDim.x / cpr;
            const int tq = (int)threadIdx.x % cpr, tr0 = (int)threadIdx.x / cpr;
            if (tr0 < rpp) {
                const int sw = tswz<Lt>(tq * CE);
                for (int g = 0; g < ng; ++g) {
                    const SIn *src = in + ((o0 + g) * n2 + a) * (int64_t)L + tq * CE;
                    Lt *dst = tile + (int64_t)g * RSA * LS + sw;
                    int r = tr0;
                    for (; r < nst; r += rpp) cp_async16_hint(dst + r * LS, src + (int64_t)r * L, pol_in);
                    if constexpr (KMAX > 1) {
                        uint4 idv;
                        {
                            Lt idl[CE];
#pragma unroll
                            for (int m = 0; m < CE; ++m) idl[m] = M::lid();
                            memcpy(&idv, idl, 16);
                        }
                        for (; r < RSA; r += rpp) *reinterpret_cast<uint4 *>(dst + r * LS) = idv;
                    }
                }
            }
            cp_async_wait_all();
        }
    }
    // T of the tile's rows, into shared memory while the tile is in flight.
    // One-dimensional tail (d == 2, R1 != nullptr): T[x] is the excluded sum
    // of the row totals R1 with box k1 (k1 <= 64), from the totals before the
    // tile (P0), those from the last row's box end on (S0), and the at most
    // nout + k1 - 1 in between, staged in Tt first.
    if (!R1) {
        for (int i = threadIdx.x; i < ng * nout; i += blockDim.x) {
            const int g = i / nout;
            const int r = i - g * nout;
            Tt[g * TR + r] = T[(o0 + g) * n2 + a + r];
        }
    } else if (warp == 0) {
        const int B1 = min(n2, a + nout - 1 + k1);
        A p0 = M::id(), s0 = M::id();
        for (int y = lane; y < a; y += 32) p0 = M::op(p0, M::get(R1[y]));
        for (int y = B1 + lane; y < n2; y += 32) s0 = M::op(s0, M::get(R1[y]));
        for (int y = a + lane; y < B1; y += 32) Tt[TR + (y - a)] = R1[y];
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
            p0 = M::op(p0, shfl_xor(p0, m));
            s0 = M::op(s0, shfl_xor(s0, m));
        }
        __syncwarp();
        for (int r = lane; r < nout; r += 32) {
            A pre = p0, suf = s0;
            for (int y = 0; y < r; ++y) pre = M::op(pre, M::get(Tt[TR + y]));
            for (int y = r + k1; y < B1 - a; ++y) suf = M::op(suf, M::get(Tt[TR + y]));
            Tt[r] = M::template put<C>(M::op(pre, suf));
        }
    }
    if (!staged) {
        for (int i = threadIdx.x; i < ng * L; i += blockDim.x) {
            const int g = i / L;
            const int c = i - g * L;
            Lt *col = tile + (int64_t)g * RSA * LS + tswz<Lt>(c);
            const SIn *src = in + (o0 + g) * n2 * (int64_t)L + c;
            if constexpr (KMAX == 1) {
                int x = a;
                for (; x + 3 < rend; x += 4) {
                    const SIn v0 = ld_hint(src + (int64_t)x * L, pol_in);
                    const SIn v1 = ld_hint(src + (int64_t)(x + 1) * L, pol_in);
                    const SIn v2 = ld_hint(src + (int64_t)(x + 2) * L, pol_in);
                    const SIn v3 = ld_hint(src + (int64_t)(x + 3) * L, pol_in);
                    col[(x - a) * LS] = M::lget(v0);
                    col[(x + 1 - a) * LS] = M::lget(v1);
                    col[(x + 2 - a) * LS] = M::lget(v2);
                    col[(x + 3 - a) * LS] = M::lget(v3);
                }
                for (; x < rend; ++x) col[(x - a) * LS] = M::lget(ld_hint(src + (int64_t)x * L, pol_in));
            } else {
                bdbs_walk<M, KMAX>(
                    k2, a, rend,
                    [&](int x) { return x < n2 ? M::lget(ld_hint(src + (int64_t)x * L, pol_in)) : M::lid(); },
                    [&](int x, Lt v) { col[(x - a) * LS] = v; });
            }
        }
    }
    __syncthreads();
    if constexpr (KMAX > 1) {
        if (staged) {
            for (int i = threadIdx.x; i < ng * L; i += blockDim.x) {
                const int g = i / L;
                const int c = i - g * L;
                smem_walk<M, KMAX>(tile + (int64_t)g * RSA * LS + tswz<Lt>(c), LS, k2, nout);
            }
            __syncthreads();
        }
    }

    // Phase 2: rpw rows per warp at a time, lpr lanes per row.  Per-lane
    // offsets do not depend on the row.
    const int sub = lane & (lpr - 1);
    const int rw = lane / lpr;
    Lt *sb = sbuf + (int64_t)(warp * rpw + rw) * LPs;
    const int e0 = sub * EPL;
    const bool has = e0 < L;
    int toff[EPL / 4];
#pragma unroll
    for (int i = 0; i < EPL / 4; ++i) toff[i] = tswz<Lt>(e0 + 4 * i);
    const int sbase = spad(e0);  // strips never cross a 32-element group
    const bool vsb = sizeof(Lt) == 4 && (k3 % 4 == 0) && (L % 4 == 0);
    bool vout = false;
    if constexpr (sizeof(SOut) == 4 || sizeof(SOut) == 8)
        vout = (e0 + EPL <= L) && (L % 4 == 0) && ((((uintptr_t)out) & 15) == 0);
    const int wstride = (int)(blockDim.x >> 5) * rpw;
    for (int g = 0; g < ng; ++g) {
        const int64_t rowbase = (o0 + g) * n2 + a;
        const Lt *tg = tile + (int64_t)g * RSA * LS;
        for (int rb = warp * rpw; rb < nout; rb += wstride) {
            const int r = rb + rw;
            const bool live = has && r < nout;
            const Lt *row = tg + r * LS;
            Lt v[EPL];
            Lt t = M::lid();
            if (live) {
#pragma unroll
                for (int i = 0; i < EPL / 4; ++i) {
                    if constexpr (sizeof(Lt) == 4) {
                        const uint4 w = *reinterpret_cast<const uint4 *>(row + toff[i]);
                        memcpy(v + 4 * i, &w, 16);
                    } else {
                        const uint4 w0 = *reinterpret_cast<const uint4 *>(row + toff[i]);
                        const uint4 w1 = *reinterpret_cast<const uint4 *>(row + (toff[i] ^ 2));
                        memcpy(v + 4 * i, &w0, 16);
                        memcpy(v + 4 * i + 2, &w1, 16);
                    }
                }
#pragma unroll
                for (int j = 0; j < EPL; ++j) t = M::lop(t, v[j]);
            }
            // segmented inclusive scans of the strip totals, forwards and
            // backwards: full-warp shuffles, the lane tests keep each scan
            // inside its lpr-lane segment
            Lt pre = t, suf = t;
#pragma unroll
            for (int lv = 0; lv < 5; ++lv) {
                const int dl = 1 << lv;
                if (dl < lpr) {
                    const Lt u = shfl_up(pre, dl);
                    const Lt w = shfl_down(suf, dl);
                    if (sub >= dl) pre = M::lop(u, pre);
                    if (sub + dl < lpr) suf = M::lop(suf, w);
                }
            }
            Lt p = shfl_up(pre, 1);
            Lt s = shfl_down(suf, 1);
            if (sub == 0) p = M::lid();
            if (sub == lpr - 1) s = M::lid();
            if (live) {
                if constexpr (sizeof(Lt) == 4) {
                    if (vsb) {
#pragma unroll
                        for (int i = EPL / 4 - 1; i >= 0; --i) {
                            Lt w4[4];
#pragma unroll
                            for (int m = 3; m >= 0; --m) {
                                s = M::lop(v[4 * i + m], s);
                                w4[m] = s;
                            }
                            uint4 w;
                            memcpy(&w, w4, 16);
                            *reinterpret_cast<uint4 *>(sb + sbase + 4 * i) = w;
                        }
                    }
                }
                if (!vsb) {
#pragma unroll
                    for (int j = EPL - 1; j >= 0; --j) {
                        s = M::lop(v[j], s);
                        sb[sbase + j] = s;
                    }
                }
            }
            __syncwarp();
            if (live) {
                const A tv = M::get(Tt[g * TR + r]);
                SOut *dst = out + (rowbase + r) * (int64_t)L + e0;
                SOut res[EPL];
                bool done = false;
                if constexpr (sizeof(Lt) == 4) {
                    if (vsb) {
#pragma unroll
                        for (int i = 0; i < EPL / 4; ++i) {
                            const int js = e0 + 4 * i + k3;
                            Lt sv[4];
                            if (js < L) {
                                const uint4 w = *reinterpret_cast<const uint4 *>(sb + spad(js));
                                memcpy(sv, &w, 16);
                            } else {
#pragma unroll
                                for (int m = 0; m < 4; ++m) sv[m] = M::lid();
                            }
#pragma unroll
                            for (int m = 0; m < 4; ++m) {
                                res[4 * i + m] = finish<M, SOut>(tv, M::lop(p, sv[m]));
                                p = M::lop(p, v[4 * i + m]);
                            }
                        }
                        done = true;
                    }
                }
                if (!done) {
#pragma unroll
                    for (int j = 0; j < EPL; ++j) {
                        const int js = min(e0 + j + k3, L);
                        res[j] = finish<M, SOut>(tv, M::lop(p, sb[spad(js)]));
                        p = M::lop(p, v[j]);
                    }
                }
                if (vout) {
                    if constexpr (sizeof(SOut) == 4) {
#pragma unroll
                        for (int j = 0; j < EPL; j += 4) {
                            uint4 w;
                            memcpy(&w, res + j, 16);
                            st_hint_v4(dst + j, w, pol_out);
                        }
                    } else if constexpr (sizeof(SOut) == 8) {
#pragma unroll
                        for (int j = 0; j < EPL; j += 2) {
                            uint4 w;
                            memcpy(&w, res + j, 16);
                            st_hint_v4(dst + j, w, pol_out);
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < EPL; ++j)
                        if (e0 + j < L) st_hint(dst + j, res[j], pol_out);
                }
            }
            __syncwarp();
        }
    }
}

template <class M, class SIn, class SOut, int KMAX, int EPL>
__global__ void __launch_bounds__(256)
k_rowx(const SIn *__restrict__ in, const typename M::car_t *__restrict__ T,
       const typename M::car_t *__restrict__ R1, int k1, SOut *__restrict__ out, int64_t O, int n2,
       int L, int k2, int k3, int TR, int GO, int ntile, int RS, int RSA, int LS, int lpr)
{
    k_rowx_body<M, SIn, SOut, KMAX, EPL>(in, T, R1, k1, out, O, n2, L, k2, k3, TR, GO, ntile, RS, RSA, LS, lpr, blockIdx.x, gridDim.x);
}

}  // namespace exsum
